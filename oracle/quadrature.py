"""Element quadrature rules (oracle, test infrastructure).

Sec. 5.2 of the paper builds one quadrature rule per element and uses it for
every integral (matrix elements, norms, energies) in every SCF iteration.
The rule is driven by the two most rapidly varying integrands that appear in
H and S: Psi_alpha^2 and grad Psi_alpha . grad Psi_alpha, for each
enrichment alpha that appears in the element's basis.

Three modes:
* FIXED: p_near^3 Gauss on elements that some atom image reaches within r_c,
  p_far^3 elsewhere.
* PADAPT (a p-adaptive reading of the paper's tolerance test): the smallest
  p in [p_min, p_max] with |I_p - I_{p+2}| < tol for every integrand; p_max
  if none passes.  Elements without enrichment take p_min.
* HADAPT (the paper's scheme): test 5^3 against the 8^3 reference on the
  cell; integrands whose absolute error is >= tol are passed down, the cell is
  split into 8 equal children and the test repeats on each child with only
  those integrands.  A cell that passes (or sits at max_depth) keeps the 8^3
  rule (the paper does not say which of the two rules is kept; the more
  accurate one is used).  Elements without enrichment take p_far^3.

Point order: tensor rules run x fastest (gauss_box); children are visited
depth first in the order a + 2 b + 4 c of their (a, b, c) offsets.

Pins (tests/test_oracle_quadrature.py): Gauss exactness on polynomials; the
rule's integral of Psi^2 against a brute-force 30^3-per-octant rule on one
element; weights sum to the element volume.
"""
from __future__ import annotations

import numpy as np

from .enrich import enrichment
from .fe import gauss_box

FIXED, PADAPT, HADAPT = 0, 1, 2


def _integrals(mesh, alphas, lo, hi, p):
    """I(Psi^2) and I(|grad Psi|^2) on box [lo, hi] with p^3 Gauss, per alpha."""
    pts, wts = gauss_box(p, lo, hi)
    out = []
    for k in alphas:
        al = mesh.alphas[k]
        psi, g = enrichment(al["orb"], al["rc"], al["tau"], mesh.a, pts)
        out.append((float(wts @ (psi * psi)), float(wts @ (g * g).sum(axis=0))))
    return np.array(out).reshape(-1, 2)


def _hadapt(mesh, alphas, lo, hi, depth, q):
    tol = q["tol"]
    i5 = _integrals(mesh, alphas, lo, hi, 5)
    i8 = _integrals(mesh, alphas, lo, hi, 8)
    err = np.abs(i5 - i8)
    failing = [k for k, row in zip(alphas, err) if (row >= tol).any()]
    if not failing or depth >= q["max_depth"]:
        return [gauss_box(8, lo, hi)]
    mid = (lo + hi) / 2.0
    parts = []
    for c in range(2):
        for b in range(2):
            for a in range(2):
                off = np.array([a, b, c])
                clo = np.where(off == 0, lo, mid)
                chi = np.where(off == 0, mid, hi)
                parts += _hadapt(mesh, failing, clo, chi, depth + 1, q)
    return parts


def element_rule(mesh, e):
    """Quadrature rule of element e: physical points (Q,3) and weights (Q,)."""
    q = mesh.wl["quad"]
    lo, hi = mesh.elem_box(e)
    mode = q["mode"]
    if mode == FIXED:
        p = q["p_near"] if mesh.near[e].any() else q["p_far"]
        return gauss_box(p, lo, hi)
    alphas = mesh.elem_alphas(e)
    if mode == PADAPT:
        if not alphas:
            return gauss_box(q["p_min"], lo, hi)
        for p in range(q["p_min"], q["p_max"] + 1):
            err = np.abs(_integrals(mesh, alphas, lo, hi, p)
                         - _integrals(mesh, alphas, lo, hi, p + 2))
            if (err < q["tol"]).all():
                return gauss_box(p, lo, hi)
        return gauss_box(q["p_max"], lo, hi)
    if mode == HADAPT:
        if not alphas:
            return gauss_box(q["p_far"], lo, hi)
        parts = _hadapt(mesh, alphas, lo, hi, 0, q)
        return (np.concatenate([p for p, _ in parts]),
                np.concatenate([w for _, w in parts]))
    raise ValueError(mode)


def all_rules(mesh):
    """Rules of all elements: (points (sumQ,3), weights (sumQ,), offsets (nelem+1,))."""
    pts, wts, off = [], [], [0]
    for e in range(mesh.nelem):
        p, w = element_rule(mesh, e)
        pts.append(p)
        wts.append(w)
        off.append(off[-1] + len(w))
    return np.concatenate(pts), np.concatenate(wts), np.array(off, dtype=np.int64)
