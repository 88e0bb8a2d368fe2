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

General (triclinic) cells: the same rules on the reference cube, mapped by
the element's affine map (weights times |det J|); children are halves of the
reference cube along each axis.

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


def _box_rule(mesh, e):
    """p^3 Gauss rule of a sub-box [lo, hi] of element e: physical boxes for
    cubic cells; for general cells boxes of the reference cube, mapped by the
    element's affine map (weights times |det J|)."""
    if not mesh.general:
        return gauss_box
    x0 = mesh.elem_origin(e)

    def rule(p, lo, hi):
        r, w = gauss_box(p, lo, hi)
        return x0 + (r + 1.0) @ mesh.J.T, w * mesh.detJ
    return rule


def _integrals(mesh, alphas, lo, hi, p, box=gauss_box):
    """I(Psi^2) and I(|grad Psi|^2) on box [lo, hi] with p^3 Gauss, per alpha."""
    pts, wts = box(p, lo, hi)
    out = []
    for k in alphas:
        al = mesh.alphas[k]
        psi, g = enrichment(al["orb"], al["rc"], al["tau"], mesh.lattice, pts)
        out.append((float(wts @ (psi * psi)), float(wts @ (g * g).sum(axis=0))))
    return np.array(out).reshape(-1, 2)


def _hadapt(mesh, alphas, lo, hi, depth, q, box=gauss_box):
    tol = q["tol"]
    i5 = _integrals(mesh, alphas, lo, hi, 5, box)
    i8 = _integrals(mesh, alphas, lo, hi, 8, box)
    err = np.abs(i5 - i8)
    failing = [k for k, row in zip(alphas, err) if (row >= tol).any()]
    if not failing or depth >= q["max_depth"]:
        return [box(8, lo, hi)]
    mid = (lo + hi) / 2.0
    parts = []
    for c in range(2):
        for b in range(2):
            for a in range(2):
                off = np.array([a, b, c])
                clo = np.where(off == 0, lo, mid)
                chi = np.where(off == 0, mid, hi)
                parts += _hadapt(mesh, failing, clo, chi, depth + 1, q, box)
    return parts


def element_rule(mesh, e):
    """Quadrature rule of element e: physical points (Q,3) and weights (Q,)."""
    q = mesh.wl["quad"]
    box = _box_rule(mesh, e)
    if mesh.general:
        lo, hi = -np.ones(3), np.ones(3)
    else:
        lo, hi = mesh.elem_box(e)
    mode = q["mode"]
    if mode == FIXED:
        p = q["p_near"] if mesh.near[e].any() else q["p_far"]
        return box(p, lo, hi)
    alphas = mesh.elem_alphas(e)
    if mode == PADAPT:
        if not alphas:
            return box(q["p_min"], lo, hi)
        for p in range(q["p_min"], q["p_max"] + 1):
            err = np.abs(_integrals(mesh, alphas, lo, hi, p, box)
                         - _integrals(mesh, alphas, lo, hi, p + 2, box))
            if (err < q["tol"]).all():
                return box(p, lo, hi)
        return box(q["p_max"], lo, hi)
    if mode == HADAPT:
        if not alphas:
            return box(q["p_far"], lo, hi)
        parts = _hadapt(mesh, alphas, lo, hi, 0, q, box)
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
