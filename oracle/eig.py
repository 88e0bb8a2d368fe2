"""Generalized eigensolve and occupations (oracle, test infrastructure).

Sec. 4: solve H c = eps S c for the lowest states (eq. Hc).  Small problems use
LAPACK's dense symmetric-definite driver through SciPy (the paper notes dense
methods suffice for small problems); large ones use SciPy's sparse
shift-invert Lanczos.  Occupations: 0 <= f <= 2 (Sec. 3, eq. rhoe), filled by
Fermi-Dirac smearing at temperature kT with the chemical potential found by
bisection on sum f = N_e.

Large cells (the 12^3 rocksalt cell has N = 51,576) factorise H - sigma S
with SuperLU on a nested-dissection order of the DOFs (SuperLU's own column
orderings fill in far more on this periodic 3D pattern).

Pins: library routines (LAPACK, ARPACK); the spectra they return are pinned
through the closed-form empty-lattice and harmonic-oscillator tests; the
nested-dissection shift-invert path and the Rayleigh-Ritz step against the
dense LAPACK eigensolve (tests/test_oracle_misc.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def lowest_eigs(H, S, k, sigma=None):
    """Lowest k eigenpairs (eps (k,), C (N, k)) of H c = eps S c."""
    N = H.shape[0]
    if N <= 6000 or sigma is None:
        Hd = H.toarray() if sp.issparse(H) else np.asarray(H)
        Sd = S.toarray() if sp.issparse(S) else np.asarray(S)
        w, v = sla.eigh(Hd, Sd, subset_by_index=[0, k - 1])
        return w, v
    w, v = spla.eigsh(H.tocsc(), k=k, M=S.tocsc(), sigma=sigma, which="LM")
    order = np.argsort(w)
    return w[order], v[:, order]


def fermi_occupations(eps, nelec, kT):
    """f_k = 2 / (1 + exp((eps_k - mu)/kT)) with sum f = nelec (bisection on mu)."""
    eps = np.asarray(eps, dtype=np.float64)

    def total(mu):
        x = np.clip((eps - mu) / kT, -700.0, 700.0)
        return (2.0 / (1.0 + np.exp(x))).sum()

    lo, hi = eps.min() - 50.0 * kT - 1.0, eps.max() + 50.0 * kT + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < nelec:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    x = np.clip((eps - mu) / kT, -700.0, 700.0)
    return 2.0 / (1.0 + np.exp(x)), mu


def fermi_occupations_k(eps, wk, nelec, kT):
    """Occupations of the states of several k-points with one Fermi level:
    f_nk = 2 / (1 + exp((eps_nk - mu)/kT)) with sum_k w_k sum_n f_nk = nelec
    (bisection on mu).  eps: a list of 1-D arrays, one per k-point (their
    lengths may differ); wk: the k-point weights.  Returns (list of f, mu)."""
    eps = [np.asarray(e, dtype=np.float64) for e in eps]
    wk = np.asarray(wk, dtype=np.float64)

    def occ(e, mu):
        x = np.clip((e - mu) / kT, -700.0, 700.0)
        return 2.0 / (1.0 + np.exp(x))

    def total(mu):
        return sum(w * occ(e, mu).sum() for w, e in zip(wk, eps))

    allv = np.concatenate(eps)
    lo, hi = allv.min() - 50.0 * kT - 1.0, allv.max() + 50.0 * kT + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < nelec:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    return [occ(e, mu) for e in eps], mu


def nested_dissection_order(coords, period):
    """A fill-reducing DOF order for the sparse shift-invert factorisation.

    coords (N, 3): integer positions of the DOFs on the periodic node grid of
    `period` points per axis (an enrichment DOF sits at its PU vertex, which
    couples like a vertex node).  The grid is cut recursively at vertex planes
    (multiples of 3, where neighbouring elements meet), the ring of each
    periodic axis at two planes; each separator is numbered after the two
    parts it separates.  A permutation only: the factorised matrix is the
    same, so the eigenpairs do not depend on it.
    """
    X = np.asarray(coords)
    out = []

    def rec(idx, lo, hi, periodic):
        ext = [hi[d] - lo[d] for d in range(3)]
        d = int(np.argmax(ext))
        mid = lo[d] + 3 * ((ext[d] // 3) // 2)
        if len(idx) < 300 or mid == lo[d]:
            out.append(idx)
            return
        x = X[idx, d]
        lo2, hi1 = list(lo), list(hi)
        hi1[d] = mid
        lo2[d] = mid
        per = list(periodic)
        if periodic[d]:
            sep = idx[(x == lo[d]) | (x == mid)]
            left, right = idx[(x > lo[d]) & (x < mid)], idx[x > mid]
            per[d] = False
        else:
            sep = idx[x == mid]
            left, right = idx[x < mid], idx[x > mid]
        rec(left, lo, hi1, per)
        rec(right, lo2, hi, per)
        out.append(sep)

    rec(np.arange(len(X)), [0, 0, 0], [period] * 3, [True, True, True])
    perm = np.concatenate(out)
    assert len(perm) == len(X) and len(np.unique(perm)) == len(X)
    return perm


def lowest_eigs_shift_invert(H, S, k, sigma, perm):
    """Lowest k eigenpairs of H c = eps S c by shift-invert Lanczos (ARPACK),
    (H - sigma S)^-1 applied through SuperLU on the rows and columns in the
    order `perm` (no further reordering, no pivoting: sigma below the
    spectrum keeps H - sigma S positive definite)."""
    A = (H - sigma * S).tocsr()[perm][:, perm].tocsc()
    lu = spla.splu(A, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    inv = np.argsort(perm)
    op = spla.LinearOperator(A.shape, matvec=lambda x: lu.solve(x[perm])[inv], dtype=np.float64)
    w, v = spla.eigsh(H.tocsc(), k=k, M=S.tocsc(), sigma=sigma, which="LM", OPinv=op)
    order = np.argsort(w)
    return w[order], v[:, order]


def rayleigh_ritz(H, S, X):
    """Eigenvalues of the pencil (H, S) restricted to span(X) (N x k): exact
    to second order in the distance of span(X) from an invariant subspace."""
    return sla.eigh(X.T @ (H @ X), X.T @ (S @ X), eigvals_only=True)
