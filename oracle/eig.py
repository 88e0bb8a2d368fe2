"""Generalized eigensolve and occupations (oracle, test infrastructure).

Sec. 4: solve H c = eps S c for the lowest states (eq. Hc).  Small problems use
LAPACK's dense symmetric-definite driver through SciPy (the paper notes dense
methods suffice for small problems); large ones use SciPy's sparse
shift-invert Lanczos.  Occupations: 0 <= f <= 2 (Sec. 3, eq. rhoe), filled by
Fermi-Dirac smearing at temperature kT with the chemical potential found by
bisection on sum f = N_e.

Pins: library routines (LAPACK, ARPACK); the spectra they return are pinned
through the closed-form empty-lattice and harmonic-oscillator tests.
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
