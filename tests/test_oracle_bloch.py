"""Pins of the Bloch (k != 0) oracle (oracle/bloch.py)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble as oasm, bloch as ob, mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import workloads as W

K_FRAC = np.array([0.3, -0.2, 0.1])


def _empty_lowest(nel, a=4.0):
    wl = W.empty_lattice(nel=nel, a=a, p=4)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    k = 2.0 * math.pi / a * K_FRAC
    H, S = ob.assemble_HS_k(m, rules, np.zeros(len(rules[1])), k)
    w = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True, subset_by_index=[0, 3])
    G = 2.0 * math.pi / a * np.array([[0, 0, 0], [-1, 0, 0], [0, 1, 0], [0, 0, -1],
                                      [1, 0, 0], [0, -1, 0], [0, 0, 1]], dtype=np.float64)
    exact = np.sort(0.5 * ((G + k) ** 2).sum(axis=1))[:4]
    return w, exact


def test_empty_lattice_spectrum_at_k():
    w3, ex = _empty_lowest(3)
    w4, _ = _empty_lowest(4)
    assert np.all(w4 >= ex - 1e-12)          # variational: from above
    e3, e4 = w3[0] - ex[0], w4[0] - ex[0]
    assert e4 < 1e-4 * ex[1]
    rate = math.log(e3 / e4) / math.log(4.0 / 3.0)
    assert rate > 5.0                         # O(h^6) for eigenvalues (tricubic)


@pytest.fixture(scope="module")
def cell():
    wl = W.small_two_atom(nel=2, quad_p=4)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    V = W.random_potential(len(rules[1]), seed=1)
    return wl, m, rules, V


def test_hermitian_periodic_in_k_and_gamma_limit(cell):
    wl, m, rules, V = cell
    k = 2.0 * math.pi / wl["a"] * K_FRAC
    H, S = ob.assemble_HS_k(m, rules, V, k)
    assert abs(H - H.conj().T).max() < 1e-13 * abs(H).max()
    assert abs(S - S.conj().T).max() < 1e-13 * abs(S).max()
    G = 2.0 * math.pi / wl["a"] * np.array([1.0, 0.0, -2.0])
    H2, S2 = ob.assemble_HS_k(m, rules, V, k + G)
    assert abs(H2 - H).max() < 1e-12 * abs(H).max()
    H0, S0 = ob.assemble_HS_k(m, rules, V, np.zeros(3))
    Hr, Sr = oasm.assemble_HS(m, rules, V)
    assert abs(H0 - Hr).max() < 1e-13 * abs(Hr).max() and abs(S0 - Sr).max() < 1e-13


def test_density_identity_at_k(cell):
    wl, m, rules, V = cell
    k = 2.0 * math.pi / wl["a"] * K_FRAC
    _, S = ob.assemble_HS_k(m, rules, V, k)
    rng = np.random.default_rng(4)
    C = rng.standard_normal((m.n_dof, 3)) + 1j * rng.standard_normal((m.n_dof, 3))
    f = np.array([2.0, 1.5, 0.3])
    n = ob.density_k(m, rules, C, f, k)
    want = sum(f[i] * np.real(np.conj(C[:, i]) @ (S @ C[:, i])) for i in range(3))
    assert abs(rules[1] @ n - want) < 1e-10 * abs(want)


def test_adjoint_at_k_is_the_derivative(cell):
    wl, m, rules, V = cell
    k = 2.0 * math.pi / wl["a"] * K_FRAC
    H, _ = ob.assemble_HS_k(m, rules, V, k)
    rng = np.random.default_rng(5)
    Hbar = H.copy()
    Hbar.data = rng.standard_normal(H.nnz) + 1j * rng.standard_normal(H.nnz)
    g = ob.adjoint_V_k(m, rules, Hbar, k)
    dV = rng.standard_normal(len(V))
    H2, _ = ob.assemble_HS_k(m, rules, V + dV, k)
    # H is linear in V: L(V + dV) - L(V) = g . dV exactly
    D = (H2 - H).tocsr()
    L = np.real((Hbar.conj().multiply(D)).sum())
    assert abs(L - g @ dV) < 1e-10 * max(1.0, abs(L))


# --- supercell folding ----------------------------------------------------------
# A 2x2x2 supercell at wavevector k_s has, in exact arithmetic, the union of
# the cell's spectra at the eight folded wavevectors k_s + (pi / a) m,
# m in {0, 1}^3 (the supercell's reciprocal lattice folds the cell's
# Brillouin zone eight times), provided both bases span the same Bloch
# space: the same per-cube mesh and rule, and every enrichment seen through
# one atom image only.  With the atom on a vertex, r_e below h and
# r_c < a - sqrt(3) h (here 1 < 8 - 6.93), the support of an enriched PU
# function meets no second image's cutoff sphere, so the cell's phi_v Psi_a
# and the supercell's phi_v' Psi_(a, m) are the same function.  The 8^3 rule
# puts enough points inside each small cutoff sphere for S to be definite.
FOLD_A, FOLD_NEL = 8.0, 2


def _fold_cell(rep):
    a = FOLD_A * rep
    sp = [W._species(W.H_LIKE_1S, 1.0, 0.5), W._species(W.LI_LIKE_1S2S2P, 1.0, 0.5)]
    base = [(0, np.array([0.0, 0.0, 0.0])), (1, np.array([4.0, 0.0, 4.0]))]
    atoms = []
    for s, tau in base:
        for mz in range(rep):
            for my in range(rep):
                for mx in range(rep):
                    atoms.append((s, tuple(tau + FOLD_A * np.array([mx, my, mz]))))
    return dict(name=f"fold_{rep}", a=a, nel=FOLD_NEL * rep, species=sp, atoms=atoms,
                quad=dict(mode=W.QUAD_FIXED, p_far=8, p_near=8, p_min=0, p_max=0,
                          tol=1e-6, max_depth=0), nocc=1, nelec=2.0)


def _fold_potential(x):
    """A smooth potential with the cell's period and no mirror symmetry."""
    t = 2.0 * math.pi / FOLD_A
    return (-0.4 * np.cos(t * x[:, 0]) - 0.3 * np.cos(t * x[:, 1])
            - 0.2 * np.cos(t * (x[:, 2] + x[:, 0])) + 0.15 * np.sin(t * (x[:, 0] - 2 * x[:, 1]))
            + 0.1 * np.sin(t * x[:, 2]))


def _spectrum(wl, k, nlow):
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    H, S = ob.assemble_HS_k(m, rules, _fold_potential(rules[0]), k)
    return sla.eigh(H.toarray(), S.toarray(), eigvals_only=True, subset_by_index=[0, nlow - 1])


def _folding_gap(nlow=12):
    ks = math.pi / FOLD_A * np.array([0.3, -0.2, 0.1])   # supercell wavevector
    sup = _spectrum(_fold_cell(2), ks, nlow)
    prim = []
    for m in np.ndindex(2, 2, 2):
        prim.append(_spectrum(_fold_cell(1), ks + math.pi / FOLD_A * np.array(m), nlow))
    prim = np.sort(np.concatenate(prim))[:nlow]
    return float(np.abs(sup - prim).max()), sup


def test_supercell_spectrum_is_the_folded_cell_spectra():
    gap, sup = _folding_gap()
    assert np.ptp(sup) > 0.1                  # a non-trivial stretch of the spectrum
    assert gap < 1e-9, gap


def test_folding_catches_inconsistent_enrichment_phases(monkeypatch):
    """Planted mistake: the enrichment columns take exp(+i k.R) where the FE
    columns take exp(-i k.R); the folding identity must then fail."""
    good = ob.elem_phases

    def bad(mesh, e, k):
        ph = good(mesh, e, k)
        ph[64:] = np.conj(ph[64:])
        return ph

    monkeypatch.setattr(ob, "elem_phases", bad)
    gap, _ = _folding_gap()
    assert gap > 1e-6, gap
