"""Pins of the oracle's H/S assembly, density and adjoint (CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble as oasm, eig as oeig, mesh as omesh, quadrature as oq
from oracle import potential as opot
from paper_1611_00731_gb300 import workloads as W


def _setup(wl):
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    return m, rules


def test_empty_lattice_spectrum_and_convergence():
    """V = 0, no enrichment: eigenvalues |G|^2/2 from above, error O(h^6)."""
    a = 4.0
    g1 = 0.5 * (2 * math.pi / a) ** 2
    errs = []
    for nel in (3, 4):
        m, rules = _setup(W.empty_lattice(nel=nel, a=a, p=4))
        H, S = oasm.assemble_HS(m, rules, np.zeros(len(rules[1])))
        w, _ = oeig.lowest_eigs(H, S, 7)
        assert abs(w[0]) < 1e-12                       # constant is in the span
        assert np.all(w[1:7] >= g1 - 1e-12)             # min-max: upper bounds
        assert np.ptp(w[1:7]) < 1e-10                   # sixfold degenerate
        errs.append(w[1] - g1)
    assert errs[1] < 1e-3
    rate = math.log(errs[0] / errs[1]) / math.log(4 / 3)
    assert 5.0 < rate < 7.0                             # O(h^6) for cubic FE


def test_harmonic_oscillator_levels():
    """V = w^2 |x - c|^2 / 2 well inside a large cell: levels w (n + 3/2)."""
    a, om = 6.0, 2.0
    wl = W.empty_lattice(nel=5, a=a, p=5)
    m, rules = _setup(wl)
    d = rules[0] - a / 2
    V = 0.5 * om ** 2 * (d * d).sum(axis=1)
    H, S = oasm.assemble_HS(m, rules, V)
    w, _ = oeig.lowest_eigs(H, S, 10)
    exact = om * np.array([1.5] + [2.5] * 3 + [3.5] * 6)
    assert np.all(w >= exact - 1e-6)                    # variational
    assert abs(w[0] - exact[0]) / exact[0] < 3e-3
    assert np.abs(w - exact).max() / exact.max() < 1e-2
    assert np.ptp(w[1:4]) < 1e-9 * w[1]                 # p-like level threefold


def test_S_spd_and_conditioning_grows_with_support_radius():
    conds = []
    for re in (None, 0.5, 1.0, 1.5):   # plain FE, then r_e enriching 1, 7, 19 vertices
        wl = (W.empty_lattice(nel=4, a=4.0, p=6) if re is None else
              W.small_two_atom(nel=4, a=4.0, quad_p=6, r_c=1.5, r_e=re))
        m, rules = _setup(wl)
        _, S = oasm.assemble_HS(m, rules, np.zeros(len(rules[1])))
        Sd = S.toarray()
        assert np.abs(Sd - Sd.T).max() < 1e-15 * np.abs(Sd).max()
        sla.cholesky(Sd)
        ev = np.linalg.eigvalsh(Sd)
        conds.append(ev[-1] / ev[0])
    assert conds[0] < conds[1] < conds[2] < conds[3]   # Table 1: cond(S) grows with r_e


def test_pu_reproduction_and_density_of_enrichment():
    """Coefficients b = 1 on every enriched vertex give psi^h = Psi (sum phi^PU = 1)."""
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=5, r_c=1.9, r_e=3.5)  # enrich every vertex
    m, rules = _setup(wl)
    pts, wts, off = rules
    k = 0  # 1s on atom 0
    c = np.zeros((m.n_dof, 1))
    for j, (al, v) in enumerate(m.enr_dof_info):
        if al == k:
            c[m.n_fe + j, 0] = 1.0
    from oracle import enrich
    al = m.alphas[k]
    psi = enrich.enrichment(al["orb"], al["rc"], al["tau"], m.a, pts, False)
    n = oasm.density(m, rules, c, np.array([1.0]))
    assert np.abs(n - psi ** 2).max() < 1e-13 * max(1.0, (psi ** 2).max())
    _, S = oasm.assemble_HS(m, rules, np.zeros(len(wts)))
    assert abs(c[:, 0] @ (S @ c[:, 0]) - wts @ psi ** 2) < 1e-12


def test_density_and_potential_energy_identities():
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=5)
    m, rules = _setup(wl)
    pts, wts, _ = rules
    V = W.random_potential(len(wts), seed=7)
    H, S = oasm.assemble_HS(m, rules, V)
    H0, _ = oasm.assemble_HS(m, rules, np.zeros(len(wts)))
    C = W.random_coefficients(m.n_dof, 3, seed=8)
    f = np.array([2.0, 1.0, 0.5])
    n = oasm.density(m, rules, C, f)
    assert abs(wts @ n - sum(f[k] * C[:, k] @ (S @ C[:, k]) for k in range(3))) < 1e-10 * abs(wts @ n)
    ev = sum(f[k] * C[:, k] @ ((H - H0) @ C[:, k]) for k in range(3))
    assert abs(ev - wts @ (V * n)) < 1e-10 * abs(ev)


def test_adjoint_matches_finite_difference():
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=4)
    m, rules = _setup(wl)
    nq = len(rules[1])
    V = W.random_potential(nq, seed=1)
    H, _ = oasm.assemble_HS(m, rules, V)
    Hbar = H.copy()
    Hbar.data = W.random_symmetric_values(H.nnz, seed=3)
    Hbar = (Hbar + Hbar.T) * 0.5
    g = oasm.adjoint_V(m, rules, Hbar)
    rng = np.random.default_rng(0)
    for q in rng.choice(nq, 6, replace=False):
        dv = np.zeros(nq)
        dv[q] = 1e-3
        Hp, _ = oasm.assemble_HS(m, rules, V + dv)
        Hm, _ = oasm.assemble_HS(m, rules, V - dv)
        fd = (Hbar.multiply(Hp - Hm)).sum() / 2e-3
        assert abs(fd - g[q]) < 1e-9 * max(1.0, abs(g[q]))


def test_translation_by_mesh_vector_preserves_spectrum():
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=5)
    m, rules = _setup(wl)
    V = opot.ionic_potential(wl, rules[0])
    H, S = oasm.assemble_HS(m, rules, V)
    w0, _ = oeig.lowest_eigs(H, S, 4)
    wl2 = dict(wl)
    wl2["atoms"] = [(s, tuple(np.array(t) + np.array([2.0, 0.0, 2.0]))) for s, t in wl["atoms"]]
    m2, rules2 = _setup(wl2)
    V2 = opot.ionic_potential(wl2, rules2[0])
    H2, S2 = oasm.assemble_HS(m2, rules2, V2)
    w2, _ = oeig.lowest_eigs(H2, S2, 4)
    assert np.abs(w0 - w2).max() < 1e-10


def test_fermi_occupations_sum():
    eps = np.array([-1.0, -0.5, -0.5, 0.2, 0.3])
    f, mu = oeig.fermi_occupations(eps, 5.0, 0.01)
    assert abs(f.sum() - 5.0) < 1e-10
    assert np.all((f >= 0) & (f <= 2))
    assert abs(f[1] - f[2]) < 1e-15
