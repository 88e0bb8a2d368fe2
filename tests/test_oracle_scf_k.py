"""Pins of the oracle's k-point SCF step (oracle/scf.py: scf_step_k).

* Gamma limit: one k-point k = 0 of weight 1 is the Gamma-point step.
* Zone folding (Sec. 4, eqs. bloch, strong): one SCF step of a 2x2x2
  supercell at a wavevector k_s is the step of its cell at the eight folded
  wavevectors k_s + (pi/a) m with weights 1/8, when both take the same
  states (the supercell's lowest M and their images among the cell's): the
  energies are eight times the cell's and the output densities agree point
  by point.  This fixes the k-weights of the occupations, the density, the
  band energy and the entropy.  A planted mistake (occupations normalised
  without the k-weights) must break it.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble as oasm, bloch as ob, eig as oeig, mesh as omesh, quadrature as oq
from oracle import scf as oscf
from paper_1611_00731_gb300 import workloads as W

FOLD_A, FOLD_NEL = 8.0, 2


def _fold_cell(rep):
    a = FOLD_A * rep
    sp = [W._species(W.H_LIKE_1S, 1.0, 0.5), W._species(W.LI_LIKE_1S2S2P, 1.0, 0.5)]
    base = [(0, np.array([0.0, 0.0, 0.0])), (1, np.array([4.0, 0.0, 4.0]))]
    atoms = []
    for s, tau in base:
        for m in np.ndindex(rep, rep, rep):
            atoms.append((s, tuple(tau + FOLD_A * np.array(m[::-1]))))
    return dict(name=f"fold_{rep}", a=a, nel=FOLD_NEL * rep, species=sp, atoms=atoms,
                quad=dict(mode=W.QUAD_FIXED, p_far=8, p_near=8, p_min=0, p_max=0,
                          tol=1e-6, max_depth=0), nocc=1, nelec=4.0 * rep ** 3)


def _setup(wl):
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    K = oscf.fe_stiffness(m)
    rho = oscf.ion_density(wl, rules[0])
    n = np.full(len(rules[1]), wl["nelec"] / wl["a"] ** 3)
    V, _, _ = oscf.effective_potential(m, rules, n, rho, K)
    return m, rules, K, rho, n, V


def _states(m, rules, V, k, count):
    H, S = ob.assemble_HS_k(m, rules, V, k)
    return sla.eigh(H.toarray(), S.toarray(), subset_by_index=[0, count - 1])


def test_single_gamma_point_is_the_gamma_step():
    wl = W.small_two_atom(nel=2, quad_p=6)
    m, rules, K, rho, n, V = _setup(wl)
    H, S = oasm.assemble_HS(m, rules, V)
    ev, C = oeig.lowest_eigs(H, S, 6)
    r0 = oscf.scf_step(m, rules, wl, ev, C, wl["nelec"], 0.01, 0.5, n, V, rho, K)
    r1 = oscf.scf_step_k(m, rules, wl, [np.zeros(3)], [1.0], [ev], [C.astype(complex)],
                         wl["nelec"], 0.01, 0.5, n, V, rho, K)
    assert abs(r1["e_total"] - r0["e_total"]) < 1e-12 * abs(r0["e_total"])
    assert np.abs(r1["n_out"] - r0["n_out"]).max() < 1e-13 * np.abs(r0["n_out"]).max()
    assert np.abs(r1["V_eff"] - r0["V_eff"]).max() < 1e-12 * np.abs(r0["V_eff"]).max()


@pytest.fixture(scope="module")
def folded():
    sup, cell = _fold_cell(2), _fold_cell(1)
    ms, rs, Ks, rhos, ns, Vs = _setup(sup)
    mc, rc, Kc, rhoc, nc, Vc = _setup(cell)
    ks = math.pi / FOLD_A * np.array([0.3, -0.2, 0.1])   # supercell wavevector
    kc = [ks + math.pi / FOLD_A * np.array(mm) for mm in np.ndindex(2, 2, 2)]
    # the supercell's lowest M states, M at a gap above the 16 electrons' 8
    es_all = _states(ms, rs, Vs, ks, 24)[0]
    M = next(j for j in range(12, 23) if es_all[j] - es_all[j - 1] > 1e-4)
    es, Cs = _states(ms, rs, Vs, ks, M)
    # their images among the cell's states at the folded wavevectors
    ec_all = [_states(mc, rc, Vc, k, 12)[0] for k in kc]
    cut = 0.5 * (es_all[M - 1] + es_all[M])
    counts = [int((e < cut).sum()) for e in ec_all]
    assert sum(counts) == M and max(counts) < 12
    cell_states = [_states(mc, rc, Vc, k, c) for k, c in zip(kc, counts)]
    return dict(sup=sup, cell=cell, ms=ms, rs=rs, Ks=Ks, rhos=rhos, ns=ns, Vs=Vs, ks=ks, es=es,
                Cs=Cs, mc=mc, rc=rc, Kc=Kc, rhoc=rhoc, nc=nc, Vc=Vc, kc=kc, cell_states=cell_states)


def _steps(F):
    rs = oscf.scf_step_k(F["ms"], F["rs"], F["sup"], [F["ks"]], [1.0], [F["es"]], [F["Cs"]],
                         F["sup"]["nelec"], 0.01, 0.5, F["ns"], F["Vs"], F["rhos"], F["Ks"])
    rc = oscf.scf_step_k(F["mc"], F["rc"], F["cell"], F["kc"], [1.0 / 8] * 8,
                         [e for e, _ in F["cell_states"]], [C for _, C in F["cell_states"]],
                         F["cell"]["nelec"], 0.01, 0.5, F["nc"], F["Vc"], F["rhoc"], F["Kc"])
    return rs, rc


def _cell_points_in_supercell(F):
    """Index of every supercell point among the cell's points (same fixed
    rule on every element; element e = ex + nel (ey + nel ez))."""
    offc, offs = F["rc"][2], F["rs"][2]
    nc, ns = FOLD_NEL, 2 * FOLD_NEL
    idx = np.empty(offs[-1], dtype=np.int64)
    for e in range(ns ** 3):
        ex, ey, ez = e % ns, (e // ns) % ns, e // ns ** 2
        ec = ex % nc + nc * (ey % nc + nc * (ez % nc))
        idx[offs[e]:offs[e + 1]] = np.arange(offc[ec], offc[ec + 1])
    return idx


def test_supercell_step_is_the_folded_cell_step(folded):
    F = folded
    rs, rc = _steps(F)
    for key in ("e_band", "e_dc", "e_es", "e_xc", "e_ts", "e_total"):
        assert abs(rs[key] - 8.0 * rc[key]) < 1e-8 * max(1.0, abs(rs[key])), (key, rs[key], rc[key])
    idx = _cell_points_in_supercell(F)
    assert np.abs(rs["n_out"] - rc["n_out"][idx]).max() < 1e-8 * np.abs(rs["n_out"]).max()
    assert abs(rs["mu"] - rc["mu"]) < 1e-8


def test_folding_catches_unweighted_occupations(folded, monkeypatch):
    """Planted mistake: the Fermi level fixed by sum_k sum_n f_nk = N (the
    k-weights dropped); the supercell (one k-point of weight 1) is unchanged,
    its folded cell is not, so the identity must fail."""
    good = oeig.fermi_occupations_k
    monkeypatch.setattr(oscf, "fermi_occupations_k",
                        lambda eps, wk, nelec, kT: good(eps, np.ones(len(wk)), nelec, kT))
    rs, rc = _steps(folded)
    assert abs(rs["e_total"] - 8.0 * rc["e_total"]) > 1e-4
