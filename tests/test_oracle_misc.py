"""Pins of the oracle's ionic potential and the 1D PU example (CPU only)."""
import math
import os

import numpy as np

from oracle import potential as opot, pu1d
from paper_1611_00731_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def test_potential_solves_poisson():
    """FD Laplacian of V_I equals 4 pi (rho_I - <rho_I>) (Sec. 3, eq. poisson)."""
    wl = W.workload("c1_two_atom_4cube")
    rng = np.random.default_rng(2)
    x = rng.uniform(0, wl["a"], size=(12, 3))
    h = 1e-3
    lap = -6 * opot.ionic_potential(wl, x)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        lap += opot.ionic_potential(wl, x + e) + opot.ionic_potential(wl, x - e)
    lap /= h * h
    Z = sum(wl["species"][s]["Z"] for s, _ in wl["atoms"])
    rho = opot.gaussian_charge(wl, x) - Z / wl["a"] ** 3
    assert np.abs(lap - 4 * math.pi * rho).max() < 2e-4 * np.abs(4 * math.pi * rho).max()


def test_potential_near_isolated_ion():
    """In a large cell V_I - V_I(far) tracks -Z erf(r/s)/r + Z/r_far."""
    sp = dict(Z=3.0, sigma=0.8, orbitals=[], r_c=1.0, r_e=1.0)
    wl = dict(a=30.0, species=[sp], atoms=[(0, (15.0, 15.0, 15.0))])
    r = np.array([0.1, 0.5, 1.0, 2.0])
    pts = np.stack([15.0 + r, np.full(4, 15.0), np.full(4, 15.0)], axis=1)
    V = opot.ionic_potential(wl, pts)
    iso = -3.0 * np.array([math.erf(t / 0.8) for t in r]) / r
    d = (V - iso)
    # the difference is the (smooth) field of the images and background
    assert np.ptp(d) < 5e-3


def test_pu1d_constants_are_the_printed_ones():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("pu1d"):
            k, *v = line.split()
            vals[k] = [float(t) for t in v]
    assert (pu1d.A, pu1d.B, pu1d.C, pu1d.D) == (vals["pu1d_a"][0], vals["pu1d_b"][0],
                                                vals["pu1d_c"][0], vals["pu1d_d"][0])
    assert np.allclose(pu1d.NODES, vals["pu1d_nodes"], atol=1e-15)


def test_pu1d_reproduces_enrichment_and_beats_fe():
    c, err = pu1d.project(pu1d.psi)
    assert err < 1e-13
    # end nodes see Psi ~ 1e-6, so their b is the least well determined
    assert np.abs(c[:7]).max() < 1e-12 and np.abs(c[7:] - 1).max() < 1e-9
    u = lambda x: pu1d.psi(x) + pu1d.delta(x)
    _, e_pufe = pu1d.project(u, True)
    _, e_fe = pu1d.project(u, False)
    assert e_pufe < 0.2 * e_fe


def test_ewald_split_potential_equals_direct_sum():
    """The Ewald-split evaluation of V_I (real-space short-range part, mean
    correction, shorter reciprocal sum) equals the direct reciprocal sum."""
    for name in ("c1_two_atom_4cube", "c2_rocksalt_12cube"):
        wl = W.workload(name)
        x = np.random.default_rng(3).uniform(0, wl["a"], size=(150, 3))
        v0 = opot.ionic_potential(wl, x)
        for eta in (1.2, 1.5, 2.0):
            v1 = opot.ionic_potential_ewald(wl, x, eta)
            assert np.abs(v1 - v0).max() < 1e-13 * np.abs(v0).max(), (name, eta)


def test_nested_dissection_shift_invert_and_rayleigh_ritz():
    """The large-cell eigensolver path (nested-dissection SuperLU shift-invert)
    returns the dense LAPACK eigenpairs on C1, and Rayleigh-Ritz on the
    unperturbed eigenvectors gives a perturbed pencil's eigenvalues to second
    order."""
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    import scipy.sparse as sp
    import oracle_pool as OP
    from oracle import assemble as oasm, eig as oeig, mesh as omesh, quadrature as oq
    wl = W.workload("c1_two_atom_4cube")
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    V = opot.ionic_potential(wl, rules[0])
    H, S = oasm.assemble_HS(m, rules, V)
    coords, period = OP.dof_grid_coords(wl)
    perm = oeig.nested_dissection_order(coords, period)
    w1, X = oeig.lowest_eigs_shift_invert(H, S, 6, V.min() - 0.1, perm)
    w0, _ = oeig.lowest_eigs(H, S, 6)
    assert np.abs(w1 - w0).max() < 1e-10
    # a perturbation of the potential by 1e-5 (a random matrix perturbation of
    # that size would be amplified by cond(S) ~ 1e9 instead)
    dV = 1e-5 * W.random_potential(len(V), seed=5)
    Hp, _ = oasm.assemble_HS(m, rules, V + dV)
    wp, _ = oeig.lowest_eigs(Hp, S, 6)
    wr = oeig.rayleigh_ritz(Hp, S, X)
    # the top of the subspace couples to states outside it: compare the
    # lowest 5 of the 6 (the C2 test keeps 12 and compares 8)
    assert np.abs(wr[:5] - wp[:5]).max() < 1e-11
    assert np.abs(wp - w0).max() > 1e-7        # the perturbation itself is first order
