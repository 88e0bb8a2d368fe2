"""Pins of the SCF oracle (oracle/scf.py): LDA, FE Poisson, energy."""
import math

import numpy as np
import pytest

from oracle import assemble as oasm, mesh as omesh, potential as opot
from oracle import quadrature as oq, scf as oscf
from paper_1611_00731_gb300 import workloads as W


def test_exchange_constant_of_the_uniform_gas():
    # eps_x = -(3 / (4 pi)) (9 pi / 4)^(1/3) / r_s  (textbook form in r_s)
    n = np.array([1e-4, 0.01, 0.3, 2.0])
    rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    ex, vx = oscf.lda_exchange(n)
    want = -(3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
    assert np.abs(ex - want).max() < 1e-14 * np.abs(want).max()


def test_potential_is_the_density_derivative_of_the_energy():
    # v_xc = d(n eps_xc)/dn, by complex-step differentiation of pz81 itself,
    # on both branches of the correlation fit (r_s < 1 and r_s > 1)
    n = np.array([5e-4, 3e-3, 0.05, 0.2, 1.0, 4.0])
    h = 1e-30
    nc = n.astype(np.complex128) + 1j * h
    e, _ = oscf.pz81(nc)
    deriv = np.imag(nc * e) / h
    _, v = oscf.pz81(n)
    assert np.abs(deriv - v).max() < 1e-12 * np.abs(v).max()


def test_correlation_fit_continuity_and_high_density_limit():
    lo, _ = oscf.pz81_correlation(np.array([1.0 - 1e-12]))
    hi, _ = oscf.pz81_correlation(np.array([1.0]))
    assert abs(lo[0] - hi[0]) < 1e-4              # the two branches meet at r_s = 1
    # d eps_c / d ln r_s -> (1 - ln 2) / pi^2 as r_s -> 0 (Gell-Mann-Brueckner)
    r1, r2 = 1e-7, 1e-8
    e, _ = oscf.pz81_correlation(np.array([r1, r2]))
    slope = (e[0] - e[1]) / (math.log(r1) - math.log(r2))
    assert abs(slope - (1.0 - math.log(2.0)) / math.pi ** 2) < 2e-4
    assert oscf.pz81(np.array([0.0, -1.0]))[0].tolist() == [0.0, 0.0]


def test_fe_stiffness_is_twice_the_assembled_kinetic_matrix():
    wl = W.empty_lattice(nel=2)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    H, _ = oasm.assemble_HS(m, rules, np.zeros(len(rules[1])))
    K = oscf.fe_stiffness(m)
    assert abs(K - 2.0 * H).max() < 1e-12 * abs(K).max()
    assert np.abs(K @ np.ones(m.n_fe)).max() < 1e-12 * abs(K).max()


def _mode_error(nel):
    a = 4.0
    wl = W.empty_lattice(nel=nel, a=a, p=6)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    k = 2.0 * math.pi / a
    x = rules[0]
    rho = np.cos(k * x[:, 0]) * np.cos(k * x[:, 1])
    _, V = oscf.coulomb_potential(m, rules, rho)
    exact = -4.0 * math.pi / (2.0 * k * k) * rho          # del^2 V = 4 pi rho
    return np.abs(V - exact).max() / np.abs(exact).max()


def test_poisson_single_mode_closed_form_and_rate():
    e3, e6 = _mode_error(3), _mode_error(6)
    assert e6 < 2e-3
    assert e3 / e6 > 8.0        # O(h^4) for the tricubic space


def _ion_error(nel):
    a = 4.0
    wl = W.empty_lattice(nel=nel, a=a, p=8)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ion = dict(a=a, atoms=[(0, (1.1, 1.7, 0.6))], species=[dict(Z=3.0, sigma=1.0)])
    rho = opot.gaussian_charge(ion, rules[0]) - 3.0 / a ** 3   # neutral
    _, V = oscf.coulomb_potential(m, rules, rho)
    want = opot.ionic_potential(ion, rules[0])                 # zero-average sum
    return np.abs(V - want).max() / np.abs(want).max()


def test_poisson_matches_reciprocal_space_ionic_potential():
    e2, e4 = _ion_error(2), _ion_error(4)
    assert e4 < 1e-2
    assert e2 / e4 > 6.0


@pytest.fixture(scope="module")
def c1_step_inputs():
    wl = W.small_two_atom(nel=2, quad_p=6)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    rho_I = oscf.ion_density(wl, rules[0])
    n0 = np.full(len(rules[1]), wl["nelec"] / wl["a"] ** 3)
    V0, _, _ = oscf.effective_potential(m, rules, n0, rho_I)
    H, S = oasm.assemble_HS(m, rules, V0)
    from oracle import eig as oeig
    eps, C = oeig.lowest_eigs(H, S, 6)
    return wl, m, rules, rho_I, n0, V0, eps, C


def test_energy_invariant_under_a_constant_potential_shift(c1_step_inputs):
    wl, m, rules, rho_I, n0, V0, eps, C = c1_step_inputs
    a = oscf.scf_step(m, rules, wl, eps, C, wl["nelec"], 0.01, 0.5, n0, V0, rho_I)
    b = oscf.scf_step(m, rules, wl, eps + 0.37, C, wl["nelec"], 0.01, 0.5, n0, V0 + 0.37, rho_I)
    assert abs(a["e_total"] - b["e_total"]) < 1e-10
    assert abs(b["mu"] - a["mu"] - 0.37) < 1e-10
    assert a["e_es"] >= 0.0                                   # neutral total charge
    assert abs(rules[1] @ a["n_out"] - wl["nelec"]) < 1e-8    # sum f = N_e, C S-orthonormal
    assert np.allclose(a["n_new"], n0 + 0.5 * (a["n_out"] - n0))


def test_pulay_solves_a_linear_fixed_point_in_dimension_plus_one_steps():
    # n -> G(n) = A n + b on R^3: Anderson/Pulay mixing with enough history
    # reaches the fixed point after at most dim + 1 residual evaluations
    rng = np.random.default_rng(1)
    A = 0.5 * rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    fixed = np.linalg.solve(np.eye(3) - A, b)
    w = np.ones(3)
    mix = oscf.PulayMixer(depth=5)
    n = np.zeros(3)
    for _ in range(4):
        n = mix.mix(n, A @ n + b, w, 0.3)
    assert np.abs(n - fixed).max() < 1e-8 * np.abs(fixed).max()
    # depth 1 is linear mixing
    one = oscf.PulayMixer(depth=1)
    x = rng.standard_normal(3)
    assert np.allclose(one.mix(x, A @ x + b, w, 0.3), x + 0.3 * (A @ x + b - x))
