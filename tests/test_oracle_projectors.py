"""Pins of the nonlocal-projector oracle (oracle/projectors.py)."""
import math

import numpy as np

from oracle import fe, mesh as omesh, projectors as onl, quadrature as oq
from paper_1611_00731_gb300 import workloads as W


def _projs(tau, rp):
    return [dict(tau=tau, l=0, m=0, rp=rp)] + [dict(tau=tau, l=1, m=m, rp=rp) for m in (-1, 0, 1)]


def test_projectors_are_orthonormal():
    a = 8.0
    x1, w1 = fe.gauss_1d(64)
    x1 = (x1 + 1.0) * a / 2.0
    w1 = w1 * a / 2.0
    X = np.array(np.meshgrid(x1, x1, x1, indexing="ij")).reshape(3, -1).T
    Wt = np.einsum("i,j,k->ijk", w1, w1, w1).reshape(-1)
    ps = _projs((4.1, 3.9, 4.0), 0.6)
    V = np.stack([onl.projector_values(p, a, X) for p in ps], axis=1)
    G = V.T @ (Wt[:, None] * V)
    assert np.abs(G - np.eye(len(ps))).max() < 1e-9


def test_projections_sum_to_the_projector_integral():
    wl = W.small_two_atom(nel=2, quad_p=10)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    rp = 0.7
    ps = _projs((0.0, 0.0, 0.0), rp)
    F = onl.projections(m, rules, ps)
    s_int = onl.projector_norm(0, rp) / math.sqrt(4.0 * math.pi) * (2.0 * math.pi * rp * rp) ** 1.5
    fe_sum = F[:m.n_fe].sum(axis=0)           # the FE functions sum to 1
    assert abs(fe_sum[0] - s_int) < 1e-6 * s_int
    assert np.abs(fe_sum[1:]).max() < 1e-12 * s_int
    h = np.array([0.7, 0.2, 0.2, 0.2])
    Hn = F @ np.diag(h) @ F.T
    assert np.abs(Hn - Hn.T).max() < 1e-15 * np.abs(Hn).max()
    assert np.linalg.eigvalsh(Hn).min() > -1e-12 * np.abs(Hn).max()


# ---- Bloch-phased projections (k != 0) ---------------------------------------

def _kvec(a, frac):
    return 2.0 * math.pi / a * np.asarray(frac, dtype=np.float64)


def test_bloch_projections_reduce_to_gamma_and_are_periodic_in_k():
    wl = W.small_two_atom(nel=2, quad_p=6)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ps = _projs((0.3, -0.2, 0.1), 0.6)
    F0 = onl.projections(m, rules, ps)
    Fk0 = onl.projections_k(m, rules, ps, (0.0, 0.0, 0.0))
    assert np.abs(Fk0.imag).max() == 0.0
    assert np.abs(Fk0.real - F0).max() < 1e-14 * np.abs(F0).max()
    k = _kvec(m.a, (0.25, -0.1, 0.4))
    G = _kvec(m.a, (1.0, -2.0, 1.0))
    Fk = onl.projections_k(m, rules, ps, k)
    FkG = onl.projections_k(m, rules, ps, k + G)
    assert np.abs(FkG - Fk).max() < 1e-12 * np.abs(Fk).max()
    # the nonlocal term F h F^H is Hermitian positive semidefinite
    Hn = Fk @ np.diag([0.5, 0.3, 0.3, 0.3]) @ Fk.conj().T
    assert np.abs(Hn - Hn.conj().T).max() < 1e-15 * np.abs(Hn).max()
    assert np.linalg.eigvalsh(Hn).min() > -1e-12 * np.abs(Hn).max()


def test_bloch_projections_of_a_plane_wave_approach_the_fourier_transform():
    """sum_g exp(-i k.x_g) F[g, p] over the FE DOFs is the projection of the
    tricubic interpolant of exp(i k.x); it converges to
    int exp(-i k.x) v(x - tau) dx = exp(-i k.tau) v~(k), with, for the
    Gaussian v = N r^l exp(-r^2 / (2 s^2)) Y_lm,
      l = 0: v~ = N Y_00 (2 pi s^2)^(3/2) exp(-|k|^2 s^2 / 2),
      l = 1: v~ = -i s^2 N c k_m (2 pi s^2)^(3/2) exp(-|k|^2 s^2 / 2),
    c = sqrt(3 / (4 pi)), k_m the Cartesian component of r Y_1m / c
    (m = -1: y, 0: z, 1: x): the transform of x_m exp(-r^2 / 2s^2) is
    i d/dk_m of the Gaussian's."""
    a, s = 4.0, 0.6
    tau = np.array([1.3, 2.1, 1.7])
    ps = _projs(tuple(tau), s)
    k = _kvec(a, (0.25, 0.125, -0.25))
    kk = float(k @ k)
    g = (2.0 * math.pi * s * s) ** 1.5 * math.exp(-kk * s * s / 2.0) * np.exp(-1j * (k @ tau))
    c = math.sqrt(3.0 / (4.0 * math.pi))
    want = np.array([onl.projector_norm(0, s) / math.sqrt(4.0 * math.pi) * g]
                    + [-1j * s * s * onl.projector_norm(1, s) * c * k[ax] * g for ax in (1, 2, 0)])
    errs = []
    for nel in (2, 4):
        wl = W.small_two_atom(nel=nel, a=a, quad_p=8)
        m = omesh.Mesh(wl)
        rules = oq.all_rules(m)
        F = onl.projections_k(m, rules, ps, k)
        mm = m.nfe_axis
        gi = np.arange(m.n_fe)
        xg = np.stack([gi % mm, (gi // mm) % mm, gi // (mm * mm)], axis=1) * (a / mm)
        got = np.exp(-1j * (xg @ k)) @ F[:m.n_fe]
        errs.append(np.abs(got - want).max() / np.abs(want).max())
    print("plane-wave projection errors", errs)
    assert errs[1] < 2e-5
    assert errs[1] < errs[0] / 8.0      # O(h^4) interpolation error: ~16x per halving
