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
