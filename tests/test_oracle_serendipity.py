"""Pins of the cubic serendipity element (oracle/fe.py: serendipity32), the
classical FE part of the paper's own PUFE runs (Sec. 6), and of the mesh
built on it (oracle/mesh.py, fe = "serendipity32")."""
import math

import numpy as np
import scipy.linalg as sla

from oracle import bloch as ob, fe, mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import workloads as W

NODES = fe.CUBIC_NODES[np.stack([fe.SERENDIPITY_LOCAL & 3, (fe.SERENDIPITY_LOCAL >> 2) & 3,
                                 fe.SERENDIPITY_LOCAL >> 4], axis=1)]


def _points(n=200, seed=0):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, 3))


def test_nodes_are_vertices_and_inner_edge_nodes():
    assert len(fe.SERENDIPITY_LOCAL) == 32
    inner = (np.abs(NODES) < 1.0).sum(axis=1)
    assert (inner == 0).sum() == 8 and (inner == 1).sum() == 24


def test_kronecker_delta_at_the_nodes():
    N, _ = fe.serendipity32(NODES)
    assert np.abs(N - np.eye(32)).max() < 1e-14


def test_partition_of_unity():
    N, dN = fe.serendipity32(_points())
    assert np.abs(N.sum(axis=1) - 1.0).max() < 1e-14
    assert np.abs(dN.sum(axis=2)).max() < 1e-13


def _monomials(x, exps):
    return np.stack([x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c for a, b, c in exps], axis=1)


CUBIC = [(a, b, c) for a in range(4) for b in range(4) for c in range(4) if a + b + c <= 3]
SUPERLINEAR = [(2, 1, 1), (1, 2, 1), (1, 1, 2), (3, 1, 0), (3, 0, 1), (1, 3, 0), (0, 3, 1),
               (1, 0, 3), (0, 1, 3), (3, 1, 1), (1, 3, 1), (1, 1, 3)]


def test_reproduces_every_cubic_polynomial_and_its_gradient():
    x = _points()
    N, dN = fe.serendipity32(x)
    for a, b, c in CUBIC:
        p = lambda y: y[:, 0] ** a * y[:, 1] ** b * y[:, 2] ** c
        coef = p(NODES)
        assert np.abs(N @ coef - p(x)).max() < 1e-13
        grad = [a * x[:, 0] ** max(a - 1, 0) * x[:, 1] ** b * x[:, 2] ** c,
                b * x[:, 0] ** a * x[:, 1] ** max(b - 1, 0) * x[:, 2] ** c,
                c * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** max(c - 1, 0)]
        for d in range(3):
            assert np.abs(dN[d] @ coef - grad[d]).max() < 1e-12


def test_spans_the_cubic_serendipity_space():
    """The 32 functions span exactly P_3 plus the 12 superlinear monomials:
    each function is a combination of those monomials (zero residual), and
    the monomials' interpolants reproduce them."""
    x = _points(400, seed=1)
    M = _monomials(x, CUBIC + SUPERLINEAR)
    assert np.linalg.matrix_rank(M) == 32
    N, _ = fe.serendipity32(x)
    coef, *_ = np.linalg.lstsq(M, N, rcond=None)
    assert np.abs(M @ coef - N).max() < 1e-12
    for exps in SUPERLINEAR:
        p = _monomials(x, [exps])[:, 0]
        assert np.abs(N @ _monomials(NODES, [exps])[:, 0] - p).max() < 1e-12


def test_gradients_are_the_derivatives():
    x = _points(50, seed=2)
    _, dN = fe.serendipity32(x)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (fe.serendipity32(x + e)[0] - fe.serendipity32(x - e)[0]) / (2 * h)
        assert np.abs(fd - dN[d]).max() < 1e-8


def test_mesh_numbering():
    wl = dict(W.empty_lattice(nel=3), fe="serendipity32")
    m = omesh.Mesh(wl)
    assert m.n_fe == 7 * 27 and m.nfe_e == 32
    seen = np.concatenate([m.fe_dofs(e) for e in range(m.nelem)])
    assert seen.min() == 0 and set(seen.tolist()) == set(range(m.n_fe))


def _empty_lowest(nel, a=4.0):
    wl = dict(W.empty_lattice(nel=nel, a=a, p=4), fe="serendipity32")
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    k = 2.0 * math.pi / a * np.array([0.3, -0.2, 0.1])
    H, S = ob.assemble_HS_k(m, rules, np.zeros(len(rules[1])), k)
    w = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True, subset_by_index=[0, 3])
    G = 2.0 * math.pi / a * np.array([[0, 0, 0], [-1, 0, 0], [0, 1, 0], [0, 0, -1],
                                      [1, 0, 0], [0, -1, 0], [0, 0, 1]], dtype=np.float64)
    return w, np.sort(0.5 * ((G + k) ** 2).sum(axis=1))[:4]


def test_empty_lattice_spectrum_converges_from_above():
    """Free-electron bands |k + G|^2 / 2 in the serendipity space: variational
    (from above) and converging at the rate of a complete cubic space."""
    w3, ex = _empty_lowest(3)
    w5, _ = _empty_lowest(5)
    assert np.all(w3 >= ex - 1e-12) and np.all(w5 >= ex - 1e-12)
    e3, e5 = w3[0] - ex[0], w5[0] - ex[0]
    rate = math.log(e3 / e5) / math.log(5.0 / 3.0)
    print(f"serendipity empty-lattice error {e3:.2e} -> {e5:.2e}, rate {rate:.2f}")
    assert rate > 5.0   # O(h^6): eigenvalue error of a complete cubic space
