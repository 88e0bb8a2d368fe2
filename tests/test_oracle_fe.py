"""Pins of the oracle's shape functions and Gauss rules (CPU only).

Each check compares the oracle against something other than itself: exact
rational arithmetic, closed-form integrals, or structural identities.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fe
from paper_1611_00731_gb300 import workloads as W
from oracle import mesh as omesh
from oracle import assemble as oasm


def test_partition_of_unity_and_zero_gradient_sum():
    rng = np.random.default_rng(0)
    xi = rng.uniform(-1, 1, size=(200, 3))
    for fn in (fe.tricubic, fe.trilinear):
        N, dN = fn(xi)
        assert np.abs(N.sum(axis=1) - 1.0).max() < 1e-13
        assert np.abs(dN.sum(axis=2)).max() < 1e-12


def test_kronecker_delta_at_nodes():
    nodes = fe.CUBIC_NODES
    pts = np.array([[nodes[a], nodes[b], nodes[c]]
                    for c in range(4) for b in range(4) for a in range(4)])
    N, _ = fe.tricubic(pts)
    assert np.abs(N - np.eye(64)).max() < 1e-14
    v = np.array([[a, b, c] for c in (-1, 1) for b in (-1, 1) for a in (-1, 1)], float)
    P, _ = fe.trilinear(v)
    assert np.abs(P - np.eye(8)).max() < 1e-15


def test_tricubic_reproduces_cubic_polynomials():
    # interpolation of x^3 y^2 z at the nodes is exact inside the element
    nodes = fe.CUBIC_NODES
    f = lambda p: p[..., 0] ** 3 * p[..., 1] ** 2 * p[..., 2] - 2 * p[..., 1] ** 3 + 0.5
    npts = np.array([[nodes[a], nodes[b], nodes[c]]
                     for c in range(4) for b in range(4) for a in range(4)])
    xi = np.random.default_rng(1).uniform(-1, 1, size=(50, 3))
    N, dN = fe.tricubic(xi)
    assert np.abs(N @ f(npts) - f(xi)).max() < 1e-13
    # derivative d/dx of the interpolant = 3 x^2 y^2 z
    assert np.abs(dN[0] @ f(npts) - 3 * xi[:, 0] ** 2 * xi[:, 1] ** 2 * xi[:, 2]).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 4, 5, 8])
def test_gauss_exactness(p):
    lo, hi = np.array([0.3, -1.0, 2.0]), np.array([1.1, 0.5, 2.25])
    pts, wts = fe.gauss_box(p, lo, hi)
    assert abs(wts.sum() - np.prod(hi - lo)) < 1e-14
    for ax in range(3):
        for k in range(2 * p):  # exact for degree <= 2p - 1
            exact = (hi[ax] ** (k + 1) - lo[ax] ** (k + 1)) / (k + 1) * np.prod(
                np.delete(hi - lo, ax))
            got = wts @ pts[:, ax] ** k
            assert abs(got - exact) <= 1e-13 * max(1.0, abs(exact))


# --- exact rational 1D matrices ------------------------------------------------

def _poly_mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _poly_int_m1_1(p):
    return sum(c * (Fraction(1) - Fraction((-1) ** (k + 1))) / (k + 1) for k, c in enumerate(p))


def _poly_deriv(p):
    return [k * c for k, c in enumerate(p)][1:]


def _lagrange_rational():
    nodes = [Fraction(-1), Fraction(-1, 3), Fraction(1, 3), Fraction(1)]
    polys = []
    for a in range(4):
        p = [Fraction(1)]
        for b in range(4):
            if b != a:
                p = _poly_mul(p, [-nodes[b] / (nodes[a] - nodes[b]), 1 / (nodes[a] - nodes[b])])
        polys.append(p)
    return polys


def test_one_element_mass_and_stiffness_exact():
    """FE block of one element against Kronecker products of exact 1D matrices."""
    L = _lagrange_rational()
    M1 = np.array([[float(_poly_int_m1_1(_poly_mul(L[a], L[b]))) for b in range(4)]
                   for a in range(4)])
    K1 = np.array([[float(_poly_int_m1_1(_poly_mul(_poly_deriv(L[a]), _poly_deriv(L[b]))))
                    for b in range(4)] for a in range(4)])
    wl = W.empty_lattice(nel=2, a=3.0, p=4)
    m = omesh.Mesh(wl)
    h = m.h
    lo, hi = m.elem_box(5)
    pts, wts = fe.gauss_box(4, lo, hi)
    c0 = -0.75
    He, Se = oasm.element_HS(m, 5, pts, wts, np.full(len(wts), c0))
    J = (h / 2) ** 3
    Mex = np.kron(M1, np.kron(M1, M1)) * J
    Kex = (np.kron(M1, np.kron(M1, K1)) + np.kron(M1, np.kron(K1, M1))
           + np.kron(K1, np.kron(M1, M1))) * J * (2 / h) ** 2
    assert np.abs(Se - Mex).max() < 1e-14 * np.abs(Mex).max() * 10
    assert np.abs(He - (0.5 * Kex + c0 * Mex)).max() < 1e-13 * np.abs(Kex).max()
