"""Finite-element shape functions and Gauss rules (oracle, test infrastructure).

* Classical FE part: tricubic Lagrange hexahedra, 64 nodes per element, nodes
  equispaced at xi in {-1, -1/3, 1/3, 1}, local node index a + 4 b + 16 c
  (x fastest); or the cubic serendipity hexahedron with 32 nodes (Sec. 6:
  the paper's PUFE runs use it), whose nodes are the 8 vertices and the two
  inner nodes of each of the 12 edges, i.e. the tricubic nodes with at most
  one index in {1, 2}.  Its functions (the classical 32-node element):
      vertex s in {-1, 1}^3:  N = 1/64 prod_d (1 + s_d xi_d) (9 |xi|^2 - 19),
      edge along axis d, inner coordinate t = -+1/3, the other two s_e = -+1:
          N = 9/64 (1 - xi_d^2) (1 + 9 t xi_d) prod_{e != d} (1 + s_e xi_e).
* Partition of unity: trilinear hexahedra, 8 vertices, local vertex index
  a + 2 b + 4 c (Sec. 5.1: trilinear PU regardless of the FE order).
* Gauss-Legendre rules: NumPy's ``leggauss`` (a library primitive).

Pins (tests/test_oracle_fe.py): partition of unity and zero gradient sum,
Kronecker-delta property at the nodes, polynomial exactness of the Gauss
rules, and the one-element mass/stiffness matrices against exact rational
Kronecker products; for the serendipity element the Kronecker property, the
partition of unity, exact reproduction of every cubic polynomial (values and
gradients), and its span: the 20 cubic monomials plus the 12 superlinear
ones x^2yz, xy^2z, xyz^2, x^3y, x^3z, xy^3, y^3z, xz^3, yz^3, x^3yz, xy^3z,
xyz^3 (the cubic serendipity space of the cube).
"""
from __future__ import annotations

import numpy as np

CUBIC_NODES = np.array([-1.0, -1.0 / 3.0, 1.0 / 3.0, 1.0])


def lagrange_cubic_1d(xi):
    """Values and derivatives of the four cubic Lagrange polynomials.

    L_a(xi) = prod_{b != a} (xi - xi_b) / (xi_a - xi_b).  The derivative is
    the product rule written out: sum over the dropped factor c.
    Returns (L, dL), each of shape xi.shape + (4,).
    """
    xi = np.asarray(xi, dtype=np.float64)
    L = np.ones(xi.shape + (4,))
    dL = np.zeros(xi.shape + (4,))
    nodes = CUBIC_NODES
    for a in range(4):
        for b in range(4):
            if b != a:
                L[..., a] *= (xi - nodes[b]) / (nodes[a] - nodes[b])
        for c in range(4):
            if c == a:
                continue
            term = np.full(xi.shape, 1.0 / (nodes[a] - nodes[c]))
            for b in range(4):
                if b != a and b != c:
                    term = term * (xi - nodes[b]) / (nodes[a] - nodes[b])
            dL[..., a] += term
    return L, dL


def linear_1d(xi):
    """The two linear hats on [-1, 1]: (1 - xi)/2 and (1 + xi)/2, and slopes."""
    xi = np.asarray(xi, dtype=np.float64)
    L = np.stack([(1.0 - xi) / 2.0, (1.0 + xi) / 2.0], axis=-1)
    dL = np.stack([np.full(xi.shape, -0.5), np.full(xi.shape, 0.5)], axis=-1)
    return L, dL


def _tensor(L1, dL1, k):
    """Tensor-product values and reference gradients from 1D tables.

    L1, dL1: lists of three arrays (one per axis) of shape (Q, k).
    Returns N (Q, k^3) and dN (3, Q, k^3) with local index a + k b + k^2 c.
    """
    Lx, Ly, Lz = L1
    dx, dy, dz = dL1
    Q = Lx.shape[0]
    N = np.einsum("qa,qb,qc->qcba", Lx, Ly, Lz).reshape(Q, k ** 3)
    Gx = np.einsum("qa,qb,qc->qcba", dx, Ly, Lz).reshape(Q, k ** 3)
    Gy = np.einsum("qa,qb,qc->qcba", Lx, dy, Lz).reshape(Q, k ** 3)
    Gz = np.einsum("qa,qb,qc->qcba", Lx, Ly, dz).reshape(Q, k ** 3)
    return N, np.stack([Gx, Gy, Gz])


def tricubic(xi):
    """64 tricubic Lagrange functions at reference points xi (Q, 3).

    Returns N (Q, 64) and reference gradients dN (3, Q, 64); local index
    a + 4 b + 16 c for node (xi_a, xi_b, xi_c).
    """
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    tabs = [lagrange_cubic_1d(xi[:, d]) for d in range(3)]
    return _tensor([t[0] for t in tabs], [t[1] for t in tabs], 4)


# local tricubic indices a + 4 b + 16 c of the 32 serendipity nodes (at most
# one of a, b, c inner), ascending: the serendipity element's column order
SERENDIPITY_LOCAL = np.array([a + 4 * b + 16 * c for c in range(4) for b in range(4)
                              for a in range(4)
                              if (a in (1, 2)) + (b in (1, 2)) + (c in (1, 2)) <= 1])


def serendipity32(xi):
    """32 cubic serendipity functions at reference points xi (Q, 3).

    Returns N (Q, 32) and reference gradients dN (3, Q, 32), columns in the
    order of SERENDIPITY_LOCAL (formulas in the module docstring).
    """
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    Q = xi.shape[0]
    N = np.zeros((Q, 32))
    dN = np.zeros((3, Q, 32))
    r2 = (xi * xi).sum(axis=1)
    for col, loc in enumerate(SERENDIPITY_LOCAL):
        idx = (loc & 3, (loc >> 2) & 3, loc >> 4)
        node = CUBIC_NODES[list(idx)]
        inner = [d for d in range(3) if idx[d] in (1, 2)]
        if not inner:                       # vertex
            lin = 1.0 + node[None, :] * xi  # (Q, 3)
            P = lin.prod(axis=1)
            G = 9.0 * r2 - 19.0
            N[:, col] = P * G / 64.0
            for d in range(3):
                others = np.prod([lin[:, e] for e in range(3) if e != d], axis=0)
                dN[d, :, col] = (node[d] * others * G + P * 18.0 * xi[:, d]) / 64.0
        else:                               # inner node of an edge along axis d
            d = inner[0]
            t = node[d]
            x = xi[:, d]
            f = (1.0 - x * x) * (1.0 + 9.0 * t * x)
            fp = -2.0 * x * (1.0 + 9.0 * t * x) + 9.0 * t * (1.0 - x * x)
            oth = [e for e in range(3) if e != d]
            l1 = 1.0 + node[oth[0]] * xi[:, oth[0]]
            l2 = 1.0 + node[oth[1]] * xi[:, oth[1]]
            N[:, col] = 9.0 / 64.0 * f * l1 * l2
            dN[d, :, col] = 9.0 / 64.0 * fp * l1 * l2
            dN[oth[0], :, col] = 9.0 / 64.0 * f * node[oth[0]] * l2
            dN[oth[1], :, col] = 9.0 / 64.0 * f * l1 * node[oth[1]]
    return N, dN


def trilinear(xi):
    """8 trilinear PU functions at reference points xi (Q, 3).

    Returns N (Q, 8) and reference gradients dN (3, Q, 8); local vertex index
    a + 2 b + 4 c for vertex (a, b, c) in {0, 1}^3.
    """
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    tabs = [linear_1d(xi[:, d]) for d in range(3)]
    return _tensor([t[0] for t in tabs], [t[1] for t in tabs], 2)


def gauss_1d(p):
    """p-point Gauss-Legendre nodes and weights on [-1, 1] (NumPy leggauss)."""
    x, w = np.polynomial.legendre.leggauss(int(p))
    return x, w


def gauss_box(p, lo, hi):
    """Tensor p^3 Gauss rule on the box [lo, hi] (each a length-3 array).

    Point order: i + p j + p^2 k with i running along x.  Returns points
    (p^3, 3) and weights (p^3,) that include the box volume factor.
    """
    x1, w1 = gauss_1d(p)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    half = (hi - lo) / 2.0
    mid = (hi + lo) / 2.0
    k, j, i = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    pts = np.stack([mid[0] + half[0] * x1[i], mid[1] + half[1] * x1[j],
                    mid[2] + half[2] * x1[k]], axis=1)
    wts = w1[i] * w1[j] * w1[k] * half[0] * half[1] * half[2]
    return pts, wts
