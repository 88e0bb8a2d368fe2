"""1D PUFE L2-projection of the supplementary material (oracle pin).

Domain [-pi, pi], seven nodes x = -pi, -2, -1, 0, 1, 2, pi, linear hats
phi_i serving both as FE basis and partition of unity, one enrichment
Psi(x) = exp(-a x^2) cos(b x); target u = Psi + delta with
delta = c (1 + d x^2) cos(x - 0.5), a = 1.3, b = 2.9, c = -0.15, d = 0.25.
The 14 coefficients solve M c = f with M_ij = (phi_i, phi_j),
f_i = (phi_i, u) over the 14 PUFE functions.

Used as a pin of the PU mechanism: with u = Psi the projection reproduces
Psi to round-off (b_i = 1, u_i = 0), and with the perturbation the PUFE
error is far below the plain FE error (the paper shows this as a figure).
"""
from __future__ import annotations

import numpy as np

NODES = np.array([-np.pi, -2.0, -1.0, 0.0, 1.0, 2.0, np.pi])
A, B, C, D = 1.3, 2.9, -0.15, 0.25


def psi(x):
    return np.exp(-A * x * x) * np.cos(B * x)


def delta(x):
    return C * (1.0 + D * x * x) * np.cos(x - 0.5)


def hats(x):
    """Values of the 7 linear hats at points x (len(x), 7)."""
    out = np.zeros((len(x), len(NODES)))
    for i, xi in enumerate(NODES):
        if i > 0:
            xl = NODES[i - 1]
            m = (x >= xl) & (x <= xi)
            out[m, i] = (x[m] - xl) / (xi - xl)
        if i < len(NODES) - 1:
            xr = NODES[i + 1]
            m = (x >= xi) & (x <= xr)
            out[m, i] = (xr - x[m]) / (xr - xi)
    return out


def quadrature(p=40):
    """p-point Gauss rule on each of the six elements."""
    g, w = np.polynomial.legendre.leggauss(p)
    xs, ws = [], []
    for l, r in zip(NODES[:-1], NODES[1:]):
        xs.append((l + r) / 2 + (r - l) / 2 * g)
        ws.append((r - l) / 2 * w)
    return np.concatenate(xs), np.concatenate(ws)


def project(u, enriched=True, p=40):
    """Coefficients c and the L2 error of the projection of u."""
    x, w = quadrature(p)
    H = hats(x)
    basis = np.concatenate([H, H * psi(x)[:, None]], axis=1) if enriched else H
    M = basis.T @ (w[:, None] * basis)
    f = basis.T @ (w * u(x))
    c = np.linalg.solve(M, f)
    err = np.sqrt(w @ (basis @ c - u(x)) ** 2)
    return c, err
