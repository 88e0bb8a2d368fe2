"""Local ionic potential of Gaussian charges in a periodic cubic cell (oracle).

Sec. 3 of the paper: the ionic potentials decay as Z_a / r and can be
generated by localized ionic charge densities rho_I,a.  The workloads use
the Gaussian charge Z e^{-r^2/sigma^2} / (pi^{3/2} sigma^3), whose isolated
potential is -Z erf(r / sigma) / r.  Its periodic sum in a cell of volume
Omega, with the G = 0 term dropped (a neutralising background), is

    V_I(x) = -(4 pi / Omega) sum_{G != 0} sum_a Z_a e^{-G^2 sigma_a^2 / 4}
             cos(G . (x - tau_a)) / G^2 ,

summed until the Gaussian factor falls below 1e-18.

Pins (tests/test_oracle_potential.py): the FD Laplacian of V_I equals
4 pi (rho_I - <rho_I>) (Poisson, Sec. 3 eq. poisson); V_I near an isolated
ion in a large cell matches -Z erf(r/sigma)/r up to a constant.
"""
from __future__ import annotations

import math

import numpy as np


def ionic_potential(wl, pts):
    a = float(wl["a"])
    Omega = a ** 3
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    out = np.zeros(pts.shape[0])
    if not wl["atoms"]:
        return out
    sig_min = min(wl["species"][s]["sigma"] for s, _ in wl["atoms"])
    # e^{-G^2 s^2/4} < 1e-18  <=>  G > sqrt(4 * 18 ln 10) / s
    gmax = math.sqrt(4.0 * 18.0 * math.log(10.0)) / sig_min
    mmax = int(math.ceil(gmax * a / (2.0 * math.pi)))
    rng = np.arange(-mmax, mmax + 1)
    M = np.array(np.meshgrid(rng, rng, rng, indexing="ij")).reshape(3, -1).T
    M = M[(M != 0).any(axis=1)]
    G = (2.0 * math.pi / a) * M.astype(np.float64)
    G2 = (G * G).sum(axis=1)
    keep = G2 <= gmax * gmax
    G, G2 = G[keep], G2[keep]
    for s, tau in wl["atoms"]:
        sp = wl["species"][s]
        amp = -(4.0 * math.pi / Omega) * sp["Z"] * np.exp(-G2 * sp["sigma"] ** 2 / 4.0) / G2
        for i in range(0, pts.shape[0], 512):   # blocks of points bound the memory
            phase = (pts[i:i + 512] - np.asarray(tau)) @ G.T
            out[i:i + 512] += np.cos(phase) @ amp
    return out


def gaussian_charge(wl, pts):
    """Total periodic ionic charge density sum_a Z_a e^{-r^2/s^2}/(pi^1.5 s^3)."""
    a = float(wl["a"])
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    out = np.zeros(pts.shape[0])
    rng = np.arange(-2, 3)
    R = a * np.array(np.meshgrid(rng, rng, rng, indexing="ij")).reshape(3, -1).T
    for s, tau in wl["atoms"]:
        sp = wl["species"][s]
        for r in R:
            d = pts - np.asarray(tau) - r
            r2 = (d * d).sum(axis=1)
            out += sp["Z"] * np.exp(-r2 / sp["sigma"] ** 2) / (math.pi ** 1.5 * sp["sigma"] ** 3)
    return out
