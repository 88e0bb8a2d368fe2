"""Local ionic potential of Gaussian charges in a periodic cell (oracle).

Sec. 3 of the paper: the ionic potentials decay as Z_a / r and can be
generated by localized ionic charge densities rho_I,a.  The workloads use
the Gaussian charge Z e^{-r^2/sigma^2} / (pi^{3/2} sigma^3), whose isolated
potential is -Z erf(r / sigma) / r.  Its periodic sum in a cell of volume
Omega, with the G = 0 term dropped (a neutralising background), is

    V_I(x) = -(4 pi / Omega) sum_{G != 0} sum_a Z_a e^{-G^2 sigma_a^2 / 4}
             cos(G . (x - tau_a)) / G^2 ,

summed until the Gaussian factor falls below 1e-18, G on the reciprocal
lattice of the cell (the cubic cell a I, or a general cell given by its
lattice vectors).

Pins (tests/test_oracle_potential.py): the FD Laplacian of V_I equals
4 pi (rho_I - <rho_I>) (Poisson, Sec. 3 eq. poisson); V_I near an isolated
ion in a large cell matches -Z erf(r/sigma)/r up to a constant.
"""
from __future__ import annotations

import math

import numpy as np


def _lattice(wl):
    """Rows a_1, a_2, a_3 of the cell (the cubic cell a I unless given)."""
    if "lattice" in wl:
        return np.array(wl["lattice"], dtype=np.float64).reshape(3, 3)
    return float(wl["a"]) * np.eye(3)


def reciprocal_vectors(wl, gmax):
    """Nonzero G = 2 pi L^-1 m (m integer) with |G| <= gmax, and |G|^2.  The
    m range per axis follows from G . a_k = 2 pi m_k: |m_k| <= gmax |a_k| / 2 pi."""
    L = _lattice(wl)
    B = 2.0 * math.pi * np.linalg.inv(L)          # columns b_k, a_i . b_k = 2 pi delta_ik
    mm = [int(math.ceil(gmax * np.linalg.norm(L[k]) / (2.0 * math.pi))) for k in range(3)]
    M = np.array(np.meshgrid(*[np.arange(-m, m + 1) for m in mm], indexing="ij")).reshape(3, -1).T
    M = M[(M != 0).any(axis=1)]
    G = M.astype(np.float64) @ B.T
    G2 = (G * G).sum(axis=1)
    keep = G2 <= gmax * gmax
    return G[keep], G2[keep]


def ionic_potential(wl, pts):
    L = _lattice(wl)
    Omega = abs(float(np.linalg.det(L)))
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    out = np.zeros(pts.shape[0])
    if not wl["atoms"]:
        return out
    sig_min = min(wl["species"][s]["sigma"] for s, _ in wl["atoms"])
    # e^{-G^2 s^2/4} < 1e-18  <=>  G > sqrt(4 * 18 ln 10) / s
    gmax = math.sqrt(4.0 * 18.0 * math.log(10.0)) / sig_min
    G, G2 = reciprocal_vectors(wl, gmax)
    for s, tau in wl["atoms"]:
        sp = wl["species"][s]
        amp = -(4.0 * math.pi / Omega) * sp["Z"] * np.exp(-G2 * sp["sigma"] ** 2 / 4.0) / G2
        for i in range(0, pts.shape[0], 512):   # blocks of points bound the memory
            phase = (pts[i:i + 512] - np.asarray(tau)) @ G.T
            out[i:i + 512] += np.cos(phase) @ amp
    return out


def gaussian_charge(wl, pts):
    """Total periodic ionic charge density sum_a Z_a e^{-r^2/s^2}/(pi^1.5 s^3)."""
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    out = np.zeros(pts.shape[0])
    rng = np.arange(-2, 3)
    R = np.array(np.meshgrid(rng, rng, rng, indexing="ij")).reshape(3, -1).T @ _lattice(wl)
    for s, tau in wl["atoms"]:
        sp = wl["species"][s]
        for r in R:
            d = pts - np.asarray(tau) - r
            r2 = (d * d).sum(axis=1)
            out += sp["Z"] * np.exp(-r2 / sp["sigma"] ** 2) / (math.pi ** 1.5 * sp["sigma"] ** 3)
    return out


def ionic_potential_ewald(wl, pts, eta=1.5):
    """The same V_I, evaluated by Ewald's splitting (Ewald 1921) so that large
    point sets are affordable.

    Each Gaussian ion's potential -Z erf(r/s)/r is split at a wider Gaussian
    width eta > s into a short-range part -Z (erf(r/s) - erf(r/eta))/r, summed
    over images in real space, and -Z erf(r/eta)/r, whose reciprocal sum
    converges after far fewer G vectors.  The short-range part has the mean
    -pi Z (eta^2 - s^2) / Omega over the cell (its G = 0 Fourier term); V_I
    drops every G = 0 term, so that mean is added back with the opposite sign:

        V_I = sum_a [ sum_R -Z_a (erf(r/s_a) - erf(r/eta)) / r
                      + pi Z_a (eta^2 - s_a^2) / Omega ]
              - (4 pi / Omega) sum_{G != 0} e^{-G^2 eta^2 / 4} / G^2
                    Re( e^{i G.x} sum_a Z_a e^{-i G.tau_a} ).

    Real-space terms are kept while erfc(r/eta) > 1e-20 (r < 6.6 eta), the
    reciprocal ones while e^{-G^2 eta^2/4} > 1e-18.  Pinned against
    ``ionic_potential`` at random points (tests/test_oracle_misc.py).
    """
    from scipy.special import erf

    a = float(wl["a"])
    Omega = a ** 3
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    out = np.zeros(pts.shape[0])
    if not wl["atoms"]:
        return out
    for _, sp in enumerate(wl["species"]):
        if wl["atoms"] and sp["sigma"] >= eta:
            raise ValueError("eta must exceed every sigma")
    rcut = 6.6 * eta
    reach = int(math.ceil(rcut / a))
    rng = np.arange(-reach, reach + 1)
    R = a * np.array(np.meshgrid(rng, rng, rng, indexing="ij")).reshape(3, -1).T
    # real space: displacements from the nearest image, then the shells around it
    for s, tau in wl["atoms"]:
        sp = wl["species"][s]
        Z, sg = sp["Z"], sp["sigma"]
        d0 = pts - np.asarray(tau)
        d0 -= a * np.round(d0 / a)
        for r_ in R:
            d = d0 + r_
            r = np.sqrt((d * d).sum(axis=1))
            sel = np.nonzero(r < rcut)[0]
            if sel.size == 0:
                continue
            rs = r[sel]
            small = rs < 1e-12
            rs_safe = np.where(small, 1.0, rs)
            val = np.where(small, 2.0 / math.sqrt(math.pi) * (1.0 / sg - 1.0 / eta),
                           (erf(rs_safe / sg) - erf(rs_safe / eta)) / rs_safe)
            out[sel] += -Z * val
        out += math.pi * Z * (eta ** 2 - sg ** 2) / Omega
    # reciprocal space with the structure factor of the atoms
    gmax = math.sqrt(4.0 * 18.0 * math.log(10.0)) / eta
    mmax = int(math.ceil(gmax * a / (2.0 * math.pi)))
    rg = np.arange(-mmax, mmax + 1)
    M = np.array(np.meshgrid(rg, rg, rg, indexing="ij")).reshape(3, -1).T
    M = M[(M != 0).any(axis=1)]
    G = (2.0 * math.pi / a) * M.astype(np.float64)
    G2 = (G * G).sum(axis=1)
    keep = G2 <= gmax * gmax
    G, G2 = G[keep], G2[keep]
    sf = np.zeros(len(G), dtype=np.complex128)
    for s, tau in wl["atoms"]:
        sf += wl["species"][s]["Z"] * np.exp(-1j * (G @ np.asarray(tau)))
    amp = -(4.0 * math.pi / Omega) * np.exp(-G2 * eta ** 2 / 4.0) / G2
    ar, ai = amp * sf.real, amp * sf.imag
    for i in range(0, pts.shape[0], 512):
        phase = pts[i:i + 512] @ G.T
        out[i:i + 512] += np.cos(phase) @ ar - np.sin(phase) @ ai
    return out
