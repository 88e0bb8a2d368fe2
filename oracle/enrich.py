"""Atomic enrichment functions (oracle, test infrastructure).

Sec. 5.1 of the paper builds each enrichment from an isolated-atom orbital
R_nl(r) Y_lm (eq. Psitilde), multiplies the radial part by the C^3 cutoff
h(r, r_c), and sums the periodic images of the atom over lattice vectors
R = i1 a1 + i2 a2 + i3 a3 with i_k = -2..2 (eq. Psi, f(R) = 1 for the
periodic enrichment used with Bloch-phased FE and PU, Sec. 6.2).

Readings taken where the paper leaves a choice (all workloads are synthetic):
* R_nl is a normalised Slater-type orbital N r^(n-1) exp(-zeta r) with
  int R^2 r^2 dr = 1, instead of the paper's spline of a numerical
  pseudo-atomic orbital.
* Y_lm are the real, unit-normalised spherical harmonics without the
  Condon-Shortley phase; m < 0 carries sin(|m| phi), m > 0 cos(m phi).
* The image sum skips images whose distance from the point is >= r_c; the
  cutoff makes those terms exactly zero, so the sum is unchanged.

Gradients are taken by complex-step differentiation of the same code path
(every operation below is complex-analytic on the branch that is taken), so
they are independent of any hand-derived gradient formula.

Pins (tests/test_oracle_enrich.py): cutoff h(0)=1, h(r_c)=0 and C^3
smoothness at both ends; STO normalisation by radial quadrature; Y_lm
orthonormality on the sphere and agreement with SciPy's complex spherical
harmonics; complex-step gradients against central differences; periodicity
of Psi.
"""
from __future__ import annotations

import math

import numpy as np

CSTEP = 1e-30  # complex-step size


def cutoff(r, rc):
    """h(r, r_c) = 1 + 20 x^7 - 70 x^6 + 84 x^5 - 35 x^4 for x = r/r_c <= 1, else 0."""
    x = r / rc
    poly = 1.0 + 20.0 * x ** 7 - 70.0 * x ** 6 + 84.0 * x ** 5 - 35.0 * x ** 4
    return np.where(np.real(x) <= 1.0, poly, 0.0 * poly)


def sto_norm(n, zeta):
    """N such that int_0^inf (N r^(n-1) e^(-zeta r))^2 r^2 dr = 1."""
    return (2.0 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))


def sto_radial(n, zeta, r):
    return sto_norm(n, zeta) * r ** (n - 1) * np.exp(-zeta * r)


def _legendre_deriv_coeffs(l, m):
    """Power-series coefficients of d^m P_l / dt^m (NumPy Legendre class)."""
    P = np.polynomial.legendre.Legendre.basis(l).deriv(m)
    return P.convert(kind=np.polynomial.Polynomial).coef


def real_ylm(l, m, x, y, z):
    """Real spherical harmonic Y_lm at direction (x, y, z) (not normalised).

    Uses P_l^|m|(cos t) sin^|m| ... written as polynomials:
    sin^|m|(theta) cos(|m| phi) = Re((x + i y)^|m|) / r^|m| and likewise Im
    for sin, built by the real recurrence C_{k+1} = x C_k - y S_k,
    S_{k+1} = x S_k + y C_k so that complex-step arguments stay valid.
    """
    r = np.sqrt(x * x + y * y + z * z)
    am = abs(m)
    t = z / r
    coef = _legendre_deriv_coeffs(l, am)
    poly = np.zeros_like(t) + 0.0 * t
    for k in range(len(coef) - 1, -1, -1):  # Horner
        poly = poly * t + coef[k]
    C = np.ones_like(x)
    S = np.zeros_like(x)
    for _ in range(am):
        C, S = x * C - y * S, x * S + y * C
    norm = math.sqrt((2 * l + 1) / (4.0 * math.pi)
                     * math.factorial(l - am) / math.factorial(l + am))
    if m == 0:
        return norm * poly
    trig = C if m > 0 else S
    return math.sqrt(2.0) * norm * poly * trig / r ** am


def orbital_value(orb, rc, d):
    """Psi~_{nlm}(d) h(|d|, r_c) for displacement(s) d (..., 3), no images."""
    n, l, m, zeta = orb
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    r = np.sqrt(x * x + y * y + z * z)
    return sto_radial(n, zeta, r) * cutoff(r, rc) * real_ylm(l, m, x, y, z)


def image_vectors(a, reach=2):
    """Lattice vectors R = i1 a1 + i2 a2 + i3 a3, i_k = -reach..reach (eq. Psi).
    `a` is the cubic edge (a scalar) or the lattice (rows a1, a2, a3)."""
    rng = np.arange(-reach, reach + 1)
    I = np.array(np.meshgrid(rng, rng, rng, indexing="ij")).reshape(3, -1).T.astype(np.float64)
    if np.ndim(a) == 0:
        return a * I
    return I @ np.asarray(a, dtype=np.float64).reshape(3, 3)


def enrichment(orb, rc, tau, a, pts, with_grad=True):
    """Periodic enrichment Psi_alpha and its gradient at points pts (Q, 3).

    Psi(x) = sum_R Psi~(x - tau - R) over R in image_vectors(a) (eq. Psi with
    f(R) = 1).  Terms with |x - tau - R| >= r_c vanish and are skipped.
    Returns (psi (Q,), grad (3, Q)) or psi alone.
    """
    pts = np.asarray(pts, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    psi = np.zeros(pts.shape[0])
    grad = np.zeros((3, pts.shape[0]))
    for R in image_vectors(a):
        d = pts - tau - R
        r = np.sqrt((d * d).sum(axis=1))
        sel = np.nonzero(r < rc)[0]
        if sel.size == 0:
            continue
        ds = d[sel]
        psi[sel] += orbital_value(orb, rc, ds)
        if with_grad:
            for k in range(3):
                dc = ds.astype(np.complex128)
                dc[:, k] += 1j * CSTEP
                grad[k, sel] += np.imag(orbital_value(orb, rc, dc)) / CSTEP
    if with_grad:
        return psi, grad
    return psi
