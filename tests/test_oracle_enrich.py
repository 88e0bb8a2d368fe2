"""Pins of the oracle's enrichment functions (CPU only)."""
import math
import os

import numpy as np
import pytest
import scipy.integrate as si

from oracle import enrich

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        out.setdefault(k, []).append([float(x) for x in v])
    return out


def test_cutoff_matches_printed_polynomial_and_factorisation():
    g = _golden()
    coeff = {int(k): c for k, c in g["cutoff_coeff"]}
    rc = 1.7
    r = np.linspace(0, rc, 101)
    x = r / rc
    printed = sum(c * x ** k for k, c in coeff.items())
    assert np.abs(enrich.cutoff(r, rc) - printed).max() < 1e-14
    # closed form: h = (1 - x)^4 (1 + 4x + 10x^2 + 20x^3)  => C^3 at x = 1
    assert np.abs(enrich.cutoff(r, rc) - (1 - x) ** 4 * (1 + 4 * x + 10 * x ** 2 + 20 * x ** 3)).max() < 5e-14
    assert enrich.cutoff(np.array([rc * 1.0001, 5.0]), rc).tolist() == [0.0, 0.0]
    # flat to third order at r = 0: (h(d) - 1) / d^4 stays bounded (-> -35 / rc^4)
    d = np.array([1e-2, 1e-3]) * rc
    assert np.allclose((enrich.cutoff(d, rc) - 1) / (d / rc) ** 4, -35, rtol=1e-1)


@pytest.mark.parametrize("n,zeta", [(1, 1.0), (2, 0.65), (3, 1.1667), (4, 3.0)])
def test_sto_normalised(n, zeta):
    val, _ = si.quad(lambda r: enrich.sto_radial(n, zeta, r) ** 2 * r * r, 0, np.inf)
    assert abs(val - 1.0) < 1e-10


def _sphere_rule(L):
    ct, wt = np.polynomial.legendre.leggauss(L + 1)
    nphi = 2 * L + 2
    phi = 2 * np.pi * np.arange(nphi) / nphi
    CT, PH = np.meshgrid(ct, phi, indexing="ij")
    W = np.outer(wt, np.full(nphi, 2 * np.pi / nphi))
    st = np.sqrt(1 - CT ** 2)
    return st * np.cos(PH), st * np.sin(PH), CT, W


def test_real_ylm_orthonormal_l_le_3():
    x, y, z, w = _sphere_rule(8)
    lm = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    Y = np.array([enrich.real_ylm(l, m, x, y, z).ravel() for l, m in lm])
    gram = (Y * w.ravel()) @ Y.T
    assert np.abs(gram - np.eye(len(lm))).max() < 1e-13


def test_real_ylm_closed_forms_l1():
    rng = np.random.default_rng(3)
    p = rng.normal(size=(20, 3))
    r = np.linalg.norm(p, axis=1)
    c = math.sqrt(3 / (4 * math.pi))
    x, y, z = p.T
    assert np.allclose(enrich.real_ylm(1, -1, x, y, z), c * y / r, atol=1e-15)
    assert np.allclose(enrich.real_ylm(1, 0, x, y, z), c * z / r, atol=1e-15)
    assert np.allclose(enrich.real_ylm(1, 1, x, y, z), c * x / r, atol=1e-15)
    assert np.allclose(enrich.real_ylm(0, 0, x, y, z), 0.5 / math.sqrt(math.pi))


def test_real_ylm_against_scipy_complex():
    sps = pytest.importorskip("scipy.special")
    fn = getattr(sps, "sph_harm_y", None)
    if fn is None:
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(4)
    p = rng.normal(size=(30, 3))
    x, y, z = p.T
    r = np.linalg.norm(p, axis=1)
    theta = np.arccos(z / r)
    phi = np.arctan2(y, x)
    for l in range(4):
        for m in range(-l, l + 1):
            Yc = fn(l, abs(m), theta, phi)  # includes the Condon-Shortley phase
            if m > 0:
                ref = math.sqrt(2) * (-1) ** m * Yc.real
            elif m < 0:
                ref = math.sqrt(2) * (-1) ** m * Yc.imag
            else:
                ref = Yc.real
            assert np.abs(enrich.real_ylm(l, m, x, y, z) - ref).max() < 1e-13


@pytest.mark.parametrize("orb", [(1, 0, 0, 2.7), (2, 1, -1, 0.65), (3, 2, 1, 1.5), (4, 3, -2, 3.0)])
def test_gradient_matches_central_difference_and_periodic(orb):
    a, rc = 4.0, 1.5
    tau = np.array([2.0, 2.0, 2.0])
    rng = np.random.default_rng(5)
    pts = tau + rng.uniform(-1.4, 1.4, size=(40, 3)) / np.sqrt(3)
    psi, g = enrich.enrichment(orb, rc, tau, a, pts)
    eps = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        fd = (enrich.enrichment(orb, rc, tau, a, pts + e, False)
              - enrich.enrichment(orb, rc, tau, a, pts - e, False)) / (2 * eps)
        assert np.abs(fd - g[k]).max() < 1e-6 * max(1.0, np.abs(g[k]).max())
    # periodic enrichment (f(R) = 1): Psi(x + a e_k) = Psi(x)
    for k in range(3):
        sh = np.zeros(3)
        sh[k] = a
        assert np.abs(enrich.enrichment(orb, rc, tau, a, pts + sh, False) - psi).max() < 1e-14


def test_image_reach_is_the_printed_one():
    g = _golden()
    reach = int(g["image_reach"][0][0])
    assert len(enrich.image_vectors(1.0)) == (2 * reach + 1) ** 3
