"""Adaptive quadrature rules built with their tests on the GPU (Sec. 5.2).

`pufe_quad.device_tests = 1` evaluates the integrals of the p-adaptive and
the recursive 5^3-against-8^3 tests (Psi^2 and |grad Psi|^2 of every
enrichment of a box) on the device.  The rule must be the one the host
construction and the oracle build: the same point count per element (the
decisions), the same points and weights.
"""
import time

import numpy as np
import pytest

from oracle import mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

pytestmark = pytest.mark.gpu


def _build(wl, device_tests):
    wl = dict(wl, quad=dict(wl["quad"], device_tests=device_tests))
    t0 = time.perf_counter()
    ctx = pufe.pufe_build_mesh(wl)
    return ctx, time.perf_counter() - t0


def _small_cases():
    c3 = W.workload("c3_cscl_4cube")
    c3["species"] = [dict(s) for s in c3["species"]]
    c3["species"][0]["orbitals"] = c3["species"][0]["orbitals"][:5]
    c3["species"][1]["orbitals"] = c3["species"][1]["orbitals"][:2]
    cases = [W.workload("c2_rocksalt_2cube"), c3]
    for mode in (W.QUAD_PADAPT, W.QUAD_HADAPT):   # general (triclinic) cell
        wl = W.ceal_like(nel=2)
        wl["quad"] = dict(mode=mode, p_far=4, p_near=8, p_min=4, p_max=8, tol=1e-4, max_depth=1)
        cases.append(wl)
    return cases


@pytest.mark.parametrize("k", range(4))
def test_device_tests_match_oracle_rules(k):
    wl = _small_cases()[k]
    ctx, _ = _build(wl, 1)
    pts, wts, off = oq.all_rules(omesh.Mesh(wl))
    x, w, goff = ctx.quadrature()
    assert np.array_equal(goff, off)   # every element's decisions
    assert np.abs(x - pts).max() < 1e-13
    assert np.abs(w - wts).max() < 1e-13 * wts.max()


@pytest.mark.parametrize("name", ["c2_rocksalt_12cube", "c3_cscl_16cube"])
def test_device_tests_match_host_rules_full_size(name):
    wl = W.workload(name)
    hctx, th = _build(wl, 0)
    dctx, td = _build(wl, 1)
    xh, wh, oh = hctx.quadrature()
    xd, wd, od = dctx.quadrature()
    assert np.array_equal(oh, od)
    # same decisions -> the same host emission of points and weights
    assert np.array_equal(xh, xd) and np.array_equal(wh, wd)
    sizes = np.diff(od)
    print(f"\n{name}: {len(wd)} points, element sizes {sorted(set(sizes.tolist()))}; "
          f"setup with host tests {th:.2f} s, with device tests {td:.2f} s")
