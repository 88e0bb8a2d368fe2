"""C ABI library checks that need no GPU: exported symbols, error statuses,
and the host-side setup (quadrature rules, numbering, CSR pattern) against
the oracle's independent construction."""
import os
import re

import numpy as np
import pytest

from oracle import assemble as oasm, mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return pufe.load_library()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "pufe.h")).read()
    declared = set(re.findall(r"\b(pufe_[a-zA-Z_0-9]+)\s*\(", hdr))
    assert declared == set(pufe.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_invalid_arguments_report_einval(lib):
    wl = W.small_two_atom(nel=2)
    wl = dict(wl, nel=0)
    with pytest.raises(pufe.PufeError) as ei:
        pufe.pufe_build_mesh(wl)
    assert ei.value.status == 1
    wl = W.small_two_atom(nel=2)
    wl["species"] = [dict(s) for s in wl["species"]]
    wl["species"][1]["orbitals"] = [(2, 2, 0, 1.0)]  # l >= n
    with pytest.raises(pufe.PufeError) as ei:
        pufe.pufe_build_mesh(wl)
    assert ei.value.status == 1
    wl = W.small_two_atom(nel=2)
    wl["quad"] = dict(wl["quad"], mode=7)
    with pytest.raises(pufe.PufeError):
        pufe.pufe_build_mesh(wl)


def _compare(wl):
    ctx = pufe.pufe_build_mesh(wl)
    m = omesh.Mesh(wl)
    pts, wts, off = oq.all_rules(m)
    x, w, goff = ctx.quadrature()
    assert ctx.n_dof == m.n_dof and ctx.n_q == len(wts)
    assert np.array_equal(goff, off)
    assert np.abs(x - pts).max() < 1e-13
    assert np.abs(w - wts).max() < 1e-14 * wts.max() * 10
    n_e, dofs = ctx.element_basis()
    assert np.array_equal(dofs, np.concatenate([m.elem_dofs(e) for e in range(m.nelem)]))
    # CSR pattern: union of element blocks
    H, _ = oasm.assemble_HS(m, (pts, wts, off), np.zeros(len(wts)))
    rowptr, col = ctx.pattern()
    assert np.array_equal(rowptr, H.indptr) and np.array_equal(col, H.indices)
    return ctx


@pytest.mark.parametrize("maker", [
    lambda: W.small_two_atom(nel=2),
    lambda: W.small_two_atom(nel=1, quad_p=3),     # one periodic element: repeated DOFs
    lambda: W.empty_lattice(nel=2),                # no enrichment at all
    lambda: W.workload("c1_two_atom_4cube"),
    lambda: W.ceal_like(nel=2),                    # general (triclinic) cells, Sec. 6.2
    lambda: W.ceal_like(nel=3, r_e=2.0),
    lambda: W.sheared_empty(nel=3),
    # the cubic serendipity FE space (32 nodes per element, Sec. 6)
    lambda: dict(W.small_two_atom(nel=2), fe="serendipity32"),
    lambda: dict(W.small_two_atom(nel=1, quad_p=3), fe="serendipity32"),
    lambda: dict(W.ceal_like(nel=2), fe="serendipity32"),
])
def test_host_setup_matches_oracle(lib, maker):
    _compare(maker())


def test_general_cell_adaptive_rules(lib):
    """p- and h-adaptive rules on the CeAl lattice: mapped reference boxes."""
    for mode in (W.QUAD_PADAPT, W.QUAD_HADAPT):
        wl = W.ceal_like(nel=2)
        wl["quad"] = dict(mode=mode, p_far=4, p_near=8, p_min=4, p_max=8, tol=1e-4, max_depth=1)
        _compare(wl)


def test_host_setup_adaptive_modes(lib):
    # p-adaptive (C2-like cell, 2^3 mesh) and h-adaptive (C3-like, few orbitals)
    wl = W.workload("c2_rocksalt_2cube")
    _compare(wl)
    wl = W.workload("c3_cscl_4cube")
    wl["species"][0]["orbitals"] = wl["species"][0]["orbitals"][:5]
    wl["species"][1]["orbitals"] = wl["species"][1]["orbitals"][:2]
    ctx = _compare(wl)
    q = np.diff(ctx.quadrature()[2])
    assert set(q.tolist()) <= {64, 512, 4096} and 4096 in q


def test_compute_calls_need_a_device_context(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    ctx = pufe.pufe_build_mesh(W.small_two_atom(nel=2))
    assert pufe._LIB.pufe_tabulate(ctx._h, 0, None) == 8  # PUFE_ESTATE
    assert b"without a CUDA device" in pufe._LIB.pufe_last_error()
    # adaptive tests on the device need one: PUFE_ECUDA, no host fallback
    wl = W.workload("c2_rocksalt_2cube")
    wl["quad"] = dict(wl["quad"], device_tests=1)
    with pytest.raises(pufe.PufeError) as ei:
        pufe.pufe_build_mesh(wl)
    assert ei.value.status == 3 and "device_tests" in str(ei.value)
