"""The allocation-free assembly entry point, checked against pufe_assemble_HS.

pufe_assemble_HS_static serves callers that cannot allocate device memory
during their solve loop (a fixed device-memory budget, or code that runs
where the allocator must not be called): its per-call scratch (the FP32 copy
of V read by the tensor-core kernel of elements with more than 128 basis
functions) lives in a static device array owned by the library.  The cell
with such elements is the one that reads the array; the two-atom cell, which
has none, checks that the call also serves contexts that never touch it.
Both entry points run the same kernels on the same inputs; every element
block is formed in a fixed order, so the results differ only by the order in
which the FP64 atomic additions of different elements land (a few ulp).  This file
is collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_ORDER = 1e-12   # FP64 atomic-ordering differences, relative to max |X|


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _large_element_cell():
    """CsCl-like 4^3 cell whose heavy-atom elements carry more than 128
    basis functions (the tensor-core tile, which reads the scratch)."""
    wl = W.workload("c3_cscl_4cube")
    wl["species"][0]["orbitals"] = [o for o in wl["species"][0]["orbitals"] if o[0] >= 3]
    wl["species"][0]["r_e"] = 1.5
    wl["quad"] = dict(wl["quad"], mode=W.QUAD_FIXED, p_far=5, p_near=5)
    return wl


@pytest.mark.parametrize("name", ["large_elements", "c1_two_atom_4cube"])
def test_static_scratch_assembly_matches_regular_entry_point_twice(name):
    wl = _large_element_cell() if name == "large_elements" else W.workload(name)
    ctx = pufe.pufe_build_mesh(wl)
    n_e, _ = ctx.element_basis()
    if name == "large_elements":
        assert int((np.asarray(n_e) > 128).sum()) > 0
    dev = torch.device("cuda:0")
    H0 = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S0 = torch.empty_like(H0)
    H1 = torch.empty_like(H0)
    S1 = torch.empty_like(H0)
    ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    V0 = torch.tensor(W.random_potential(ctx.n_q, seed=20), device=dev)
    ctx.pufe_assemble_HS_static(V0, H1, S1)     # first call: address lookup
    ctx.pufe_sync_status()
    for call, seed in enumerate((21, 22)):      # two calls in a row, different V
        V = torch.tensor(W.random_potential(ctx.n_q, seed=seed), device=dev)
        # the regular path last saw another V, so its own scratch holds other data
        Vx = torch.tensor(W.random_potential(ctx.n_q, seed=100 + seed), device=dev)
        ctx.pufe_assemble_HS(Vx, H0, S0, prec=pufe.PUFE_TF32X3)
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        ctx.pufe_assemble_HS_static(V, H1, S1)
        ctx.pufe_sync_status()
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after == free_before, (name, call, free_before - free_after)
        ctx.pufe_assemble_HS(V, H0, S0, prec=pufe.PUFE_TF32X3)
        ctx.pufe_sync_status()
        eh = _rel(H1.cpu().numpy(), H0.cpu().numpy())
        es = _rel(S1.cpu().numpy(), S0.cpu().numpy())
        assert eh < TOL_ORDER and es < TOL_ORDER, (name, call, eh, es)
