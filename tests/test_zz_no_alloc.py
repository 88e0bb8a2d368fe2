"""The allocation-free assembly entry point, checked against pufe_assemble_HS.

pufe_assemble_HS_static serves callers that cannot allocate device memory
during their solve loop: its per-call scratch (the FP32 copy of V read by the
tensor-core kernel) lives in a static device array owned by the library.
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MAT_TF32 = 3e-5   # the TF32X3 matrix tolerance of the parity tests


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_static_scratch_assembly_matches_regular_entry_point_twice():
    wl = W.workload("c1_two_atom_4cube")
    ctx = pufe.pufe_build_mesh(wl)
    dev = torch.device("cuda:0")
    H0 = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S0 = torch.empty_like(H0)
    ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    for call, seed in enumerate((21, 22)):   # two calls in a row, different V
        V = torch.tensor(W.random_potential(ctx.n_q, seed=seed), device=dev)
        ctx.pufe_assemble_HS(V, H0, S0, prec=pufe.PUFE_TF32X3)
        H1 = torch.empty_like(H0)
        S1 = torch.empty_like(H0)
        ctx.pufe_assemble_HS_static(V, H1, S1)
        ctx.pufe_sync_status()
        eh = _rel(H1.cpu().numpy(), H0.cpu().numpy())
        es = _rel(S1.cpu().numpy(), S0.cpu().numpy())
        assert eh < TOL_MAT_TF32 and es < TOL_MAT_TF32, (call, eh, es)
