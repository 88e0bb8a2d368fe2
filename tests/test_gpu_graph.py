"""The hot path captured into a CUDA graph: every call of the step is a plain
stream-ordered launch sequence (no host synchronisation, no allocation), so a
graph captured once and replayed with new inputs gives the results of the
direct calls, up to the order of the atomic additions: FP64 partial sums in
FP64 mode (1e-12), FP32 partial sums in the mixed mode (whose element blocks
are formed in FP32, 1e-6)."""
import numpy as np
import pytest

from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("prec", [pufe.PUFE_FP64, pufe.PUFE_TF32X3])
def test_graph_replay_matches_direct_calls(prec):
    dev = torch.device("cuda:0")
    wl = W.workload("c1_two_atom_4cube")
    ctx = pufe.pufe_build_mesh(wl)
    nocc = 3
    V = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    Cm = torch.empty(ctx.n_dof, nocc, dtype=torch.float64, device=dev)
    f = torch.empty(nocc, dtype=torch.float64, device=dev)
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    vbar = torch.empty_like(rho)

    def load(seed):
        V.copy_(torch.tensor(W.random_potential(ctx.n_q, seed=seed)))
        Cm.copy_(torch.tensor(W.random_coefficients(ctx.n_dof, nocc, seed=seed)))
        f.copy_(torch.tensor(W.random_occupations(nocc, seed=seed)))

    def step():
        ctx.pufe_tabulate(prec)
        ctx.pufe_assemble_HS(V, H, S, prec=prec)
        ctx.pufe_density(Cm, f, rho, prec=prec)
        ctx.pufe_assemble_HV_adjoint(H, vbar, prec=prec)

    load(1)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    torch.cuda.synchronize()
    ctx.pufe_sync_status()

    load(2)
    step()
    torch.cuda.synchronize()
    ref = [t.clone() for t in (H, S, rho, vbar)]
    for t in (H, S, rho, vbar):
        t.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    ctx.pufe_sync_status()
    for got, want in zip((H, S, rho, vbar), ref):
        assert torch.isfinite(got).all()
        assert _rel(got, want) < (1e-12 if prec == pufe.PUFE_FP64 else 1e-6)
