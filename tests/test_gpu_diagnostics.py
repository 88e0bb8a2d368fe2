"""Failure reporting on the GPU, without a fault: a bounded device wait that
runs out, and a non-finite potential.

The pipelined tensor-core kernels wait on mbarriers with a time limit; the
timeout test runs that same bounded wait on a barrier nothing completes (a
flag that nothing sets) and checks that the context reports PUFE_ETIMEOUT,
clears the flag, and keeps computing correct results afterwards."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as oasm, mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PUFE_EINVAL, PUFE_ETIMEOUT = 1, 6


def _small():
    wl = W.small_two_atom(nel=2, quad_p=4)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    return wl, m, rules, pufe.pufe_build_mesh(wl)


def _assemble(ctx, V, prec):
    dev = torch.device("cuda:0")
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    ctx.pufe_tabulate(prec)
    ctx.pufe_assemble_HS(torch.tensor(V, device=dev), H, S, prec=prec)
    return H, S


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    wl, m, rules, ctx = _small()
    ctx.pufe_selftest_timeout(50_000_000)          # 50 ms, nothing arrives
    with pytest.raises(pufe.PufeError) as ex:
        ctx.pufe_sync_status()
    assert ex.value.status == PUFE_ETIMEOUT
    ctx.pufe_sync_status()                          # the flag was cleared
    V = W.random_potential(len(rules[1]), seed=3)
    H, S = _assemble(ctx, V, pufe.PUFE_FP64)
    ctx.pufe_sync_status()
    Ho, So = oasm.assemble_HS(m, rules, V)
    rowptr, col = ctx.pattern()
    Hg = sp.csr_matrix((H.cpu().numpy(), col, rowptr), shape=Ho.shape)
    assert abs(Hg - Ho).max() < 1e-12 * abs(Ho).max()


def test_wait_limit_is_checked_on_the_host():
    _, _, _, ctx = _small()
    for bad in (0, 10, 3_000_000_000):
        with pytest.raises(pufe.PufeError) as ex:
            ctx.pufe_selftest_timeout(bad)
        assert ex.value.status == PUFE_EINVAL


@pytest.mark.parametrize("prec", [pufe.PUFE_FP64, pufe.PUFE_TF32X3])
def test_nonfinite_potential_is_reported(prec):
    wl, m, rules, ctx = _small()
    for bad in (np.nan, np.inf, -np.inf):
        V = W.random_potential(len(rules[1]), seed=4)
        V[17] = bad
        _assemble(ctx, V, prec)
        with pytest.raises(pufe.PufeError) as ex:
            ctx.pufe_sync_status()
        assert ex.value.status == PUFE_EINVAL
    V = W.random_potential(len(rules[1]), seed=4)
    _assemble(ctx, V, prec)
    ctx.pufe_sync_status()                          # a finite V passes again
