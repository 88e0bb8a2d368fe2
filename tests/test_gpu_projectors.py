"""GPU parity of the nonlocal projections (pufe_nonlocal_projections) with the
oracle (oracle/projectors.py), FP64, max |error| / max |F| <= 1e-12."""
import numpy as np
import pytest

from oracle import mesh as omesh, projectors as onl, quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "two_atom_2cube": lambda: W.small_two_atom(nel=2, quad_p=6),
    "one_element": lambda: W.small_two_atom(nel=1, quad_p=5),
    "c1_two_atom_4cube": lambda: W.workload("c1_two_atom_4cube"),
}


def _projs(wl):
    out = []
    for i, (_, tau) in enumerate(wl["atoms"]):
        rp = 0.6 + 0.2 * i
        out.append(dict(tau=tau, l=0, m=0, rp=rp))
        out += [dict(tau=tau, l=1, m=m, rp=rp) for m in (-1, 0, 1)]
        out.append(dict(tau=tau, l=2, m=1, rp=rp))
        out.append(dict(tau=tau, l=3, m=-2, rp=1.1 * rp))
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_projections_match_oracle(name):
    wl = CASES[name]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    ps = _projs(wl)
    Fo = onl.projections(m, rules, ps)
    F = torch.empty(ctx.n_dof, len(ps), dtype=torch.float64, device="cuda:0")
    ctx.pufe_nonlocal_projections(ps, F)
    ctx.pufe_sync_status()
    Fg = F.cpu().numpy()
    assert np.abs(Fg - Fo).max() < 1e-12 * np.abs(Fo).max(), name
