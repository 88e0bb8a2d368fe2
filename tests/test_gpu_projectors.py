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


def test_nonlocal_term_in_the_eigenproblem():
    """C1 with a separable nonlocal term: eigenvalues of H + F h F^T (GPU H
    and F) against the oracle's, and the term shifts the spectrum."""
    import scipy.linalg as sla
    import scipy.sparse as sp

    from oracle import assemble as oasm
    wl = W.workload("c1_two_atom_4cube")
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    dev = torch.device("cuda:0")
    V = W.random_potential(len(rules[1]), seed=31)
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(torch.tensor(V, device=dev), H, S)
    ps = _projs(wl)[:8]
    F = torch.empty(ctx.n_dof, len(ps), dtype=torch.float64, device=dev)
    ctx.pufe_nonlocal_projections(ps, F)
    ctx.pufe_sync_status()
    h = np.linspace(0.5, 1.5, len(ps))
    rowptr, col = ctx.pattern()
    N = ctx.n_dof
    Hg = sp.csr_matrix((H.cpu().numpy(), col, rowptr), shape=(N, N)).toarray()
    Sg = sp.csr_matrix((S.cpu().numpy(), col, rowptr), shape=(N, N)).toarray()
    Fg = F.cpu().numpy()
    wg = sla.eigh(Hg + Fg @ np.diag(h) @ Fg.T, Sg, eigvals_only=True, subset_by_index=[0, 5])
    Ho, So = oasm.assemble_HS(m, rules, V)
    Fo = onl.projections(m, rules, ps)
    wo = sla.eigh(Ho.toarray() + Fo @ np.diag(h) @ Fo.T, So.toarray(), eigvals_only=True,
                  subset_by_index=[0, 5])
    w0 = sla.eigh(Ho.toarray(), So.toarray(), eigvals_only=True, subset_by_index=[0, 5])
    assert np.abs(wg - wo).max() < 1e-10
    assert np.all(wo >= w0 - 1e-12) and (wo - w0).max() > 1e-3   # h > 0 raises the levels


@pytest.mark.parametrize("name", ["two_atom_2cube", "c1_two_atom_4cube"])
def test_bloch_projections_match_oracle(name):
    """F(k) at a general k (images and element columns phased) against the
    oracle's complex F, and k = 0 against the Gamma-point call."""
    wl = CASES[name]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    ps = _projs(wl)
    dev = torch.device("cuda:0")
    k = 2.0 * np.pi / m.a * np.array([0.25, -0.125, 0.375])
    Fo = onl.projections_k(m, rules, ps, k)
    Fr = torch.empty(ctx.n_dof, len(ps), dtype=torch.float64, device=dev)
    Fi = torch.empty_like(Fr)
    ctx.pufe_nonlocal_projections_bloch(k, ps, (Fr, Fi))
    ctx.pufe_sync_status()
    Fg = Fr.cpu().numpy() + 1j * Fi.cpu().numpy()
    assert np.abs(Fg - Fo).max() < 1e-12 * np.abs(Fo).max(), name
    F0 = torch.empty_like(Fr)
    ctx.pufe_nonlocal_projections(ps, F0)
    ctx.pufe_nonlocal_projections_bloch((0.0, 0.0, 0.0), ps, (Fr, Fi))
    ctx.pufe_sync_status()
    assert np.abs(Fi.cpu().numpy()).max() == 0.0
    assert np.abs(Fr.cpu().numpy() - F0.cpu().numpy()).max() < 1e-14 * np.abs(Fo).max()
