"""General (triclinic) cells on the GPU: the CeAl lattice of Sec. 6.2 (eq.
ceal-primitive) with parallelepiped elements and a constant Jacobian, through
the FP64 path, against the oracle.

* H, S (Gamma and Bloch k), density and adjoint on the CeAl-like cell with
  2^3 and 3^3 elements (Ce-like 4s 4p and Al-like 3s 3p enrichments), and
  on the sheared empty lattice: max |dX| / max |X| <= 1e-12;
* the sheared empty lattice's spectrum from the GPU's matrices: |G|^2 / 2 on
  the reciprocal lattice from above (upper bounds), the constant at 0;
* the mixed-precision calls refuse general cells with PUFE_EINVAL.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as oasm, bloch as ob, eig as oeig, mesh as omesh, potential as opot
from oracle import quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
CASES = {
    "ceal_like_2cube": lambda: W.ceal_like(nel=2),
    "ceal_like_3cube": lambda: W.ceal_like(nel=3, r_e=2.0),
    "sheared_empty_3cube": lambda: W.sheared_empty(nel=3),
}


def _rel(a, b):
    d = a - b
    if sp.issparse(d):
        return max(abs(d).max() / abs(b).max(), sp.linalg.norm(d) / sp.linalg.norm(b))
    return max(np.abs(d).max() / np.abs(b).max(), np.linalg.norm(d) / np.linalg.norm(b))


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    wl = CASES[request.param]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    return request.param, wl, m, rules, ctx


def _csr(ctx, vals):
    rowptr, col = ctx.pattern()
    return sp.csr_matrix((vals, col, rowptr), shape=(ctx.n_dof, ctx.n_dof))


def test_general_cell_assembly_density_adjoint(case):
    name, wl, m, rules, ctx = case
    dev = torch.device("cuda:0")
    V = W.random_potential(len(rules[1]), seed=61)
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(torch.tensor(V, device=dev), H, S)
    ctx.pufe_sync_status()
    Ho, So = oasm.assemble_HS(m, rules, V)
    Hg, Sg = _csr(ctx, H.cpu().numpy()), _csr(ctx, S.cpu().numpy())
    assert _rel(Hg, Ho) < TOL64 and _rel(Sg, So) < TOL64, (name, _rel(Hg, Ho), _rel(Sg, So))
    Cm = W.random_coefficients(m.n_dof, 5, seed=62)
    f = W.random_occupations(5, seed=62)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_density(torch.tensor(Cm, device=dev), torch.tensor(f, device=dev), rho)
    Hbar = Ho.copy()
    Hbar.data = W.random_potential(Ho.nnz, seed=63)
    vbar = torch.empty_like(rho)
    ctx.pufe_assemble_HV_adjoint(torch.tensor(Hbar.data, device=dev), vbar)
    ctx.pufe_sync_status()
    assert _rel(rho.cpu().numpy(), oasm.density(m, rules, Cm, f)) < TOL64, name
    assert _rel(vbar.cpu().numpy(), oasm.adjoint_V(m, rules, Hbar)) < TOL64, name


def test_general_cell_bloch_assembly(case):
    name, wl, m, rules, ctx = case
    dev = torch.device("cuda:0")
    L = np.array(wl["lattice"])
    k = 2.0 * math.pi * np.linalg.inv(L) @ np.array([0.3, -0.2, 0.1])   # general k
    V = W.random_potential(len(rules[1]), seed=64)
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    Hr, Hi, Sr, Si = mk(), mk(), mk(), mk()
    ctx.pufe_assemble_HS_bloch(list(k), torch.tensor(V, device=dev), (Hr, Hi), (Sr, Si))
    ctx.pufe_sync_status()
    rowptr, col = ctx.pattern()
    N = ctx.n_dof
    csr = lambda re, im: sp.csr_matrix((re.cpu().numpy() + 1j * im.cpu().numpy(), col, rowptr),
                                       shape=(N, N))
    Ho, So = ob.assemble_HS_k(m, rules, V, k)
    assert _rel(csr(Hr, Hi), Ho) < TOL64 and _rel(csr(Sr, Si), So) < TOL64, name


def test_sheared_empty_lattice_spectrum_on_gpu():
    wl = W.sheared_empty(nel=4, p=4)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    dev = torch.device("cuda:0")
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(torch.zeros(ctx.n_q, dtype=torch.float64, device=dev), H, S)
    ctx.pufe_sync_status()
    w, _ = oeig.lowest_eigs(_csr(ctx, H.cpu().numpy()), _csr(ctx, S.cpu().numpy()), 7)
    _, G2 = opot.reciprocal_vectors(wl, 4.0)
    exact = np.sort(np.concatenate([[0.0], 0.5 * G2]))[:7]
    assert abs(w[0]) < 1e-12 and np.all(w >= exact - 1e-12)
    assert (w - exact)[1:].max() < 1e-4      # 6.8e-5 at this mesh (oracle)


def test_mixed_precision_refuses_general_cells():
    ctx = pufe.pufe_build_mesh(W.ceal_like(nel=2))
    with pytest.raises(pufe.PufeError) as ex:
        ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    assert ex.value.status == 1
