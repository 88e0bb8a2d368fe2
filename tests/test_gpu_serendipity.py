"""GPU parity of the FP64 path on the cubic serendipity FE space (32 nodes per
element, the classical FE part of the paper's PUFE runs, Sec. 6) against the
oracle, through the C ABI: H and S, the density, the adjoint, and their Bloch
forms at a wavevector; cubic and general (triclinic) cells; max |error| /
max |X| <= 1e-12.  The mixed, SCF and projector calls refuse the space."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import assemble as oasm, bloch as ob, mesh as omesh, potential as opot
from oracle import quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
K_FRAC = np.array([0.3, -0.2, 0.1])

CASES = {
    "two_atom_2cube": lambda: dict(W.small_two_atom(nel=2, quad_p=6), fe="serendipity32"),
    "one_element": lambda: dict(W.small_two_atom(nel=1, quad_p=5), fe="serendipity32"),
    "c1_two_atom_4cube": lambda: dict(W.workload("c1_two_atom_4cube"), fe="serendipity32"),
    "ceal_like_2cube": lambda: dict(W.ceal_like(nel=2), fe="serendipity32"),
}


def _rel(a, b):
    d = a - b
    if sp.issparse(d):
        return float(abs(d).max() / abs(b).max())
    return float(np.abs(d).max() / np.abs(b).max())


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    wl = CASES[request.param]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    return request.param, wl, m, rules, ctx


def _csr(ctx, re, im=None):
    rowptr, col = ctx.pattern()
    v = re.cpu().numpy() if im is None else re.cpu().numpy() + 1j * im.cpu().numpy()
    return sp.csr_matrix((v, col, rowptr), shape=(ctx.n_dof, ctx.n_dof))


def test_assembly_density_adjoint_match_oracle(case):
    name, wl, m, rules, ctx = case
    assert m.nfe_e == 32 and ctx.n_dof == m.n_dof
    dev = torch.device("cuda:0")
    V = W.random_potential(len(rules[1]), seed=41)
    Ho, So = oasm.assemble_HS(m, rules, V)
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(torch.tensor(V, device=dev), H, S)
    Cm = W.random_coefficients(m.n_dof, 7, seed=42)
    f = W.random_occupations(7, seed=42)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_density(torch.tensor(Cm, device=dev), torch.tensor(f, device=dev), rho)
    Hbar = Ho.copy()
    Hbar.data = W.random_symmetric_values(Ho.nnz, seed=43)
    vbar = torch.empty_like(rho)
    ctx.pufe_assemble_HV_adjoint(torch.tensor(Hbar.data, device=dev), vbar)
    ctx.pufe_sync_status()
    assert _rel(_csr(ctx, H), Ho) < TOL and _rel(_csr(ctx, S), So) < TOL, name
    assert _rel(rho.cpu().numpy(), oasm.density(m, rules, Cm, f)) < TOL, name
    assert _rel(vbar.cpu().numpy(), oasm.adjoint_V(m, rules, Hbar)) < TOL, name


def test_bloch_calls_match_oracle(case):
    name, wl, m, rules, ctx = case
    dev = torch.device("cuda:0")
    if m.general:
        k = 2.0 * math.pi * np.linalg.solve(np.asarray(wl["lattice"]), K_FRAC)
    else:
        k = 2.0 * math.pi / wl["a"] * K_FRAC
    V = W.random_potential(len(rules[1]), seed=44)
    Ho, So = ob.assemble_HS_k(m, rules, V, k)
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    Hr, Hi, Sr, Si = mk(), mk(), mk(), mk()
    ctx.pufe_assemble_HS_bloch(k, torch.tensor(V, device=dev), (Hr, Hi), (Sr, Si))
    rng = np.random.default_rng(45)
    C = rng.standard_normal((m.n_dof, 5)) + 1j * rng.standard_normal((m.n_dof, 5))
    f = W.random_occupations(5, seed=45)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_density_bloch(k, torch.tensor(np.ascontiguousarray(C.real), device=dev),
                           torch.tensor(np.ascontiguousarray(C.imag), device=dev),
                           torch.tensor(f, device=dev), rho)
    Hbar = Ho.copy()
    Hbar.data = rng.standard_normal(Ho.nnz) + 1j * rng.standard_normal(Ho.nnz)
    vbar = torch.empty_like(rho)
    ctx.pufe_assemble_HV_adjoint_bloch(k, torch.tensor(Hbar.data.real.copy(), device=dev),
                                       torch.tensor(Hbar.data.imag.copy(), device=dev), vbar)
    ctx.pufe_sync_status()
    assert _rel(_csr(ctx, Hr, Hi), Ho) < TOL and _rel(_csr(ctx, Sr, Si), So) < TOL, name
    assert _rel(rho.cpu().numpy(), ob.density_k(m, rules, C, f, k)) < TOL, name
    assert _rel(vbar.cpu().numpy(), ob.adjoint_V_k(m, rules, Hbar, k)) < TOL, name


def test_c1_eigenvalues_in_the_serendipity_basis():
    """C1's four lowest states in the PUFE basis on the serendipity space
    from the GPU's matrices against the oracle's (1e-10 Ha)."""
    wl = CASES["c1_two_atom_4cube"]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    dev = torch.device("cuda:0")
    V = opot.ionic_potential(wl, rules[0])
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(torch.tensor(V, device=dev), H, S)
    ctx.pufe_sync_status()
    Ho, So = oasm.assemble_HS(m, rules, V)
    wg = sla.eigh(_csr(ctx, H).toarray(), _csr(ctx, S).toarray(), eigvals_only=True,
                  subset_by_index=[0, 3])
    wo = sla.eigh(Ho.toarray(), So.toarray(), eigvals_only=True, subset_by_index=[0, 3])
    print(f"\nC1 on the serendipity space (N = {ctx.n_dof}): {wg}")
    assert np.abs(wg - wo).max() < 1e-10


def test_mixed_scf_and_projector_calls_refuse_the_space():
    ctx = pufe.pufe_build_mesh(CASES["two_atom_2cube"]())
    with pytest.raises(pufe.PufeError) as ei:
        ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    assert ei.value.status == 1 and "serendipity" in str(ei.value)
    dev = torch.device("cuda:0")
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    with pytest.raises(pufe.PufeError) as ei:
        ctx.pufe_ion_density(np.zeros((1, 3)), np.ones(1), np.ones(1), rho)
    assert ei.value.status == 1
