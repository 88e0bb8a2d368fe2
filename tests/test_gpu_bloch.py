"""GPU parity of the Bloch (k != 0) calls against the oracle (oracle/bloch.py),
through the C ABI: H(k), S(k), the density of complex states and the adjoint,
FP64, max |error| / max |X| <= 1e-12."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import bloch as ob, mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
K_FRAC = np.array([0.3, -0.2, 0.1])

CASES = {
    "two_atom_2cube": lambda: W.small_two_atom(nel=2, quad_p=4),
    "one_element": lambda: W.small_two_atom(nel=1, quad_p=4),   # repeated DOFs, other shifts
    "c1_two_atom_4cube": lambda: W.workload("c1_two_atom_4cube"),
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
    k = 2.0 * math.pi / wl["a"] * K_FRAC
    return request.param, wl, m, rules, ctx, k


def _gpu_HS_k(ctx, V, k):
    dev = torch.device("cuda:0")
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    Hr, Hi, Sr, Si = mk(), mk(), mk(), mk()
    ctx.pufe_assemble_HS_bloch(k, torch.tensor(V, device=dev), (Hr, Hi), (Sr, Si))
    ctx.pufe_sync_status()
    rowptr, col = ctx.pattern()
    N = ctx.n_dof
    H = sp.csr_matrix((Hr.cpu().numpy() + 1j * Hi.cpu().numpy(), col, rowptr), shape=(N, N))
    S = sp.csr_matrix((Sr.cpu().numpy() + 1j * Si.cpu().numpy(), col, rowptr), shape=(N, N))
    return H, S


def test_bloch_assembly_matches_oracle(case):
    name, wl, m, rules, ctx, k = case
    V = W.random_potential(len(rules[1]), seed=21)
    Ho, So = ob.assemble_HS_k(m, rules, V, k)
    Hg, Sg = _gpu_HS_k(ctx, V, k)
    assert _rel(Hg, Ho) < TOL, name
    assert _rel(Sg, So) < TOL, name
    assert abs(Hg - Hg.conj().T).max() < TOL * abs(Hg).max()


def test_bloch_density_and_adjoint_match_oracle(case):
    name, wl, m, rules, ctx, k = case
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(22)
    nocc = 5
    C = rng.standard_normal((m.n_dof, nocc)) + 1j * rng.standard_normal((m.n_dof, nocc))
    f = W.random_occupations(nocc, seed=22)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_density_bloch(k, torch.tensor(np.ascontiguousarray(C.real), device=dev),
                           torch.tensor(np.ascontiguousarray(C.imag), device=dev),
                           torch.tensor(f, device=dev), rho)
    V = W.random_potential(len(rules[1]), seed=23)
    Ho, _ = ob.assemble_HS_k(m, rules, V, k)
    Hbar = Ho.copy()
    Hbar.data = rng.standard_normal(Ho.nnz) + 1j * rng.standard_normal(Ho.nnz)
    # the GPU's pattern equals the oracle's (checked on CPU), so the CSR data align
    vbar = torch.empty_like(rho)
    ctx.pufe_assemble_HV_adjoint_bloch(k, torch.tensor(Hbar.data.real.copy(), device=dev),
                                       torch.tensor(Hbar.data.imag.copy(), device=dev), vbar)
    ctx.pufe_sync_status()
    assert _rel(rho.cpu().numpy(), ob.density_k(m, rules, C, f, k)) < TOL, name
    assert _rel(vbar.cpu().numpy(), ob.adjoint_V_k(m, rules, Hbar, k)) < TOL, name


def test_empty_lattice_bands_at_k_on_the_gpu():
    a = 4.0
    wl = W.empty_lattice(nel=4, a=a, p=4)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    k = 2.0 * math.pi / a * K_FRAC
    H, S = _gpu_HS_k(ctx, np.zeros(ctx.n_q), k)
    w = sla.eigh(H.toarray(), S.toarray(), eigvals_only=True, subset_by_index=[0, 3])
    G = 2.0 * math.pi / a * np.array([[0, 0, 0], [-1, 0, 0], [0, 1, 0], [0, 0, -1],
                                      [1, 0, 0], [0, -1, 0], [0, 0, 1]], dtype=np.float64)
    exact = np.sort(0.5 * ((G + k) ** 2).sum(axis=1))[:4]
    assert np.all(w >= exact - 1e-12)
    assert np.abs(w - exact).max() < 2e-4 * exact[1]     # tricubic error at h = 1 bohr


# ---- mixed precision (PUFE_TF32X3): FP32 element blocks, phased scatter -----
TOL_TF32 = 5e-6     # the Gamma-point FP32 block bound (tests/test_gpu_parity.py), FP32 phases

MIXED_CASES = {
    "two_atom_2cube": lambda: W.small_two_atom(nel=2, quad_p=6),
    "c1_two_atom_4cube": lambda: W.workload("c1_two_atom_4cube"),
}


@pytest.mark.parametrize("name", list(MIXED_CASES))
def test_mixed_bloch_assembly_matches_oracle(name):
    """H(k), S(k) of the mixed path against the oracle's FP64 ones; k = 0
    against the Gamma-point mixed assembly; the C1 band energies at k within
    the 1e-5 Ha eigenvalue target."""
    wl = MIXED_CASES[name]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    dev = torch.device("cuda:0")
    k = 2.0 * math.pi / wl["a"] * K_FRAC
    V = W.random_potential(len(rules[1]), seed=23)
    Vd = torch.tensor(V, device=dev)
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    Hr, Hi, Sr, Si = mk(), mk(), mk(), mk()
    ctx.pufe_assemble_HS_bloch(k, Vd, (Hr, Hi), (Sr, Si), prec=pufe.PUFE_TF32X3)
    ctx.pufe_sync_status()
    rowptr, col = ctx.pattern()
    N = ctx.n_dof
    csr = lambda re, im: sp.csr_matrix((re.cpu().numpy() + 1j * im.cpu().numpy(), col, rowptr),
                                       shape=(N, N))
    Hg, Sg = csr(Hr, Hi), csr(Sr, Si)
    Ho, So = ob.assemble_HS_k(m, rules, V, k)
    assert _rel(Hg, Ho) < TOL_TF32 and _rel(Sg, So) < TOL_TF32, (_rel(Hg, Ho), _rel(Sg, So))
    assert abs(Hg - Hg.conj().T).max() < TOL_TF32 * abs(Hg).max()
    if name == "c1_two_atom_4cube":
        wg = sla.eigh(Hg.toarray(), Sg.toarray(), eigvals_only=True, subset_by_index=[0, 3])
        wo = sla.eigh(Ho.toarray(), So.toarray(), eigvals_only=True, subset_by_index=[0, 3])
        assert np.abs(wg - wo).max() < 1e-5
    # k = 0: the Gamma-point mixed matrices, imaginary parts zero
    H0, S0 = mk(), mk()
    ctx.pufe_assemble_HS(Vd, H0, S0, prec=pufe.PUFE_TF32X3)
    ctx.pufe_assemble_HS_bloch((0.0, 0.0, 0.0), Vd, (Hr, Hi), (Sr, Si), prec=pufe.PUFE_TF32X3)
    ctx.pufe_sync_status()
    assert float(Hi.abs().max()) == 0.0 and float(Si.abs().max()) == 0.0
    assert _rel(Hr.cpu().numpy(), H0.cpu().numpy()) < 1e-6
    assert _rel(Sr.cpu().numpy(), S0.cpu().numpy()) < 1e-6


def _c3_like_large():
    wl = W.workload("c3_cscl_4cube")
    wl["species"] = [dict(s) for s in wl["species"]]
    wl["species"][0]["orbitals"] = [o for o in wl["species"][0]["orbitals"] if o[0] >= 3]
    wl["species"][0]["r_e"] = 1.5
    wl["quad"] = dict(wl["quad"], mode=W.QUAD_FIXED, p_far=5, p_near=5)
    return wl


def _mixed_rule_sizes():
    wl = W.small_two_atom(nel=4, a=6.0, r_c=1.2, r_e=3.0)
    wl["quad"] = dict(mode=W.QUAD_PADAPT, p_far=6, p_near=10, p_min=9, p_max=11, tol=1e-6,
                      max_depth=0)
    return wl


# every FP32 adjoint kernel: the FE-FE form and the slot-form strip (first
# two), the tensor-core-class kernel (n_e > 128) and the per-point strip (11^3
# rules)
MIXED_DA_CASES = {
    "two_atom_2cube": lambda: W.small_two_atom(nel=2, quad_p=6),
    "c1_two_atom_4cube": lambda: W.workload("c1_two_atom_4cube"),
    "c3_like_large_elements": _c3_like_large,
    "p_adaptive_9_11": _mixed_rule_sizes,
}


@pytest.mark.parametrize("name", list(MIXED_DA_CASES))
def test_mixed_bloch_density_and_adjoint_match_oracle(name):
    """PUFE_TF32X3 density of complex states and adjoint of V -> H(k) against
    the oracle's FP64 ones (the Gamma-point mixed bounds: 1e-5 for the FP32
    density sums, 1e-4 for the adjoint); at k = 0 with real inputs both equal
    the Gamma-point mixed calls bit for bit (phase 1 + 0i multiplies exactly)."""
    wl = MIXED_DA_CASES[name]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    dev = torch.device("cuda:0")
    k = 2.0 * math.pi / wl["a"] * K_FRAC
    rng = np.random.default_rng(31)
    nocc = 6
    C = rng.standard_normal((m.n_dof, nocc)) + 1j * rng.standard_normal((m.n_dof, nocc))
    f = W.random_occupations(nocc, seed=31)
    Cr = torch.tensor(np.ascontiguousarray(C.real), device=dev)
    Ci = torch.tensor(np.ascontiguousarray(C.imag), device=dev)
    fd = torch.tensor(f, device=dev)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_density_bloch(k, Cr, Ci, fd, rho, prec=pufe.PUFE_TF32X3)
    V = W.random_potential(len(rules[1]), seed=32)
    Ho, _ = ob.assemble_HS_k(m, rules, V, k)
    Hbar = Ho.copy()
    Hbar.data = rng.standard_normal(Ho.nnz) + 1j * rng.standard_normal(Ho.nnz)
    Hre = torch.tensor(Hbar.data.real.copy(), device=dev)
    Him = torch.tensor(Hbar.data.imag.copy(), device=dev)
    vbar = torch.empty_like(rho)
    ctx.pufe_assemble_HV_adjoint_bloch(k, Hre, Him, vbar, prec=pufe.PUFE_TF32X3)
    ctx.pufe_sync_status()
    e_rho = _rel(rho.cpu().numpy(), ob.density_k(m, rules, C, f, k))
    e_adj = _rel(vbar.cpu().numpy(), ob.adjoint_V_k(m, rules, Hbar, k))
    print(f"\n{name}: mixed Bloch density {e_rho:.1e}, adjoint {e_adj:.1e}")
    assert e_rho < 1e-5 and e_adj < 1e-4, (name, e_rho, e_adj)
    # k = 0, real inputs: the Gamma-point mixed calls
    zero = torch.zeros_like(Cr)
    ctx.pufe_density_bloch((0.0, 0.0, 0.0), Cr, zero, fd, rho, prec=pufe.PUFE_TF32X3)
    rho0 = torch.empty_like(rho)
    ctx.pufe_density(Cr, fd, rho0, prec=pufe.PUFE_TF32X3)
    ctx.pufe_assemble_HV_adjoint_bloch((0.0, 0.0, 0.0), Hre, torch.zeros_like(Hre), vbar,
                                       prec=pufe.PUFE_TF32X3)
    v0 = torch.empty_like(rho)
    ctx.pufe_assemble_HV_adjoint(Hre, v0, prec=pufe.PUFE_TF32X3)
    ctx.pufe_sync_status()
    assert torch.equal(rho, rho0)
    assert torch.equal(vbar, v0)


def test_mixed_bloch_gram_form_of_the_EE_overlap_block():
    """An h-adaptive CsCl-like cell whose Ce-like elements carry 25 one-vertex
    enrichment slots on eight 8^3 sub-cells: their cells hold more Psi values
    than the projection form's shared-memory stage, so the E-E block of S
    takes the Gram form.  H(k), S(k) of the mixed path against the oracle at
    k, and S's E-E block against its own largest entry (the mixed bound 5e-6)."""
    wl = W.workload("c3_cscl_4cube")
    wl["species"] = [dict(s) for s in wl["species"]]
    wl["species"][0]["orbitals"] = [o for o in wl["species"][0]["orbitals"] if o[0] >= 3]
    wl["species"][0]["r_e"] = 0.8
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    assert 4096 in set(np.diff(rules[2]).tolist())
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    dev = torch.device("cuda:0")
    k = 2.0 * math.pi / wl["a"] * K_FRAC
    V = W.random_potential(len(rules[1]), seed=61)
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    Hr, Hi, Sr, Si = mk(), mk(), mk(), mk()
    ctx.pufe_assemble_HS_bloch(k, torch.tensor(V, device=dev), (Hr, Hi), (Sr, Si),
                               prec=pufe.PUFE_TF32X3)
    ctx.pufe_sync_status()
    rowptr, col = ctx.pattern()
    N = ctx.n_dof
    csr = lambda re, im: sp.csr_matrix((re.cpu().numpy() + 1j * im.cpu().numpy(), col, rowptr),
                                       shape=(N, N))
    Hg, Sg = csr(Hr, Hi), csr(Sr, Si)
    Ho, So = ob.assemble_HS_k(m, rules, V, k)
    assert _rel(Hg, Ho) < TOL_TF32 and _rel(Sg, So) < TOL_TF32, (_rel(Hg, Ho), _rel(Sg, So))
    nfe = (3 * int(wl["nel"])) ** 3
    D = (Sg - So).tocsr()[nfe:, nfe:]
    ee = float(abs(D).max() / abs(So.tocsr()[nfe:, nfe:]).max())
    print(f"\nGram form at k: S E-E block {ee:.1e}")
    assert ee < 5e-6
