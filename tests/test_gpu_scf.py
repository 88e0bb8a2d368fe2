"""GPU parity of the SCF calls (ionic charge, effective potential, one SCF
step, a short SCF loop) against the oracle (oracle/scf.py), through the
C ABI.  FP64 throughout, tolerance 1e-10 of the largest value (the two sides
solve the Poisson problem by different exact methods: a sparse direct solve
and the fast diagonalization of the tensor-product stiffness)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as oasm, eig as oeig, mesh as omesh, quadrature as oq
from oracle import scf as oscf
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _dev():
    return torch.device("cuda:0")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _atoms(wl):
    tau = np.array([t for _, t in wl["atoms"]], dtype=np.float64).reshape(-1, 3)
    Z = np.array([wl["species"][s]["Z"] for s, _ in wl["atoms"]], dtype=np.float64)
    sig = np.array([wl["species"][s]["sigma"] for s, _ in wl["atoms"]], dtype=np.float64)
    return tau, Z, sig


CASES = {
    "two_atom_2cube": lambda: W.small_two_atom(nel=2, quad_p=6),
    "c1_two_atom_4cube": lambda: W.workload("c1_two_atom_4cube"),
}


@pytest.fixture(scope="module", params=list(CASES))
def setup(request):
    wl = CASES[request.param]()
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    dev = _dev()
    rho_I = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_ion_density(*_atoms(wl), rho_I)
    ctx.pufe_sync_status()
    K = oscf.fe_stiffness(m)
    return request.param, wl, m, rules, ctx, rho_I, K


def test_ion_density_matches_oracle(setup):
    name, wl, m, rules, ctx, rho_I, K = setup
    want = oscf.ion_density(wl, rules[0])
    assert _rel(rho_I.cpu().numpy(), want) < 1e-12, name
    # neutral with the electrons up to the rule's accuracy for the Gaussians
    assert abs(rules[1] @ want - wl["nelec"]) < 1e-2


def test_effective_potential_matches_oracle(setup):
    name, wl, m, rules, ctx, rho_I, K = setup
    dev = _dev()
    w = rules[1]
    n = np.random.default_rng(3).uniform(0.2, 1.0, len(w))
    n *= wl["nelec"] / (w @ n)                          # neutral total charge
    V, VC, exc = oscf.effective_potential(m, rules, n, rho_I.cpu().numpy(), K)
    nd = torch.tensor(n, device=dev)
    Vg = torch.empty_like(nd)
    VCg = torch.empty_like(nd)
    eg = torch.empty_like(nd)
    ctx.pufe_effective_potential(nd, rho_I, Vg, VCg, eg)
    ctx.pufe_sync_status()
    assert _rel(VCg.cpu().numpy(), VC) < TOL, name
    assert _rel(eg.cpu().numpy(), exc) < 1e-13, name
    assert _rel(Vg.cpu().numpy(), V) < TOL, name


def _start(wl, m, rules, rho_I_h, K, nstates):
    n0 = np.full(len(rules[1]), wl["nelec"] / wl["a"] ** 3)
    V0, _, _ = oscf.effective_potential(m, rules, n0, rho_I_h, K)
    H, S = oasm.assemble_HS(m, rules, V0)
    eps, C = oeig.lowest_eigs(H, S, nstates)
    return n0, V0, eps, C


@pytest.mark.parametrize("prec", [pufe.PUFE_FP64, pufe.PUFE_TF32X3])
def test_scf_step_matches_oracle(setup, prec):
    name, wl, m, rules, ctx, rho_I, K = setup
    dev = _dev()
    rho_h = rho_I.cpu().numpy()
    n0, V0, eps, C = _start(wl, m, rules, rho_h, K, 6)
    kT, alpha = 0.01, 0.4
    ref = oscf.scf_step(m, rules, wl, eps, C, wl["nelec"], kT, alpha, n0, V0, rho_h, K)
    ctx.pufe_tabulate(prec)
    n = torch.tensor(n0, device=dev)
    Vout = torch.empty_like(n)
    f, info = ctx.pufe_scf_step(eps, torch.tensor(np.ascontiguousarray(C), device=dev),
                                wl["nelec"], kT, alpha, rho_I, torch.tensor(V0, device=dev), n,
                                Vout, prec=prec)
    ctx.pufe_sync_status()
    tol = TOL if prec == pufe.PUFE_FP64 else 1e-5       # FP32 density in the mixed mode
    assert np.abs(f - ref["f"]).max() < 1e-12
    assert abs(info["mu"] - ref["mu"]) < 1e-12
    assert _rel(n.cpu().numpy(), ref["n_new"]) < tol, name
    assert _rel(Vout.cpu().numpy(), ref["V_eff"]) < tol, name
    for k in ("e_band", "e_dc", "e_es", "e_self", "e_xc", "e_ts", "e_total"):
        assert abs(info[k] - ref[k]) < tol * max(1.0, abs(ref[k])), (name, k, info[k], ref[k])
    assert abs(info["residual"] - ref["residual"]) < tol * max(1.0, ref["residual"]) + 1e-12


@pytest.mark.parametrize("pulay", [0, 4])
def test_scf_loop_matches_oracle_loop(pulay):
    """Six SCF iterations on the 2^3 two-atom cell, both sides from the same
    start: GPU = pufe_assemble_HS + host eigensolve + pufe_scf_step, oracle =
    its own assembly, eigensolve and step; linear and Pulay mixing.
    Eigenvalues, energy and residual agree, and the residual falls."""
    wl = W.small_two_atom(nel=2, quad_p=6)
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    dev = _dev()
    K = oscf.fe_stiffness(m)
    rho_I = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_ion_density(*_atoms(wl), rho_I)
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    rho_h = oscf.ion_density(wl, rules[0])
    nst, kT, alpha = 6, 0.01, 0.5
    n_o = np.full(len(rules[1]), wl["nelec"] / wl["a"] ** 3)
    V_o, _, _ = oscf.effective_potential(m, rules, n_o, rho_h, K)
    n_g = torch.tensor(n_o, device=dev)
    V_g = torch.tensor(V_o, device=dev)
    V_next = torch.empty_like(V_g)
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    rowptr, col = ctx.pattern()
    mixer = oscf.PulayMixer(pulay) if pulay > 1 else None
    ctx.pufe_scf_reset()
    res = []
    for it in range(6):
        Ho, So = oasm.assemble_HS(m, rules, V_o)
        eo, Co = oeig.lowest_eigs(Ho, So, nst)
        ro = oscf.scf_step(m, rules, wl, eo, Co, wl["nelec"], kT, alpha, n_o, V_o, rho_h, K,
                           mixer=mixer)
        n_o, V_o = ro["n_new"], ro["V_eff"]
        ctx.pufe_assemble_HS(V_g, H, S)
        ctx.pufe_sync_status()
        Hg = sp.csr_matrix((H.cpu().numpy(), col, rowptr), shape=(ctx.n_dof, ctx.n_dof))
        Sg = sp.csr_matrix((S.cpu().numpy(), col, rowptr), shape=(ctx.n_dof, ctx.n_dof))
        eg, Cg = oeig.lowest_eigs(Hg, Sg, nst)
        _, info = ctx.pufe_scf_step(eg, torch.tensor(np.ascontiguousarray(Cg), device=dev),
                                    wl["nelec"], kT, alpha, rho_I, V_g, n_g, V_next,
                                    pulay=pulay)
        V_g, V_next = V_next, V_g
        assert np.abs(eg - eo).max() < 1e-9, it
        assert abs(info["e_total"] - ro["e_total"]) < 1e-9, it
        assert abs(info["residual"] - ro["residual"]) < 1e-9, it
        res.append(info["residual"])
    assert res[-1] < res[0]
    assert _rel(n_g.cpu().numpy(), n_o) < 1e-9
    print(f"pulay={pulay}: residuals", ["%.2e" % r for r in res])
