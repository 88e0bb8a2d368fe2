"""The differentiable assembly map V -> H (paper_1611_00731_gb300/autograd.py):
its backward, the hand-written adjoint kernel, against the oracle's adjoint;
the Hellmann-Feynman identity dE_band/dV_q = w_q n_q (Sec. 3 eq. rhoe) for
fixed eigenstates; and central finite differences of the band energy
sum_n f_n eps_n(V) at 64 random quadrature points (seed 0, h = 1e-6)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import assemble as oasm, mesh as omesh, potential as opot, quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    return torch.device("cuda:0")


def _setup(wl, prec):
    from paper_1611_00731_gb300.autograd import assemble_H
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_FP64)        # S and the reference H are FP64
    ctx.pufe_tabulate(prec)
    return m, rules, ctx, assemble_H


def _csr(ctx, vals):
    rowptr, col = ctx.pattern()
    return sp.csr_matrix((vals, col, rowptr), shape=(ctx.n_dof, ctx.n_dof))


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec", [pufe.PUFE_FP64, pufe.PUFE_TF32X3])
def test_backward_is_the_oracle_adjoint(prec):
    """L = sum Hbar_ij H_ij(V) with a general (non-symmetric) Hbar on the
    pattern: autograd's dL/dV against the oracle's adjoint, and the forward
    values against pufe_assemble_HS."""
    m, rules, ctx, assemble_H = _setup(W.workload("c1_two_atom_4cube"), prec)
    dev = _dev()
    V = torch.tensor(W.random_potential(ctx.n_q, seed=51), device=dev, requires_grad=True)
    H = assemble_H(ctx, V, prec)
    H2 = torch.empty_like(H)
    ctx.pufe_assemble_HS(V.detach(), H2, None, prec=prec)
    hb = W.random_potential(ctx.nnz, seed=52)
    (H * torch.tensor(hb, device=dev)).sum().backward()
    ctx.pufe_sync_status()
    # same values as the plain call up to summation order (FP64 atomics; in the
    # mixed mode also the FP32 shared-memory sums of the E x E tiles)
    same = 1e-13 if prec == pufe.PUFE_FP64 else 1e-6
    assert _rel(H.detach().cpu().numpy(), H2.cpu().numpy()) < same
    go = oasm.adjoint_V(m, rules, _csr(ctx, hb))
    tol = 1e-12 if prec == pufe.PUFE_FP64 else 1e-4
    assert _rel(V.grad.cpu().numpy(), go) < tol


@pytest.mark.parametrize("prec", [pufe.PUFE_FP64, pufe.PUFE_TF32X3])
def test_band_energy_gradient_is_the_density(prec):
    """E_band = sum_n f_n c_n^T H c_n with the S-normalised lowest states of
    C1 held fixed: E_band equals sum f eps, and its gradient through the
    backward kernel equals w_q n_q of the same states (GPU density kernel and
    oracle)."""
    wl = W.workload("c1_two_atom_4cube")
    m, rules, ctx, assemble_H = _setup(wl, prec)
    dev = _dev()
    V = torch.tensor(opot.ionic_potential(wl, rules[0]), device=dev, requires_grad=True)
    H = assemble_H(ctx, V, prec)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(V.detach(), None, S, prec=pufe.PUFE_FP64)
    ctx.pufe_sync_status()
    eps, C = sla.eigh(_csr(ctx, H.detach().cpu().numpy()).toarray(),
                      _csr(ctx, S.cpu().numpy()).toarray(), subset_by_index=[0, 3])
    f = np.array([2.0, 2.0])
    Cf = C[:, :2]
    rowptr, col = ctx.pattern()
    rows = np.repeat(np.arange(ctx.n_dof), np.diff(rowptr))
    G = (Cf[rows] * Cf[col]) @ f               # dE_band / dH_ij on the pattern
    E = (H * torch.tensor(G, device=dev)).sum()
    E.backward()
    assert abs(float(E.detach()) - f @ eps[:2]) < 1e-10 * abs(f @ eps[:2])
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_density(torch.tensor(np.ascontiguousarray(Cf), device=dev),
                     torch.tensor(f, device=dev), rho, prec=prec)
    ctx.pufe_sync_status()
    w = rules[1]
    grad = V.grad.cpu().numpy()
    tol = 1e-12 if prec == pufe.PUFE_FP64 else 1e-4
    assert _rel(grad, w * rho.cpu().numpy()) < tol
    assert _rel(grad, w * oasm.density(m, rules, Cf, f)) < tol


def test_band_energy_finite_differences():
    """d/dV_q of sum_n f_n eps_n(V), eps from the generalized eigenproblem of
    the GPU's H(V) and S, by central differences (h = 1e-6) at 64 random
    points, against the backward kernel's w_q n_q (Hellmann-Feynman; the two
    occupied states are non-degenerate).  The bound is the differences'
    round-off, measured with the oracle's H: 3e-8 at this step."""
    wl = W.small_two_atom(nel=2, quad_p=6)
    m, rules, ctx, assemble_H = _setup(wl, pufe.PUFE_FP64)
    dev = _dev()
    V0 = opot.ionic_potential(wl, rules[0])
    V = torch.tensor(V0, device=dev, requires_grad=True)
    H = assemble_H(ctx, V, pufe.PUFE_FP64)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(V.detach(), None, S)
    Sd = _csr(ctx, S.cpu().numpy()).toarray()
    eps, C = sla.eigh(_csr(ctx, H.detach().cpu().numpy()).toarray(), Sd, subset_by_index=[0, 2])
    assert eps[2] - eps[1] > 0.1 and eps[1] - eps[0] > 0.1
    f = np.array([2.0, 2.0])
    rowptr, col = ctx.pattern()
    rows = np.repeat(np.arange(ctx.n_dof), np.diff(rowptr))
    G = (C[rows, :2] * C[col, :2]) @ f
    (H * torch.tensor(G, device=dev)).sum().backward()
    g = V.grad.cpu().numpy()
    h = 1e-6
    Hp = torch.empty_like(H)
    qs = np.random.default_rng(0).choice(ctx.n_q, 64, replace=False)
    err = 0.0
    for q in qs:
        E = []
        for sgn in (1.0, -1.0):
            Vp = V0.copy()
            Vp[q] += sgn * h
            ctx.pufe_assemble_HS(torch.tensor(Vp, device=dev), Hp, None)
            Hd = _csr(ctx, Hp.cpu().numpy()).toarray()
            E.append(f @ sla.eigh(Hd, Sd, eigvals_only=True, subset_by_index=[0, 1]))
        err = max(err, abs((E[0] - E[1]) / (2.0 * h) - g[q]))
    ctx.pufe_sync_status()
    print(f"finite differences: max |FD - w n| = {err:.2e} (max |w n| = {np.abs(g).max():.2e})")
    assert err < 2e-7
