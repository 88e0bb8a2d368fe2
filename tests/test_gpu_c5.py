"""The equation-of-state configuration at its full size: the 2x2x2 supercell
of the rocksalt cube (64 atoms, 32^3 elements, 7.15 M quadrature points,
N = 982,336, 188.6 M non-zeros) at k = (1/4, 1/4, 1/4) 2 pi / a, the first
of the sweep's four k-points.  The oracle cannot assemble a cell this size in
a test's time, so the checks are properties that hold at any size (Sec. 4,
eqs. bloch, strong): H(k) and S(k) Hermitian on the symmetric pattern; the
mixed-precision blocks against the FP64 ones (the FP64 kernels match the
oracle to 1e-12 on every smaller cell), each block normalised by its own
largest entry, with the mixed bounds of the parity tests; and the density
identity sum_q w_q n_q = sum_j f_j c_j^H S(k) c_j for 64 random complex
states, in both precisions."""
import math

import numpy as np
import pytest

from paper_1611_00731_gb300 import eos, pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_BLOCK = 5e-6       # FP32 element blocks (round-to-nearest sums), as for the rocksalt cube
TOL_DENSITY = 1e-5     # FP32 density sums


@pytest.fixture(scope="module")
def c5():
    wl = W.workload("c5_rocksalt_2x2x2_16cube")
    ctx = pufe.pufe_build_mesh(wl)
    dev = torch.device("cuda:0")
    rowptr, col = ctx.pattern()
    rp = torch.tensor(rowptr, device=dev)
    cl = torch.tensor(col.astype(np.int64), device=dev)
    rows = torch.repeat_interleave(torch.arange(ctx.n_dof, device=dev), rp[1:] - rp[:-1])
    # the transpose of the (symmetric) pattern: entry i of the transpose sits
    # at position perm[i] of the pattern's own order
    perm = torch.argsort(cl * ctx.n_dof + rows)
    k = 2.0 * math.pi / wl["a"] * np.asarray(eos.MP2_SHIFTED[0][0])
    return wl, ctx, dev, rp, cl, rows, perm, k


def _assemble(ctx, dev, k, V, prec):
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    H, S = (mk(), mk()), (mk(), mk())
    ctx.pufe_tabulate(prec)
    ctx.pufe_assemble_HS_bloch(k, V, H, S, prec=prec)
    ctx.pufe_sync_status()
    return H, S


def _block_err(A, B, fe_r, fe_c):
    """max |A - B| / max |B| on the FE-FE, FE-E and E-E entries."""
    out = {}
    for name, sel in (("FF", fe_r & fe_c), ("FE", fe_r ^ fe_c), ("EE", ~fe_r & ~fe_c)):
        d = torch.maximum((A[0] - B[0])[sel].abs().max(), (A[1] - B[1])[sel].abs().max())
        m = torch.maximum(B[0][sel].abs().max(), B[1][sel].abs().max())
        out[name] = float(d / m)
    return out


def test_c5_matrices_hermitian_and_mixed_against_fp64(c5):
    wl, ctx, dev, rp, cl, rows, perm, k = c5
    assert ctx.n_elem == 32 ** 3 and len(wl["atoms"]) == 64
    V = torch.tensor(W.random_potential(ctx.n_q, seed=51), device=dev)
    H64, S64 = _assemble(ctx, dev, k, V, pufe.PUFE_FP64)
    for X in (H64, S64):
        scale = float(X[0].abs().max())
        assert float((X[0] - X[0][perm]).abs().max()) < 1e-12 * scale
        assert float((X[1] + X[1][perm]).abs().max()) < 1e-12 * scale
    H32, S32 = _assemble(ctx, dev, k, V, pufe.PUFE_TF32X3)
    n_fe = (3 * int(wl["nel"])) ** 3
    fe_r, fe_c = rows < n_fe, cl < n_fe
    eh = _block_err(H32, H64, fe_r, fe_c)
    es = _block_err(S32, S64, fe_r, fe_c)
    print(f"\nC5 (N = {ctx.n_dof}, nnz = {ctx.nnz}) mixed vs FP64 at k: H {eh}, S {es}")
    for e in list(eh.values()) + [es["FE"], es["EE"]]:
        assert e < TOL_BLOCK
    assert es["FF"] < 1e-12   # exact FP64 constants in both


@pytest.mark.parametrize("prec", [pufe.PUFE_FP64, pufe.PUFE_TF32X3])
def test_c5_density_identity(c5, prec):
    wl, ctx, dev, rp, cl, rows, perm, k = c5
    nocc = int(wl["nocc"])
    rng = np.random.default_rng(52)
    Cr = torch.tensor(rng.standard_normal((ctx.n_dof, nocc)), device=dev)
    Ci = torch.tensor(rng.standard_normal((ctx.n_dof, nocc)), device=dev)
    f = torch.tensor(W.random_occupations(nocc, seed=52), device=dev)
    V = torch.zeros(ctx.n_q, dtype=torch.float64, device=dev)
    _, S = _assemble(ctx, dev, k, V, prec)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_density_bloch(k, Cr, Ci, f, rho, prec=prec)
    ctx.pufe_sync_status()
    _, w, _ = ctx.quadrature()
    lhs = float(torch.tensor(w, device=dev) @ rho)
    # c^H S c for S = Sr + i Si (Hermitian): the real part
    #   cr.(Sr cr - Si ci) + ci.(Sr ci + Si cr)
    Sr = torch.sparse_csr_tensor(rp, cl, S[0], (ctx.n_dof, ctx.n_dof))
    Si = torch.sparse_csr_tensor(rp, cl, S[1], (ctx.n_dof, ctx.n_dof))
    re = (Cr * (Sr @ Cr - Si @ Ci)).sum(0) + (Ci * (Sr @ Ci + Si @ Cr)).sum(0)
    rhs = float(f @ re)
    tol = 1e-11 if prec == pufe.PUFE_FP64 else TOL_DENSITY
    print(f"\nC5 density identity prec {prec}: {lhs:.12e} vs {rhs:.12e}, "
          f"rel {abs(lhs - rhs) / abs(rhs):.1e}")
    assert abs(lhs - rhs) < tol * abs(rhs)
