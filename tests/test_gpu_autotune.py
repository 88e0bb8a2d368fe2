"""The autotuner of the strip's enrichment-enrichment form (pufe_autotune).

On the two-atom cell on a 4^3 mesh (64 strip elements in four classes, 1-6
enrichment slots each):

* tuning sets at least one class and writes one cache line per class;
* with the cache rewritten to force the slot-pair form (1) on every class, and
  again the direct 4 x 4 tiles (2), a fresh context reads the decisions
  without timing, and H and S from either form match the oracle block by
  block at the mixed path's bounds (5e-6 of the block's largest entry; the
  FE-FE block of S is FP64 arithmetic, 1e-12);
* the two forced forms agree with each other to the same bound, and the
  tuned context's assembly too.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as oasm, mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import pufe, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {("H", "FF"): 5e-6, ("H", "FE"): 5e-6, ("H", "EE"): 5e-6,
       ("S", "FF"): 1e-12, ("S", "FE"): 5e-6, ("S", "EE"): 5e-6}


def _block_err(G, O, nfe):
    out = {}
    D = (G - O).tocsr()
    O = O.tocsr()
    for name, X in (("D", D), ("O", O)):
        row = np.repeat(np.arange(X.shape[0]), np.diff(X.indptr))
        fr, fc = row < nfe, X.indices < nfe
        for blk, sel in (("FF", fr & fc), ("FE", fr ^ fc), ("EE", ~fr & ~fc)):
            out[(name, blk)] = float(np.abs(X.data[sel]).max()) if sel.any() else 0.0
    return {b: out[("D", b)] / out[("O", b)] for b in ("FF", "FE", "EE") if out[("O", b)] > 0}


def _assemble(ctx, V):
    dev = torch.device("cuda:0")
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    ctx.pufe_assemble_HS(torch.tensor(V, device=dev), H, S, prec=pufe.PUFE_TF32X3)
    ctx.pufe_sync_status()
    rowptr, col = ctx.pattern()
    mk = lambda x: sp.csr_matrix((x.cpu().numpy(), col, rowptr), shape=(ctx.n_dof, ctx.n_dof))
    return mk(H), mk(S)


def _check(label, Hg, Sg, Ho, So, nfe):
    for name, G, O in (("H", Hg, Ho), ("S", Sg, So)):
        errs = _block_err(G, O, nfe)
        print(f"{label} {name}: " + ", ".join(f"{b} {e:.1e}" for b, e in errs.items()))
        for b, e in errs.items():
            assert e < TOL[(name, b)], (label, name, b, e)


def test_autotune_cache_and_forced_forms(tmp_path, monkeypatch):
    wl = W.workload("c1_two_atom_4cube")
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    V = W.random_potential(len(rules[1]), seed=5)
    Ho, So = oasm.assemble_HS(m, rules, V)
    nfe = (3 * int(wl["nel"])) ** 3
    cache = tmp_path / "forms.txt"
    monkeypatch.setenv("PUFE_AUTOTUNE_CACHE", str(cache))
    ctx = pufe.pufe_build_mesh(wl)
    ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    n = ctx.pufe_autotune()
    lines = [ln.split() for ln in cache.read_text().splitlines() if ln.strip()]
    print(f"autotune: {n} classes, decisions " + ", ".join(f"{k}:{f}" for k, f in lines))
    assert n >= 1 and len(lines) == n and all(f in ("1", "2") for _, f in lines)
    Ht, St = _assemble(ctx, V)
    _check("tuned", Ht, St, Ho, So, nfe)
    forced = {}
    for form in ("1", "2"):
        cache.write_text("".join(f"{k} {form}\n" for k, _ in lines))
        c = pufe.pufe_build_mesh(wl)
        c.pufe_tabulate(pufe.PUFE_TF32X3)
        assert c.pufe_autotune() == n
        # every class came from the cache: nothing was appended
        assert len(cache.read_text().splitlines()) == n
        forced[form] = _assemble(c, V)
        _check(f"form {form}", *forced[form], Ho, So, nfe)
    # the two forms differ by FP32 rounding only
    _check("pair vs tiles", *forced["1"], *forced["2"], nfe)
    assert os.environ["PUFE_AUTOTUNE_CACHE"] == str(cache)
