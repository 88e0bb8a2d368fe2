"""Pins of the oracle's quadrature rules (CPU only)."""
import numpy as np

from oracle import enrich, fe, mesh as omesh, quadrature as oq
from paper_1611_00731_gb300 import workloads as W


def _brute(mesh, k, lo, hi, p=24):
    """Psi^2 integral on [lo, hi] by p^3 Gauss on each of the 8 octants."""
    al = mesh.alphas[k]
    mid = (lo + hi) / 2
    tot = 0.0
    for c in range(2):
        for b in range(2):
            for a in range(2):
                off = np.array([a, b, c])
                pts, w = fe.gauss_box(p, np.where(off == 0, lo, mid), np.where(off == 0, mid, hi))
                psi = enrich.enrichment(al["orb"], al["rc"], al["tau"], mesh.a, pts, False)
                tot += w @ psi ** 2
    return tot


def test_fixed_rule_classes_and_volume():
    m = omesh.Mesh(W.workload("c1_two_atom_4cube"))
    pts, wts, off = oq.all_rules(m)
    q = np.diff(off)
    assert set(q.tolist()) <= {64, 512}
    assert abs(wts.sum() - m.a ** 3) < 1e-11
    for e in range(m.nelem):
        lo, hi = m.elem_box(e)
        s = slice(off[e], off[e + 1])
        assert np.all(pts[s] > lo) and np.all(pts[s] < hi)
        assert abs(wts[s].sum() - m.h ** 3) < 1e-14


def test_hadapt_rule_integrates_psi2_within_tolerance():
    """Recursive 5^3-vs-8^3 rule (Sec. 5.2) with room to recurse: the leaves'
    accepted errors add up, so the element integral is within a few tol."""
    wl = W.small_two_atom(nel=4, a=4.0, r_c=1.5, r_e=1.0)
    wl["quad"] = dict(mode=oq.HADAPT, p_far=4, p_near=8, p_min=5, p_max=8,
                      tol=1e-6, max_depth=4)
    m = omesh.Mesh(wl)
    e = 0  # corner element touching the Z=1 atom at the origin
    p, w = oq.element_rule(m, e)
    lo, hi = m.elem_box(e)
    assert abs(w.sum() - m.h ** 3) < 1e-14
    assert len(w) > 512 and len(w) % 512 == 0     # it did subdivide
    for k in m.elem_alphas(e):
        al = m.alphas[k]
        psi = enrich.enrichment(al["orb"], al["rc"], al["tau"], m.a, p, False)
        ref = _brute(m, k, lo, hi)
        assert abs(w @ psi ** 2 - ref) < 1e-7


def test_hadapt_depth_one_sizes():
    wl = W.workload("c3_cscl_4cube")
    wl["species"][0]["orbitals"] = wl["species"][0]["orbitals"][:2]
    wl["species"][1]["orbitals"] = wl["species"][1]["orbitals"][:1]
    m = omesh.Mesh(wl)
    for e in (0, 1, 21):
        p, w = oq.element_rule(m, e)
        assert len(w) in (64, 512, 4096)
        assert abs(w.sum() - m.h ** 3) < 1e-14
        assert (len(w) == 64) == (not m.elem_alphas(e))


def test_padapt_choice_satisfies_tolerance():
    wl = W.workload("c2_rocksalt_4cube")
    m = omesh.Mesh(wl)
    q = wl["quad"]
    for e in (0, 7, 21):
        pts, w = oq.element_rule(m, e)
        p = round(len(w) ** (1 / 3))
        assert q["p_min"] <= p <= q["p_max"]
        lo, hi = m.elem_box(e)
        alphas = m.elem_alphas(e)
        if p < q["p_max"]:
            err = np.abs(oq._integrals(m, alphas, lo, hi, p) - oq._integrals(m, alphas, lo, hi, p + 2))
            assert (err < q["tol"]).all()
        if p > q["p_min"]:
            err = np.abs(oq._integrals(m, alphas, lo, hi, p - 1) - oq._integrals(m, alphas, lo, hi, p + 1))
            assert (err >= q["tol"]).any()
