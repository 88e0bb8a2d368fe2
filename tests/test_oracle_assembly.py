"""Pins of the oracle's H/S assembly, density and adjoint (CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble as oasm, eig as oeig, mesh as omesh, quadrature as oq
from oracle import potential as opot
from paper_1611_00731_gb300 import workloads as W


def _setup(wl):
    m = omesh.Mesh(wl)
    rules = oq.all_rules(m)
    return m, rules


def test_empty_lattice_spectrum_and_convergence():
    """V = 0, no enrichment: eigenvalues |G|^2/2 from above, error O(h^6)."""
    a = 4.0
    g1 = 0.5 * (2 * math.pi / a) ** 2
    errs = []
    for nel in (3, 4):
        m, rules = _setup(W.empty_lattice(nel=nel, a=a, p=4))
        H, S = oasm.assemble_HS(m, rules, np.zeros(len(rules[1])))
        w, _ = oeig.lowest_eigs(H, S, 7)
        assert abs(w[0]) < 1e-12                       # constant is in the span
        assert np.all(w[1:7] >= g1 - 1e-12)             # min-max: upper bounds
        assert np.ptp(w[1:7]) < 1e-10                   # sixfold degenerate
        errs.append(w[1] - g1)
    assert errs[1] < 1e-3
    rate = math.log(errs[0] / errs[1]) / math.log(4 / 3)
    assert 5.0 < rate < 7.0                             # O(h^6) for cubic FE


def test_harmonic_oscillator_levels():
    """V = w^2 |x - c|^2 / 2 well inside a large cell: levels w (n + 3/2)."""
    a, om = 6.0, 2.0
    wl = W.empty_lattice(nel=5, a=a, p=5)
    m, rules = _setup(wl)
    d = rules[0] - a / 2
    V = 0.5 * om ** 2 * (d * d).sum(axis=1)
    H, S = oasm.assemble_HS(m, rules, V)
    w, _ = oeig.lowest_eigs(H, S, 10)
    exact = om * np.array([1.5] + [2.5] * 3 + [3.5] * 6)
    assert np.all(w >= exact - 1e-6)                    # variational
    assert abs(w[0] - exact[0]) / exact[0] < 3e-3
    assert np.abs(w - exact).max() / exact.max() < 1e-2
    assert np.ptp(w[1:4]) < 1e-9 * w[1]                 # p-like level threefold


def test_S_spd_and_conditioning_grows_with_support_radius():
    conds = []
    for re in (None, 0.5, 1.0, 1.5):   # plain FE, then r_e enriching 1, 7, 19 vertices
        wl = (W.empty_lattice(nel=4, a=4.0, p=6) if re is None else
              W.small_two_atom(nel=4, a=4.0, quad_p=6, r_c=1.5, r_e=re))
        m, rules = _setup(wl)
        _, S = oasm.assemble_HS(m, rules, np.zeros(len(rules[1])))
        Sd = S.toarray()
        assert np.abs(Sd - Sd.T).max() < 1e-15 * np.abs(Sd).max()
        sla.cholesky(Sd)
        ev = np.linalg.eigvalsh(Sd)
        conds.append(ev[-1] / ev[0])
    assert conds[0] < conds[1] < conds[2] < conds[3]   # Table 1: cond(S) grows with r_e


def test_pu_reproduction_and_density_of_enrichment():
    """Coefficients b = 1 on every enriched vertex give psi^h = Psi (sum phi^PU = 1)."""
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=5, r_c=1.9, r_e=3.5)  # enrich every vertex
    m, rules = _setup(wl)
    pts, wts, off = rules
    k = 0  # 1s on atom 0
    c = np.zeros((m.n_dof, 1))
    for j, (al, v) in enumerate(m.enr_dof_info):
        if al == k:
            c[m.n_fe + j, 0] = 1.0
    from oracle import enrich
    al = m.alphas[k]
    psi = enrich.enrichment(al["orb"], al["rc"], al["tau"], m.a, pts, False)
    n = oasm.density(m, rules, c, np.array([1.0]))
    assert np.abs(n - psi ** 2).max() < 1e-13 * max(1.0, (psi ** 2).max())
    _, S = oasm.assemble_HS(m, rules, np.zeros(len(wts)))
    assert abs(c[:, 0] @ (S @ c[:, 0]) - wts @ psi ** 2) < 1e-12


def test_density_and_potential_energy_identities():
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=5)
    m, rules = _setup(wl)
    pts, wts, _ = rules
    V = W.random_potential(len(wts), seed=7)
    H, S = oasm.assemble_HS(m, rules, V)
    H0, _ = oasm.assemble_HS(m, rules, np.zeros(len(wts)))
    C = W.random_coefficients(m.n_dof, 3, seed=8)
    f = np.array([2.0, 1.0, 0.5])
    n = oasm.density(m, rules, C, f)
    assert abs(wts @ n - sum(f[k] * C[:, k] @ (S @ C[:, k]) for k in range(3))) < 1e-10 * abs(wts @ n)
    ev = sum(f[k] * C[:, k] @ ((H - H0) @ C[:, k]) for k in range(3))
    assert abs(ev - wts @ (V * n)) < 1e-10 * abs(ev)


def test_adjoint_matches_finite_difference():
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=4)
    m, rules = _setup(wl)
    nq = len(rules[1])
    V = W.random_potential(nq, seed=1)
    H, _ = oasm.assemble_HS(m, rules, V)
    Hbar = H.copy()
    Hbar.data = W.random_symmetric_values(H.nnz, seed=3)
    Hbar = (Hbar + Hbar.T) * 0.5
    g = oasm.adjoint_V(m, rules, Hbar)
    rng = np.random.default_rng(0)
    for q in rng.choice(nq, 6, replace=False):
        dv = np.zeros(nq)
        dv[q] = 1e-3
        Hp, _ = oasm.assemble_HS(m, rules, V + dv)
        Hm, _ = oasm.assemble_HS(m, rules, V - dv)
        fd = (Hbar.multiply(Hp - Hm)).sum() / 2e-3
        assert abs(fd - g[q]) < 1e-9 * max(1.0, abs(g[q]))


def test_translation_by_mesh_vector_preserves_spectrum():
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=5)
    m, rules = _setup(wl)
    V = opot.ionic_potential(wl, rules[0])
    H, S = oasm.assemble_HS(m, rules, V)
    w0, _ = oeig.lowest_eigs(H, S, 4)
    wl2 = dict(wl)
    wl2["atoms"] = [(s, tuple(np.array(t) + np.array([2.0, 0.0, 2.0]))) for s, t in wl["atoms"]]
    m2, rules2 = _setup(wl2)
    V2 = opot.ionic_potential(wl2, rules2[0])
    H2, S2 = oasm.assemble_HS(m2, rules2, V2)
    w2, _ = oeig.lowest_eigs(H2, S2, 4)
    assert np.abs(w0 - w2).max() < 1e-10


def test_fermi_occupations_sum():
    eps = np.array([-1.0, -0.5, -0.5, 0.2, 0.3])
    f, mu = oeig.fermi_occupations(eps, 5.0, 0.01)
    assert abs(f.sum() - 5.0) < 1e-10
    assert np.all((f >= 0) & (f <= 2))
    assert abs(f[1] - f[2]) < 1e-15


# ---------------------------------------------------------------------------
# Pins of the enrichment columns' gradients (the enriched kinetic block).
#
# The trilinear PU reproduces every multilinear function exactly: for the 8
# monomials m(xi) = xi^a eta^b zeta^c (a, b, c in {0, 1}) of the reference
# coordinates, sum_v phi_v(x) m(xi_v) = m(xi(x)) on an element (Sec. 2 eq. pum:
# the PU sums to one, and the trilinear space contains these functions).  So
# the coefficient vector b_v = m(xi_v) on an enrichment's 8 columns of one
# element represents m Psi there, whose gradient Psi grad m + m grad Psi is a
# closed form of grad m (= (2/h) times the reference gradient of the monomial)
# and the enrichment's own value and gradient.  With P[v, m] = m(xi_v) (an
# invertible 8 x 8 matrix) the element's E x E block is therefore fixed
# entirely:  P^T H_e P = sum_q w_q [1/2 grad(m Psi_a) . grad(m' Psi_b)
# + V_q m m' Psi_a Psi_b]  (Sec. 4 eq. disceig3d).  Likewise the tricubic FE
# functions reproduce every polynomial t of degree <= 3 per axis, which fixes
# the FE x E block through u_i = t(xi_i).  A dropped Psi grad phi term, a
# wrong 2/h scale or a permuted vertex in the PU gradient fails these.
# ---------------------------------------------------------------------------
from oracle import enrich as oenr, fe as ofe


def _monomials(xi, h):
    """The 8 multilinear monomials at reference points xi (Q, 3): values
    (Q, 8) and physical gradients (3, Q, 8); index a + 2b + 4c."""
    Q = xi.shape[0]
    val = np.ones((Q, 8))
    grad = np.zeros((3, Q, 8))
    for k in range(8):
        e = [(k >> d) & 1 for d in range(3)]
        f = [xi[:, d] if e[d] else np.ones(Q) for d in range(3)]
        val[:, k] = f[0] * f[1] * f[2]
        for d in range(3):
            if e[d]:
                g = np.ones(Q) * (2.0 / h)
                for d2 in range(3):
                    if d2 != d:
                        g = g * f[d2]
                grad[d, :, k] = g
    return val, grad


def _vertex_matrix():
    """P[v, m] = m(xi_v) for the 8 element vertices v = a + 2b + 4c at xi = +-1."""
    P = np.zeros((8, 8))
    for v in range(8):
        x = np.array([2.0 * ((v >> d) & 1) - 1.0 for d in range(3)])
        P[v] = _monomials(x[None, :], 1.0)[0][0]
    return P


def _tricubic_poly(xi, h, powers):
    """t(xi) = xi^i eta^j zeta^k and its physical gradient, for i, j, k <= 3."""
    i, j, k = powers
    x, y, z = xi[:, 0], xi[:, 1], xi[:, 2]
    t = x ** i * y ** j * z ** k
    s = 2.0 / h
    gx = (i * x ** max(i - 1, 0)) * y ** j * z ** k * s
    gy = x ** i * (j * y ** max(j - 1, 0)) * z ** k * s
    gz = x ** i * y ** j * (k * z ** max(k - 1, 0)) * s
    return t, np.stack([gx, gy, gz])


def _enriched_element_identities(m, rules, e, V):
    """Largest deviation of the oracle's element blocks from the closed forms
    above (E x E and FE x E, H and S), relative to the block maxima."""
    pts, wts, off = rules
    s = slice(off[e], off[e + 1])
    p, w, v = pts[s], wts[s], V[s]
    He, Se = oasm.element_HS(m, e, p, w, v)
    lo, _ = m.elem_box(e)
    xi = 2.0 * (p - lo) / m.h - 1.0
    mono, gmono = _monomials(xi, m.h)
    Pv = _vertex_matrix()
    nf = m.nfe_e   # FE columns: 64 tricubic or 32 serendipity
    by_alpha = {}
    for j, (dof, lv, k) in enumerate(m.elem_cols[e]):
        by_alpha.setdefault(k, {})[lv] = nf + j
    full = {k: c for k, c in by_alpha.items() if len(c) == 8}
    assert full, "the element needs an enrichment on all 8 vertices"
    psi = {}
    for k in full:
        al = m.alphas[k]
        psi[k] = oenr.enrichment(al["orb"], al["rc"], al["tau"], m.a, p)
    hs, ss = np.abs(He).max(), np.abs(Se).max()   # scales of the element matrices
    worst = 0.0
    for ka in full:
        ca = [full[ka][lv] for lv in range(8)]
        pa, ga = psi[ka]
        fa = mono * pa[:, None]                                  # m Psi_a   (Q, 8)
        Ga = gmono * pa[None, :, None] + mono[None] * ga[:, :, None]
        for kb in full:
            cb = [full[kb][lv] for lv in range(8)]
            pb, gb = psi[kb]
            fb = mono * pb[:, None]
            Gb = gmono * pb[None, :, None] + mono[None] * gb[:, :, None]
            Hc = 0.5 * np.einsum("dqi,q,dqj->ij", Ga, w, Gb) + np.einsum("qi,q,qj->ij", fa, w * v, fb)
            Sc = np.einsum("qi,q,qj->ij", fa, w, fb)
            Ho = Pv.T @ He[np.ix_(ca, cb)] @ Pv
            So = Pv.T @ Se[np.ix_(ca, cb)] @ Pv
            worst = max(worst, np.abs(Ho - Hc).max() / hs, np.abs(So - Sc).max() / ss)
        # FE x E through the FE space's reproduction u_i = t(node_i): any
        # polynomial of degree <= 3 per axis for the tricubic space; the
        # cubic serendipity space's own monomials (P3 and the superlinear
        # ones) for the serendipity space
        nodes = np.array([[ofe.CUBIC_NODES[i & 3], ofe.CUBIC_NODES[(i >> 2) & 3],
                           ofe.CUBIC_NODES[i >> 4]] for i in m.fe_local])
        polys = (((0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 1, 2), (2, 3, 3)) if nf == 64 else
                 ((0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 1, 1), (1, 1, 3)))
        for powers in polys:
            u = _tricubic_poly(nodes, m.h, powers)[0]
            t, gt = _tricubic_poly(xi, m.h, powers)
            hc = 0.5 * np.einsum("dq,q,dqj->j", gt, w, Ga) + np.einsum("q,q,qj->j", t, w * v, fa)
            sc = np.einsum("q,q,qj->j", t, w, fa)
            ho = u @ He[:nf, ca] @ Pv
            so = u @ Se[:nf, ca] @ Pv
            worst = max(worst, np.abs(ho - hc).max() / hs, np.abs(so - sc).max() / ss)
    return worst


def _all_enriched_cell(nel):
    return W.small_two_atom(nel=nel, a=4.0, quad_p=6, r_c=1.9, r_e=3.5)


def test_enriched_blocks_reproduce_multilinear_times_enrichment():
    """E x E and FE x E blocks of H and S on enriched elements against the
    closed forms of the PU and FE reproduction properties, with V = 0 and a
    random V, on a 2^3 and a 3^3 cell (several enrichments per element)."""
    for nel in (2, 3):
        m, rules = _setup(_all_enriched_cell(nel))
        nq = len(rules[1])
        for V in (np.zeros(nq), W.random_potential(nq, seed=31)):
            for e in (0, m.nelem - 1):
                assert _enriched_element_identities(m, rules, e, V) < 1e-12, (nel, e)


def test_enriched_blocks_on_the_serendipity_space():
    """The same closed forms with the cubic serendipity FE part (its FE x E
    block through the serendipity space's own reproduced monomials)."""
    for nel in (2, 3):
        m, rules = _setup(dict(_all_enriched_cell(nel), fe="serendipity32"))
        assert m.nfe_e == 32
        nq = len(rules[1])
        for V in (np.zeros(nq), W.random_potential(nq, seed=33)):
            for e in (0, m.nelem - 1):
                assert _enriched_element_identities(m, rules, e, V) < 1e-12, (nel, e)


def test_enrichment_times_one_global_kinetic_identity():
    """b = 1 on every PU vertex of one enrichment gives psi^h = Psi (sum
    phi^PU = 1), so c^T H c = 1/2 sum_q w_q |grad Psi|^2 + sum_q w_q V Psi^2
    and c^T S c = sum_q w_q Psi^2 over the whole cell."""
    for nel in (2, 3):
        m, rules = _setup(_all_enriched_cell(nel))
        pts, wts, _ = rules
        nq = len(wts)
        for k in (0, 2, 4):
            c = np.zeros(m.n_dof)
            for j, (al, v) in enumerate(m.enr_dof_info):
                if al == k:
                    c[m.n_fe + j] = 1.0
            al = m.alphas[k]
            psi, g = oenr.enrichment(al["orb"], al["rc"], al["tau"], m.a, pts)
            for V in (np.zeros(nq), W.random_potential(nq, seed=32)):
                H, S = oasm.assemble_HS(m, rules, V)
                want_h = 0.5 * wts @ (g * g).sum(axis=0) + wts @ (V * psi * psi)
                want_s = wts @ (psi * psi)
                assert abs(c @ (H @ c) - want_h) < 1e-12 * abs(want_h), (nel, k)
                assert abs(c @ (S @ c) - want_s) < 1e-12 * want_s, (nel, k)


@pytest.mark.parametrize("mistake", ["dropped_psi_grad_phi", "permuted_vertex", "half_scale"])
def test_enriched_block_pin_catches_planted_mistakes(monkeypatch, mistake):
    """Plant a plausible mistake in the oracle's PU gradient (on the CPU) and
    check that the multilinear-reproduction pin rejects it."""
    good = ofe.trilinear

    def bad(xi):
        N, dN = good(xi)
        if mistake == "dropped_psi_grad_phi":
            dN = 0.0 * dN
        elif mistake == "permuted_vertex":
            dN = dN[:, :, [1, 0, 2, 3, 4, 5, 6, 7]]
        else:
            dN = 0.5 * dN
        return N, dN

    m, rules = _setup(_all_enriched_cell(2))
    V = W.random_potential(len(rules[1]), seed=33)
    assert _enriched_element_identities(m, rules, 0, V) < 1e-12
    monkeypatch.setattr(oasm, "trilinear", bad)
    assert _enriched_element_identities(m, rules, 0, V) > 1e-4
