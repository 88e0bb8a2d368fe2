"""Pins of the oracle on general (triclinic) cells: the paper's CeAl lattice
(Sec. 6.2, eq. ceal-primitive) with parallelepiped elements and a constant
Jacobian (CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble as oasm, eig as oeig, enrich as oenr, fe as ofe
from oracle import mesh as omesh, potential as opot, quadrature as oq
from paper_1611_00731_gb300 import workloads as W


def _setup(wl):
    m = omesh.Mesh(wl)
    return m, oq.all_rules(m)


def test_mapped_elements_partition_of_unity_and_weights():
    m, (pts, wts, off) = _setup(W.sheared_empty(nel=2, p=5))
    L = np.array(W.sheared_empty()["lattice"])
    vol = abs(np.linalg.det(L))
    assert abs(wts.sum() - vol) < 1e-12 * vol
    for e in range(m.nelem):
        s = slice(off[e], off[e + 1])
        assert abs(wts[s].sum() - vol / m.nelem) < 1e-12 * vol
        # lattice coordinates of the element's points stay inside its range
        frac = np.linalg.solve(L.T, pts[s].T).T * m.nel - np.array(m.elem_coords(e))
        assert frac.min() > 0.0 and frac.max() < 1.0
        B, G = oasm.element_basis(m, e, pts[s])
        assert np.abs(B.sum(axis=1) - 1.0).max() < 1e-13          # sum N_i = 1
        assert np.abs(G.sum(axis=2)).max() < 1e-12                 # sum grad N_i = 0
    # trilinear PU on a mapped element, gradients against central differences
    e = 3
    x0 = m.elem_origin(e)
    xi = np.array([[0.3, -0.2, 0.5]])
    x = x0 + (xi + 1.0) @ m.J.T
    P, dP = ofe.trilinear(m.to_reference(e, x))
    assert abs(P.sum() - 1.0) < 1e-15
    g = m.grad_to_physical(dP)[:, 0, :]
    for d in range(3):
        dx = np.zeros(3)
        dx[d] = 1e-6
        fd = (ofe.trilinear(m.to_reference(e, x + dx))[0] -
              ofe.trilinear(m.to_reference(e, x - dx))[0])[0] / 2e-6
        assert np.abs(fd - g[d]).max() < 1e-8


def test_parallelepiped_distance_against_brute_force():
    rng = np.random.default_rng(4)
    M = np.array([[2.0, 0.3, -0.2], [0.1, 1.7, 0.4], [0.2, -0.3, 2.2]])
    x0 = np.array([0.5, -0.2, 0.1])
    P = rng.uniform(-3.0, 5.0, size=(40, 3))
    d = omesh.parallelepiped_dist(x0, M, P)
    t = np.linspace(0.0, 1.0, 41)
    T = np.array(np.meshgrid(t, t, t, indexing="ij")).reshape(3, -1).T
    Q = x0 + T @ M.T
    brute = np.sqrt(((P[:, None, :] - Q[None]) ** 2).sum(axis=2)).min(axis=1)
    step = np.linalg.norm(M, axis=0).sum() / 40          # farthest a grid point can be
    assert np.all(d <= brute + 1e-12) and np.all(d >= brute - step)
    inside = x0 + np.array([0.3, 0.6, 0.2]) @ M.T
    assert omesh.parallelepiped_dist(x0, M, inside[None])[0] < 1e-12


def test_sheared_empty_lattice_spectrum_and_rate():
    """V = 0 without enrichment on the CeAl lattice: eigenvalues bound the
    free-electron levels |G|^2 / 2 (G on the reciprocal lattice) from above,
    the constant gives 0, and the error falls as O(h^6)."""
    wl = W.sheared_empty()
    G, G2 = opot.reciprocal_vectors(wl, 4.0)
    exact = np.sort(np.concatenate([[0.0], 0.5 * G2]))[:7]
    errs = []
    for nel in (3, 4):
        m, rules = _setup(W.sheared_empty(nel=nel, p=4))
        H, S = oasm.assemble_HS(m, rules, np.zeros(len(rules[1])))
        w, _ = oeig.lowest_eigs(H, S, 7)
        assert abs(w[0]) < 1e-12
        assert np.all(w >= exact - 1e-12)
        errs.append((w - exact)[1:].max())
    rate = math.log(errs[0] / errs[1]) / math.log(4 / 3)
    assert 5.0 < rate < 7.0, (errs, rate)


def test_cubic_cell_written_as_a_lattice_is_the_cubic_assembly():
    wl = W.small_two_atom(nel=2, a=4.0, quad_p=4)
    m0, r0 = _setup(wl)
    wl2 = dict(wl, lattice=[[4.0, 0, 0], [0, 4.0, 0], [0, 0, 4.0]])
    m1, r1 = _setup(wl2)
    assert m1.general and np.array_equal(r0[2], r1[2])
    assert np.abs(r0[0] - r1[0]).max() < 1e-14 and np.abs(r0[1] - r1[1]).max() < 1e-15
    V = W.random_potential(len(r0[1]), seed=5)
    H0, S0 = oasm.assemble_HS(m0, r0, V)
    H1, S1 = oasm.assemble_HS(m1, r1, V)
    assert abs(H1 - H0).max() < 1e-13 * abs(H0).max()
    assert abs(S1 - S0).max() < 1e-13 * abs(S0).max()


def test_general_cell_potential_solves_poisson():
    wl = W.ceal_like(nel=2)
    wl["species"][0]["sigma"], wl["species"][1]["sigma"] = 0.9, 0.8   # a smooth charge
    L = np.array(wl["lattice"])
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 1, size=(8, 3)) @ L
    h = 1e-3
    lap = -6 * opot.ionic_potential(wl, x)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        lap += opot.ionic_potential(wl, x + e) + opot.ionic_potential(wl, x - e)
    lap /= h * h
    Z = sum(wl["species"][s]["Z"] for s, _ in wl["atoms"])
    rho = opot.gaussian_charge(wl, x) - Z / abs(np.linalg.det(L))
    assert np.abs(lap - 4 * math.pi * rho).max() < 2e-4 * np.abs(4 * math.pi * rho).max()


def _monomials(xi, m):
    """The 8 multilinear monomials of the reference coordinates: values (Q, 8)
    and physical gradients (3, Q, 8) through the element's J^-T."""
    Q = xi.shape[0]
    val = np.ones((Q, 8))
    gref = np.zeros((3, Q, 8))
    for k in range(8):
        e = [(k >> d) & 1 for d in range(3)]
        f = [xi[:, d] if e[d] else np.ones(Q) for d in range(3)]
        val[:, k] = f[0] * f[1] * f[2]
        for d in range(3):
            if e[d]:
                gref[d, :, k] = np.prod([f[d2] for d2 in range(3) if d2 != d], axis=0)
    return val, m.grad_to_physical(gref)


def test_mapped_enriched_blocks_reproduce_multilinear_times_enrichment():
    """On a mapped element every vertex of which is enriched, P^T H_e P and
    P^T S_e P for the 8 multilinear monomials equal the closed forms of
    m Psi (PU reproduction, Sec. 2 eq. pum), gradients through J^-T."""
    wl = W.ceal_like(nel=2, r_e=6.0)
    m, (pts, wts, off) = _setup(wl)
    rng = np.random.default_rng(7)
    for e in (0, 5):
        s = slice(off[e], off[e + 1])
        V = rng.uniform(-1, 0, off[e + 1] - off[e])
        He, Se = oasm.element_HS(m, e, pts[s], wts[s], V)
        xi = m.to_reference(e, pts[s])
        mono, gmono = _monomials(xi, m)
        Pv = np.array([_monomials(np.array([[2.0 * ((v >> d) & 1) - 1.0 for d in range(3)]]),
                                  m)[0][0] for v in range(8)])
        cols = {}
        for j, (dof, lv, k) in enumerate(m.elem_cols[e]):
            cols.setdefault(k, {})[lv] = 64 + j
        full = [k for k, c in cols.items() if len(c) == 8]
        assert full
        for k in full[:3]:
            al = m.alphas[k]
            psi, gpsi = oenr.enrichment(al["orb"], al["rc"], al["tau"], m.lattice, pts[s])
            f = mono * psi[:, None]
            G = gmono * psi[None, :, None] + mono[None] * gpsi[:, :, None]
            Hc = 0.5 * np.einsum("dqi,q,dqj->ij", G, wts[s], G) + np.einsum("qi,q,qj->ij", f, wts[s] * V, f)
            Sc = np.einsum("qi,q,qj->ij", f, wts[s], f)
            c = [cols[k][lv] for lv in range(8)]
            assert np.abs(Pv.T @ He[np.ix_(c, c)] @ Pv - Hc).max() < 1e-12 * np.abs(He).max()
            assert np.abs(Pv.T @ Se[np.ix_(c, c)] @ Pv - Sc).max() < 1e-12 * np.abs(Se).max()


def test_ceal_like_cell_pu_reproduction_and_spd():
    wl = W.ceal_like(nel=2, r_e=6.0)
    m, rules = _setup(wl)
    pts, wts, _ = rules
    H, S = oasm.assemble_HS(m, rules, np.zeros(len(wts)))
    Sd = S.toarray()
    assert np.abs(Sd - Sd.T).max() < 1e-15 * np.abs(Sd).max()
    sla.cholesky(Sd)
    k = 0
    c = np.zeros(m.n_dof)
    for j, (al, v) in enumerate(m.enr_dof_info):
        if al == k:
            c[m.n_fe + j] = 1.0
    al = m.alphas[k]
    psi, g = oenr.enrichment(al["orb"], al["rc"], al["tau"], m.lattice, pts)
    assert abs(c @ (S @ c) - wts @ psi ** 2) < 1e-12 * (wts @ psi ** 2)
    assert abs(c @ (H @ c) - 0.5 * wts @ (g * g).sum(axis=0)) < 1e-12 * abs(c @ (H @ c))


def test_general_cell_bloch_hermitian_periodic_gamma_limit():
    """H(k), S(k) on the CeAl lattice: Hermitian, periodic under k -> k + G
    for G on the reciprocal lattice, and the real matrices at k = 0."""
    from oracle import bloch as ob
    wl = W.ceal_like(nel=2)
    m, rules = _setup(wl)
    V = W.random_potential(len(rules[1]), seed=8)
    L = np.array(wl["lattice"])
    B = 2.0 * math.pi * np.linalg.inv(L)
    k = B @ np.array([0.3, -0.2, 0.1])
    H, S = ob.assemble_HS_k(m, rules, V, k)
    assert abs(H - H.conj().T).max() < 1e-14 * abs(H).max()
    assert abs(S - S.conj().T).max() < 1e-14 * abs(S).max()
    H2, S2 = ob.assemble_HS_k(m, rules, V, k + B @ np.array([1.0, 0.0, -1.0]))
    assert abs(H2 - H).max() < 1e-13 * abs(H).max() and abs(S2 - S).max() < 1e-13 * abs(S).max()
    H0, S0 = ob.assemble_HS_k(m, rules, V, np.zeros(3))
    Hr, Sr = oasm.assemble_HS(m, rules, V)
    assert abs(H0 - Hr).max() < 1e-14 * abs(Hr).max() and abs(H0.imag).max() == 0.0
