"""Self-consistent-field pieces (oracle, test infrastructure only).

Sec. 3 of the paper: the effective potential of the Kohn-Sham equations is
V_eff = V_C + V_xc.  The total Coulomb potential V_C = V_I + V_H comes from
one Poisson equation for the total charge rho = rho_I + rho_e (eq. poisson,
del^2 V_C = 4 pi rho), with the ionic charges rho_I localized Gaussians and
rho_e = -n the electronic charge (eq. rhoe).  The cell is neutral, so the
periodic solution exists; it is fixed by a zero cell average.  V_xc is the
LDA (the paper names the LDA, not its parametrisation): Perdew-Zunger 1981
fit of the Ceperley-Alder correlation, unpolarised, plus Dirac exchange.
The fixed-point (SCF) iteration of Sec. 3 (fig. scf) is taken one step at a
time: occupations by Fermi-Dirac smearing, the output density, linear or
Pulay mixing, the new effective potential, and the total energy

    E = sum_k f_k eps_k - int n_out V_eff,in + E_es[n_out] - E_self
        + E_xc[n_out] - kT S,
    E_es = -1/2 int (rho_I - n) V_C[n],   E_self = sum_a Z_a^2 / (sigma_a sqrt(2 pi)),
    E_xc = int n eps_xc(n),   S = -2 sum_k [g ln g + (1 - g) ln(1 - g)], g = f_k / 2,

(the paper computes total energies as in an earlier work that it does not
restate; this is the Kohn-Sham energy with the Gaussian ions' self-energy
removed).  Every integral uses the shared element quadrature rule.

Poisson in the classical FE space (Sec. 3: the tricubic functions of the
mesh): weak form  -K v = 4 pi b  with  K_ij = int grad phi_i . grad phi_j
(exact: a 4-point Gauss rule per element) and  b_i = int phi_i rho  (shared
rule), solved by a sparse direct solve with one DOF pinned, then shifted to
zero cell average (int V = m^T v, m_i = int phi_i).  The net charge that the
quadrature leaves (the rule integrates the ionic Gaussians only to its
accuracy) is spread as a uniform background: b -= (sum_i b_i / Omega) m.

Pins (tests/test_oracle_scf.py): the LDA's exchange constant in its
(9 pi / 4)^(1/3) form, v_xc = d(n eps_xc)/dn by complex-step
differentiation, continuity of the PZ81 correlation at r_s = 1 and its
high-density coefficient against (1 - ln 2) / pi^2; Poisson against the
closed-form solution for a single Fourier mode and against the reciprocal-
space ionic potential, both with their O(h^4) convergence; the energy's
invariance under a constant shift of V_eff and eigenvalues, and
E_es >= 0 for a neutral charge.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assemble import density
from .bloch import density_k
from .eig import fermi_occupations, fermi_occupations_k
from .fe import gauss_1d, tricubic
from .potential import gaussian_charge

# Perdew-Zunger 1981, unpolarised correlation
_PZ_GAMMA, _PZ_B1, _PZ_B2 = -0.1423, 1.0529, 0.3334
_PZ_A, _PZ_B, _PZ_C, _PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def lda_exchange(n):
    """Dirac exchange of the uniform gas: eps_x = -(3/4)(3 n / pi)^(1/3),
    v_x = d(n eps_x)/dn = (4/3) eps_x."""
    ex = -0.75 * (3.0 * n / math.pi) ** (1.0 / 3.0)
    return ex, 4.0 / 3.0 * ex


def pz81_correlation(rs):
    """Perdew-Zunger 1981 unpolarised correlation eps_c(r_s) and v_c(r_s)."""
    rs = np.asarray(rs)
    ec = np.zeros(rs.shape, dtype=rs.dtype)
    vc = np.zeros(rs.shape, dtype=rs.dtype)
    hi = np.real(rs) >= 1.0
    r = rs[hi]
    sq = np.sqrt(r)
    den = 1.0 + _PZ_B1 * sq + _PZ_B2 * r
    ec[hi] = _PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * _PZ_B1 * sq + 4.0 / 3.0 * _PZ_B2 * r) / den
    r = rs[~hi]
    lr = np.log(r)
    ec[~hi] = _PZ_A * lr + _PZ_B + _PZ_C * r * lr + _PZ_D * r
    vc[~hi] = (_PZ_A * lr + (_PZ_B - _PZ_A / 3.0) + 2.0 / 3.0 * _PZ_C * r * lr
               + (2.0 * _PZ_D - _PZ_C) / 3.0 * r)
    return ec, vc


def pz81(n):
    """LDA energy per electron eps_xc(n) and potential v_xc(n); 0 where n <= 1e-30."""
    n = np.asarray(n)
    out_e = np.zeros(n.shape, dtype=n.dtype)
    out_v = np.zeros(n.shape, dtype=n.dtype)
    pos = np.real(n) > 1e-30
    nn = n[pos]
    rs = (3.0 / (4.0 * math.pi * nn)) ** (1.0 / 3.0)
    ex, vx = lda_exchange(nn)
    ec, vc = pz81_correlation(rs)
    out_e[pos] = ex + ec
    out_v[pos] = vx + vc
    return out_e, out_v


def fe_stiffness(mesh):
    """K_ij = int grad phi_i . grad phi_j over the tricubic FE space (N_fe^2)."""
    x1, w1 = gauss_1d(4)
    X = np.array(np.meshgrid(x1, x1, x1, indexing="ij")).reshape(3, -1).T[:, ::-1]
    W = np.einsum("i,j,k->ijk", w1, w1, w1).reshape(-1)   # ordering irrelevant: symmetric
    _, dN = tricubic(X)
    h = mesh.h
    G = dN * (2.0 / h)
    Ke = np.einsum("q,dqi,dqj->ij", W * (h / 2.0) ** 3, G, G)
    rows, cols, vals = [], [], []
    for e in range(mesh.nelem):
        d = mesh.elem_dofs(e)[:64]
        rows.append(np.repeat(d, 64))
        cols.append(np.tile(d, 64))
        vals.append(Ke.reshape(-1))
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.n_fe, mesh.n_fe))
    return K


def fe_load(mesh, rules, f):
    """b_i = int phi_i f over the FE functions, on the shared rule."""
    pts, wts, off = rules
    b = np.zeros(mesh.n_fe)
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        if off[e + 1] == off[e]:
            continue
        lo, _ = mesh.elem_box(e)
        xi = 2.0 * (pts[s] - lo) / mesh.h - 1.0
        N, _ = tricubic(xi)
        np.add.at(b, mesh.elem_dofs(e)[:64], N.T @ (wts[s] * f[s]))
    return b


def fe_interp(mesh, rules, v):
    """sum_i v_i phi_i at every quadrature point."""
    pts, wts, off = rules
    out = np.zeros(len(wts))
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        if off[e + 1] == off[e]:
            continue
        lo, _ = mesh.elem_box(e)
        xi = 2.0 * (pts[s] - lo) / mesh.h - 1.0
        N, _ = tricubic(xi)
        out[s] = N @ v[mesh.elem_dofs(e)[:64]]
    return out


def coulomb_potential(mesh, rules, rho, K=None):
    """V_C with del^2 V_C = 4 pi rho (rho neutral), zero cell average.

    Returns the FE coefficients v and V_C at the quadrature points."""
    if K is None:
        K = fe_stiffness(mesh)
    b = fe_load(mesh, rules, rho)
    # the shared rule integrates the ionic Gaussians only approximately, so
    # the discrete total charge sum_i b_i may differ slightly from zero: it
    # is spread as a uniform background (b -= (sum b / Omega) m), the
    # compatibility condition of the periodic problem
    m = fe_load(mesh, rules, np.ones(len(rules[1])))      # m_i = int phi_i
    b = b - (b.sum() / m.sum()) * m
    rhs = -4.0 * math.pi * b
    # pin DOF 0 (K is singular: constants), then shift to zero average
    Kp = K.tolil()
    Kp[0, :] = 0.0
    Kp[:, 0] = 0.0
    Kp[0, 0] = 1.0
    rhs = rhs.copy()
    rhs[0] = 0.0
    v = spla.spsolve(Kp.tocsc(), rhs)
    v = v - (m @ v) / m.sum()
    return v, fe_interp(mesh, rules, v)


def ion_density(wl, pts):
    """rho_I at the points: the Gaussian ionic charges of the workload."""
    return gaussian_charge(wl, pts)


def self_energy(wl):
    return sum(wl["species"][s]["Z"] ** 2 / (wl["species"][s]["sigma"] * math.sqrt(2.0 * math.pi))
               for s, _ in wl["atoms"])


def effective_potential(mesh, rules, n, rho_I, K=None):
    """V_eff = V_C[rho_I - n] + v_xc(n); also returns V_C and eps_xc."""
    _, VC = coulomb_potential(mesh, rules, rho_I - n, K)
    exc, vxc = pz81(n)
    return VC + vxc, VC, exc


def entropy(f):
    g = np.clip(np.asarray(f) / 2.0, 1e-300, 1.0 - 1e-16)
    t = g * np.log(g) + (1.0 - g) * np.log1p(-g)
    t[(g <= 1e-300) | (g >= 1.0 - 1e-16)] = 0.0
    return -2.0 * t.sum()


class PulayMixer:
    """Pulay (DIIS / Anderson) density mixing: with the last `depth` input
    densities n_i and residuals R_i = n_out,i - n_i, the coefficients c
    minimise || sum_i c_i R_i ||_w (w: the quadrature weights) subject to
    sum_i c_i = 1, and n_new = sum_i c_i (n_i + alpha R_i).  depth = 1 is
    linear mixing."""

    def __init__(self, depth):
        self.depth = int(depth)
        self.n, self.R = [], []

    def mix(self, n_in, n_out, w, alpha):
        self.n.append(np.array(n_in, copy=True))
        self.R.append(np.asarray(n_out) - n_in)
        if len(self.n) > self.depth:
            self.n.pop(0)
            self.R.pop(0)
        m = len(self.R)
        A = np.array([[w @ (self.R[i] * self.R[j]) for j in range(m)] for i in range(m)])
        A += 1e-12 * np.trace(A) / m * np.eye(m)          # keeps near-parallel residuals solvable
        M = np.zeros((m + 1, m + 1))
        M[:m, :m] = A
        M[:m, m] = M[m, :m] = 1.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        c = np.linalg.solve(M, rhs)[:m]
        return sum(c[i] * (self.n[i] + alpha * self.R[i]) for i in range(m))


def scf_step(mesh, rules, wl, eps, C, nelec, kT, alpha, n_in, V_eff_in, rho_I, K=None,
             mixer=None):
    """One fixed-point step (Sec. 3, fig. scf) after the eigensolve.

    eps (k,), C (N, k): the lowest states of H[V_eff_in].  Returns a dict with
    the occupations, n_out, n_new = n_in + alpha (n_out - n_in) (or the Pulay
    mix of `mixer`), V_eff[n_new],
    the energy terms of n_out and the residual int |n_out - n_in|."""
    f, mu = fermi_occupations(eps, nelec, kT)
    n_out = density(mesh, rules, C, f)
    return _finish(mesh, rules, wl, f, mu, n_out, float(f @ eps), -kT * entropy(f), alpha, n_in,
                   V_eff_in, rho_I, K, mixer)


def scf_step_k(mesh, rules, wl, kpts, wk, eps, C, nelec, kT, alpha, n_in, V_eff_in, rho_I,
               K=None, mixer=None):
    """One fixed-point step with k-point sampling (Sec. 4, eqs. bloch, strong:
    Bloch states at wavevectors k; Sec. 3 for the rest).

    kpts (nk, 3) Cartesian wavevectors, wk their weights (summing to 1),
    eps[i] and C[i] (N, n_i) complex: the lowest states of H(k_i)[V_eff_in].
    One Fermi level for all k (fermi_occupations_k); the output density, the
    band energy and the entropy are the k-weighted sums
        n_out = sum_k w_k sum_n f_nk |psi_nk|^2,  e_band = sum_k w_k sum_n f_nk eps_nk,
        S = sum_k w_k S(f_k);
    the rest as scf_step."""
    f, mu = fermi_occupations_k(eps, wk, nelec, kT)
    n_out = sum(w * density_k(mesh, rules, Ck, fk, k) for w, Ck, fk, k in zip(wk, C, f, kpts))
    e_band = float(sum(w * (fk @ np.asarray(ek)) for w, fk, ek in zip(wk, f, eps)))
    e_ts = -kT * float(sum(w * entropy(fk) for w, fk in zip(wk, f)))
    return _finish(mesh, rules, wl, f, mu, n_out, e_band, e_ts, alpha, n_in, V_eff_in, rho_I, K,
                   mixer)


def _finish(mesh, rules, wl, f, mu, n_out, e_band, e_ts, alpha, n_in, V_eff_in, rho_I, K, mixer):
    """The energy terms of n_out, the mixing and V_eff of the mixed density."""
    w = rules[1]
    _, VC_out = coulomb_potential(mesh, rules, rho_I - n_out, K)
    exc_out, _ = pz81(n_out)
    e_dc = -float(w @ (n_out * V_eff_in))
    e_es = -0.5 * float(w @ ((rho_I - n_out) * VC_out))
    e_xc = float(w @ (n_out * exc_out))
    e_self = self_energy(wl)
    if mixer is None:
        n_new = n_in + alpha * (n_out - n_in)
    else:
        n_new = mixer.mix(n_in, n_out, w, alpha)
    V_new, _, _ = effective_potential(mesh, rules, n_new, rho_I, K)
    return dict(f=f, mu=mu, n_out=n_out, n_new=n_new, V_eff=V_new, e_band=e_band, e_dc=e_dc,
                e_es=e_es, e_self=e_self, e_xc=e_xc, e_ts=e_ts,
                e_total=e_band + e_dc + e_es - e_self + e_xc + e_ts,
                residual=float(w @ np.abs(n_out - n_in)))
