"""Separable nonlocal projector terms (oracle, test infrastructure only).

Sec. 4 (eq. disceig3d): for a separable nonlocal potential the nonlocal part
of H is  sum_{a,L} f_L^{ai} h_L^a (f_L^{aj})*  with the projections
f_L^{ai} = int phi_i*(x) sum_n v_L^a(x - tau_a - a_n) dx  of the basis onto
the projector functions of atom a (image sum over lattice vectors a_n; at the
Gamma point every phase is 1).  The term is a rank-(number of projectors)
update of H; it is returned as the dense N x P matrix F of projections (the
caller forms H + F h F^T), since two basis functions that meet the same
projector need not share an element (the update fills the sparse pattern).

The paper's projectors come from HGH pseudopotentials, which are not in this
container; the workloads use synthetic Gaussian projectors
    v_{lm}(r) = N_l r^l exp(-r^2 / (2 r_p^2)) Y_lm(r_hat),
    N_l = sqrt(2 / (Gamma(l + 3/2) r_p^(2l + 3)))   (int v^2 = 1),
summed over the images within the range where the Gaussian exceeds 1e-20.
Every integral uses the shared element rule.

Pins (tests/test_oracle_projectors.py): int v_p v_q = delta_pq on a fine product
rule; the projections of an s projector summed over the FE functions (a
partition of unity) equal int v dx = N_0 Y_00 (2 pi r_p^2)^(3/2) to the rule's
accuracy, and those of p projectors vanish by the rule's symmetry about the
atom; F h F^T is symmetric positive semidefinite for h >= 0.

At a wavevector k (Sec. 4, eqs. bloch, strong) the projector is the Bloch sum
p^k(x) = sum_n exp(i k.a_n) v(x - tau - a_n) and the basis function of global
DOF g is its Bloch sum too; on element e, local column i is the image of g_i
shifted by R_i (see oracle/bloch.py), so
    F(k)[g_i, p] += exp(-i k.R_i) sum_q w_q b_i(x_q) p^k(x_q),
and the nonlocal term is F h F^H.  Pins (same test file): k = 0 gives the
real F, F(k + G) = F(k) for a reciprocal lattice vector G, and for the FE
interpolant u = sum_g exp(i k.x_g) phi_g^k of the plane wave exp(i k.x),
sum_g exp(-i k.x_g) F[g, p] approaches int exp(-i k.x) v(x - tau) dx =
exp(-i k.tau) (-i)^l r_p^(2l) N (2 pi r_p^2)^(3/2) |k|^l Y_lm(k_hat)
exp(-|k|^2 r_p^2 / 2)  (the Fourier transform of the Gaussian, written out
for l = 0, 1 in the test) as the mesh is refined.
"""
from __future__ import annotations

import math

import numpy as np

from .assemble import element_basis
from .enrich import real_ylm


def projector_norm(l, rp):
    return math.sqrt(2.0 / (math.gamma(l + 1.5) * rp ** (2 * l + 3)))


def projector_values(proj, a, pts, k=None):
    """sum over images of v_p at the points; proj = dict(tau, l, m, rp).
    With a wavevector k the image at lattice vector a_n carries exp(i k.a_n)
    (complex result)."""
    pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    l, m, rp = int(proj["l"]), int(proj["m"]), float(proj["rp"])
    N = projector_norm(l, rp)
    rcut = rp * math.sqrt(2.0 * 20.0 * math.log(10.0))
    reach = int(math.ceil(rcut / a)) + 1
    out = np.zeros(pts.shape[0], dtype=np.float64 if k is None else np.complex128)
    rng = range(-reach, reach + 1)
    for i in rng:
        for j in rng:
            for kk in rng:
                an = a * np.array([i, j, kk], dtype=np.float64)
                ph = 1.0 if k is None else np.exp(1j * (np.asarray(k, dtype=np.float64) @ an))
                d = pts - np.asarray(proj["tau"]) - an
                r2 = (d * d).sum(axis=1)
                near = r2 < rcut * rcut
                if not near.any():
                    continue
                dd = d[near]
                r = np.sqrt(r2[near])
                # r^l Y_lm, which tends to 0 at the centre for l >= 1
                rly = np.full(len(r), 1.0 / math.sqrt(4.0 * math.pi))
                if l > 0:
                    rly = np.zeros(len(r))
                    pos = r > 0.0
                    rly[pos] = r[pos] ** l * real_ylm(l, m, dd[pos, 0], dd[pos, 1], dd[pos, 2])
                out[near] += ph * N * np.exp(-r2[near] / (2.0 * rp * rp)) * rly
    return out


def projections(mesh, rules, projs):
    """F (N x P): F[i, p] = int phi_i v_p on the shared rule."""
    pts, wts, off = rules
    V = np.stack([projector_values(p, mesh.a, pts) for p in projs], axis=1)
    F = np.zeros((mesh.n_dof, len(projs)))
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        B, _ = element_basis(mesh, e, pts[s])
        np.add.at(F, mesh.elem_dofs(e), B.T @ (wts[s][:, None] * V[s]))
    return F


def projections_k(mesh, rules, projs, k):
    """Complex F(k) (N x P): F[g_i, p] = sum_e exp(-i k.R_i) int b_i p_p^k."""
    from .bloch import elem_phases
    pts, wts, off = rules
    Vk = np.stack([projector_values(p, mesh.a, pts, k) for p in projs], axis=1)
    F = np.zeros((mesh.n_dof, len(projs)), dtype=np.complex128)
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        B, _ = element_basis(mesh, e, pts[s])
        ph = elem_phases(mesh, e, k)
        np.add.at(F, mesh.elem_dofs(e), np.conj(ph)[:, None] * (B.T @ (wts[s][:, None] * Vk[s])))
    return F
