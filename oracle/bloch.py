"""Bloch-periodic (k != 0) H, S, density and adjoint (oracle, test infrastructure).

Sec. 4 (eqs. bloch, strong): at wavevector k the wavefunction satisfies
psi(x + R) = exp(i k.R) psi(x), so the basis functions are Bloch sums of the
cell's functions.  The FE and PU functions of a node or vertex outside the
cell are the images of a cell node shifted by a lattice vector R; the
enrichments are periodic (Sec. 5.1 eq. Psi with f(R) = 1), so the product
phi_v^PU Psi_alpha takes its phase from the PU vertex.  On element e, local
column i is the image of global DOF g_i shifted by R_i, so

    H(k)[g_i, g_j] += exp(-i k.R_i) H_e[i, j] exp(i k.R_j)

with the element matrices H_e, S_e of the Gamma-point assembly (real).  The
density of complex coefficients C is n = sum_k f_k | sum_j B_qj e^{i k.R_j}
C_jk |^2, and the adjoint of V -> H(k) for a complex cotangent Hbar is
dL/dV_q = w_q Re sum_ij conj(Hbar[g_i, g_j]) e^{i k.(R_j - R_i)} b_i b_j
(L = Re sum conj(Hbar) H(k)).

Pins (tests/test_oracle_bloch.py): the empty-lattice spectrum |G + k|^2 / 2
from above with its O(h^6) convergence, H(k) Hermitian, H(k + G) = H(k) for a
reciprocal lattice vector G, k = 0 equals the real assembly, the density
identity sum_q w_q n_q = sum_k f_k c_k^H S(k) c_k, and Brillouin-zone
folding: a 2x2x2 supercell at k_s has the union of the cell's spectra at the
eight wavevectors k_s + (pi/a) m (to 6e-15; conjugating the enrichment
columns' phases alone breaks it by 2e-4).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .assemble import element_HS, element_basis


def elem_shifts(mesh, e):
    """Lattice shift (in cells, per axis, 0 or 1) of every element column."""
    ex, ey, ez = mesh.elem_coords(e)
    m, n = mesh.nfe_axis, mesh.nel
    out = []
    for loc in mesh.fe_local:
        a, b, c = loc & 3, (loc >> 2) & 3, loc >> 4
        out.append(((3 * ex + a) // m, (3 * ey + b) // m, (3 * ez + c) // m))
    for (_, lv, _) in mesh.elem_cols[e]:
        out.append(((ex + (lv & 1)) // n, (ey + ((lv >> 1) & 1)) // n, (ez + (lv >> 2)) // n))
    return np.array(out, dtype=np.int64)


def elem_phases(mesh, e, k):
    """exp(i k . R_i) of every element column, R_i = sum_d shift_d a_d (the
    cubic cell's edge a, or the lattice vectors of a general cell)."""
    sh = elem_shifts(mesh, e)
    R = sh @ mesh.L if mesh.general else sh * mesh.a
    return np.exp(1j * (R @ np.asarray(k, dtype=np.float64)))


def assemble_HS_k(mesh, rules, Vq, k):
    """Complex H(k), S(k) (scipy CSR, complex128)."""
    pts, wts, off = rules
    rows, cols, hv, sv = [], [], [], []
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        He, Se = element_HS(mesh, e, pts[s], wts[s], Vq[s])
        ph = elem_phases(mesh, e, k)
        P = np.conj(ph)[:, None] * ph[None, :]
        d = mesh.elem_dofs(e)
        n = len(d)
        rows.append(np.repeat(d, n))
        cols.append(np.tile(d, n))
        hv.append((P * He).reshape(-1))
        sv.append((P * Se).reshape(-1))
    r, c = np.concatenate(rows), np.concatenate(cols)
    N = mesh.n_dof
    H = sp.csr_matrix((np.concatenate(hv), (r, c)), shape=(N, N))
    S = sp.csr_matrix((np.concatenate(sv), (r, c)), shape=(N, N))
    H.sum_duplicates()
    S.sum_duplicates()
    return H, S


def density_k(mesh, rules, C, f, k):
    """n(x_q) = sum_k f_k |sum_j B_qj e^{i k.R_j} C_{g_j k}|^2, C complex."""
    pts, wts, off = rules
    out = np.zeros(len(wts))
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        B, _ = element_basis(mesh, e, pts[s])
        Y = (B * elem_phases(mesh, e, k)[None, :]) @ C[mesh.elem_dofs(e)]
        out[s] = (np.abs(Y) ** 2) @ f
    return out


def adjoint_V_k(mesh, rules, Hbar, k):
    """dL/dV_q for L = Re sum conj(Hbar) H(k), Hbar complex on the pattern."""
    pts, wts, off = rules
    out = np.zeros(len(wts))
    Hd = Hbar.tocsr()
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        B, _ = element_basis(mesh, e, pts[s])
        d = mesh.elem_dofs(e)
        ph = elem_phases(mesh, e, k)
        Hl = np.real(np.conj(Hd[d][:, d].toarray()) * (np.conj(ph)[:, None] * ph[None, :]))
        out[s] = wts[s] * np.einsum("qi,ij,qj->q", B, Hl, B)
    return out
