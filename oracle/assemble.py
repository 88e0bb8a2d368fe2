"""H and S assembly, density and the V -> H adjoint (oracle, test infrastructure).

The discrete eigenproblem of Sec. 4 (eq. disceig3d), at the Gamma point and
with the local potential only:

    H_ij = int ( 1/2 grad phi_i . grad phi_j + phi_i V phi_j ) dx
    S_ij = int phi_i phi_j dx

with every integral replaced by the single shared element quadrature rule of
Sec. 5.2, so that  H = sum_e sum_q w_q [ 1/2 G_q^T G_q + V_q b_q b_q^T ]
and S = sum_e sum_q w_q b_q b_q^T  on the element's basis columns b_q.

The basis of an element (eq. pufebasis): the FE functions (64 tricubic or 32
serendipity, mesh.fe_functions), then
phi_v^PU Psi_alpha for each enrichment column (v, alpha) of the element; its
gradient is Psi grad phi^PU + phi^PU grad Psi.

Density (Sec. 3 eq. rhoe, sign dropped: the electron number density
n = sum_k f_k |psi_k|^2 >= 0 is returned; rho_e = -n):
    n(x_q) = sum_k f_k | sum_j B_qj C_jk |^2.

Adjoint of V -> H: for a cotangent Hbar (same sparsity), dL/dV_q =
w_q b_q^T Hbar_e b_q, summed over the element that owns q.

Parity status: pinned (tests/test_oracle_assembly.py) by exact rational
one-element FE mass/stiffness, the empty-lattice spectrum |G|^2/2, the
harmonic-oscillator spectrum, PU reproduction, the density identity
sum_q w_q n_q = sum_k f_k c_k^T S c_k and finite differences of the adjoint.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .enrich import enrichment
from .fe import trilinear


def element_basis(mesh, e, pts):
    """Basis values B (Q, n) and physical gradients G (3, Q, n) of element e."""
    xi = mesh.to_reference(e, pts)
    N, dN = mesh.fe_functions(xi)
    P, dP = trilinear(xi)
    dN = mesh.grad_to_physical(dN)
    dP = mesh.grad_to_physical(dP)
    cols = mesh.elem_cols[e]
    nf = mesh.nfe_e
    n = nf + len(cols)
    Q = pts.shape[0]
    B = np.zeros((Q, n))
    G = np.zeros((3, Q, n))
    B[:, :nf] = N
    G[:, :, :nf] = dN
    cache = {}
    for j, (dof, lv, k) in enumerate(cols):
        if k not in cache:
            al = mesh.alphas[k]
            cache[k] = enrichment(al["orb"], al["rc"], al["tau"], mesh.lattice, pts)
        psi, gpsi = cache[k]
        B[:, nf + j] = P[:, lv] * psi
        G[:, :, nf + j] = dP[:, :, lv] * psi + P[:, lv] * gpsi
    return B, G


def element_HS(mesh, e, pts, wts, V):
    """Element matrices H_e (n, n) and S_e (n, n) on the element's rule."""
    B, G = element_basis(mesh, e, pts)
    He = 0.5 * np.einsum("dqi,q,dqj->ij", G, wts, G) + np.einsum("qi,q,qj->ij", B, wts * V, B)
    Se = np.einsum("qi,q,qj->ij", B, wts, B)
    return He, Se


def assemble_HS(mesh, rules, Vq):
    """Global H and S (scipy CSR, float64) by element quadrature."""
    pts, wts, off = rules
    rows, cols, hv, sv = [], [], [], []
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        He, Se = element_HS(mesh, e, pts[s], wts[s], Vq[s])
        d = mesh.elem_dofs(e)
        I, J = np.meshgrid(d, d, indexing="ij")
        rows.append(I.ravel())
        cols.append(J.ravel())
        hv.append(He.ravel())
        sv.append(Se.ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    N = mesh.n_dof
    H = sp.coo_matrix((np.concatenate(hv), (rows, cols)), shape=(N, N)).tocsr()
    S = sp.coo_matrix((np.concatenate(sv), (rows, cols)), shape=(N, N)).tocsr()
    H.sum_duplicates()
    S.sum_duplicates()
    return H, S


def assemble_rows(mesh, rules, Vq, dofs):
    """Rows `dofs` of H and S, computed only from the elements touching them.

    Returns dense arrays (len(dofs), N); used to sample full-size outputs.
    """
    pts, wts, off = rules
    want = {int(d): r for r, d in enumerate(dofs)}
    Hr = np.zeros((len(dofs), mesh.n_dof))
    Sr = np.zeros((len(dofs), mesh.n_dof))
    for e in range(mesh.nelem):
        d = mesh.elem_dofs(e)
        hit = [i for i, g in enumerate(d) if int(g) in want]
        if not hit:
            continue
        s = slice(off[e], off[e + 1])
        He, Se = element_HS(mesh, e, pts[s], wts[s], Vq[s])
        for i in hit:
            r = want[int(d[i])]
            np.add.at(Hr[r], d, He[i])
            np.add.at(Sr[r], d, Se[i])
    return Hr, Sr


def density(mesh, rules, C, f):
    """n(x_q) = sum_k f_k |psi_k(x_q)|^2 with psi_k = sum_j phi_j C_jk."""
    pts, wts, off = rules
    out = np.zeros(len(wts))
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        B, _ = element_basis(mesh, e, pts[s])
        Y = B @ C[mesh.elem_dofs(e)]
        out[s] = (np.abs(Y) ** 2) @ f
    return out


def adjoint_V(mesh, rules, Hbar):
    """dL/dV_q = w_q b_q^T Hbar_e b_q for a cotangent Hbar (sparse or dense)."""
    pts, wts, off = rules
    Hd = Hbar.toarray() if sp.issparse(Hbar) else np.asarray(Hbar)
    out = np.zeros(len(wts))
    for e in range(mesh.nelem):
        s = slice(off[e], off[e + 1])
        B, _ = element_basis(mesh, e, pts[s])
        d = mesh.elem_dofs(e)
        He = Hd[np.ix_(d, d)]
        out[s] = wts[s] * np.einsum("qi,ij,qj->q", B, He, B)
    return out
