"""The oracle's element loops spread over host processes (test helper).

Full-size parity needs the oracle's H and S of a whole workload cell (the
12^3 rocksalt cell has 1,728 elements and 389,664 points).  The oracle stays
exactly as it is: this module only hands disjoint element ranges to worker
processes, each of which runs the oracle's own ``element_rule`` and
``element_HS`` on its range, and sums the partial matrices.  The pool uses the
``spawn`` start method, so no worker inherits a CUDA context from a test
process that has already touched the GPU.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np
import scipy.sparse as sp


def _workers():
    return max(1, min(16, os.cpu_count() or 1))


def _chunks(n, k):
    b = np.linspace(0, n, k + 1).astype(int)
    return [(int(b[i]), int(b[i + 1])) for i in range(k) if b[i + 1] > b[i]]


def _rules_chunk(args):
    wl, lo, hi = args
    from oracle import mesh as omesh, quadrature as oq
    m = omesh.Mesh(wl)
    out = []
    for e in range(lo, hi):
        out.append(oq.element_rule(m, e))
    return out


def _hs_chunk(args):
    wl, lo, hi, pts, wts, V, off = args
    from oracle import assemble as oasm, mesh as omesh
    m = omesh.Mesh(wl)
    rows, cols, hv, sv = [], [], [], []
    for e in range(lo, hi):
        s = slice(off[e] - off[lo], off[e + 1] - off[lo])
        He, Se = oasm.element_HS(m, e, pts[s], wts[s], V[s])
        d = m.elem_dofs(e)
        I, J = np.meshgrid(d, d, indexing="ij")
        rows.append(I.ravel())
        cols.append(J.ravel())
        hv.append(He.ravel())
        sv.append(Se.ravel())
    N = m.n_dof
    r, c = np.concatenate(rows), np.concatenate(cols)
    H = sp.coo_matrix((np.concatenate(hv), (r, c)), shape=(N, N)).tocsr()
    S = sp.coo_matrix((np.concatenate(sv), (r, c)), shape=(N, N)).tocsr()
    return H, S


def _potential_chunk(args):
    wl, pts = args
    from oracle import potential as opot
    return opot.ionic_potential_ewald(wl, pts)


def _pool(nproc):
    return mp.get_context("spawn").Pool(nproc)


def all_rules(wl, nelem, nproc=None):
    """Oracle rules of every element: (points, weights, offsets), as
    ``oracle.quadrature.all_rules`` returns them."""
    nproc = nproc or _workers()
    with _pool(nproc) as pool:
        parts = pool.map(_rules_chunk, [(wl, lo, hi) for lo, hi in _chunks(nelem, 4 * nproc)])
    rules = [r for part in parts for r in part]
    off = np.zeros(len(rules) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(w) for _, w in rules])
    return (np.concatenate([p for p, _ in rules]), np.concatenate([w for _, w in rules]), off)


def assemble_HS(wl, rules, V, nproc=None):
    """Oracle H and S (scipy CSR) of the whole cell: the element matrices of
    ``oracle.assemble.element_HS`` summed over every element."""
    pts, wts, off = rules
    nelem = len(off) - 1
    nproc = nproc or _workers()
    jobs = []
    for lo, hi in _chunks(nelem, 4 * nproc):
        s = slice(off[lo], off[hi])
        jobs.append((wl, lo, hi, pts[s], wts[s], V[s], off))
    with _pool(nproc) as pool:
        parts = pool.map(_hs_chunk, jobs)
    H = parts[0][0]
    S = parts[0][1]
    for h, s in parts[1:]:
        H = H + h
        S = S + s
    H.sum_duplicates()
    S.sum_duplicates()
    return H.tocsr(), S.tocsr()


def ionic_potential(wl, pts, nproc=None):
    """The oracle's Gaussian-ion potential (Ewald-split evaluation) at every
    point, the points split between the workers."""
    nproc = nproc or _workers()
    jobs = [(wl, pts[lo:hi]) for lo, hi in _chunks(len(pts), 4 * nproc)]
    with _pool(nproc) as pool:
        parts = pool.map(_potential_chunk, jobs)
    return np.concatenate(parts)


def dof_grid_coords(wl):
    """Integer positions of every DOF on the (3 nel)^3 node grid of the
    oracle's mesh (FE nodes; enrichment DOFs at their PU vertex), for the
    oracle's nested-dissection order."""
    from oracle import mesh as omesh
    m = omesh.Mesh(wl)
    nf, n = m.nfe_axis, m.nel
    g = np.arange(m.n_fe)
    ev = np.array([v for (_, v) in m.enr_dof_info], dtype=np.int64)
    fe = np.stack([g % nf, (g // nf) % nf, g // (nf * nf)], axis=1)
    en = 3 * np.stack([ev % n, (ev // n) % n, ev // (n * n)], axis=1)
    return np.concatenate([fe, en.reshape(-1, 3)]), nf


def _density_chunk(args):
    wl, lo, hi, pts, C, f, off = args
    from oracle import assemble as oasm, mesh as omesh
    m = omesh.Mesh(wl)
    out = np.zeros(len(pts))
    for e in range(lo, hi):
        s = slice(off[e] - off[lo], off[e + 1] - off[lo])
        B, _ = oasm.element_basis(m, e, pts[s])
        Y = B @ C[m.elem_dofs(e)]
        out[s] = (np.abs(Y) ** 2) @ f
    return out


def density(wl, rules, C, f, nproc=None):
    """The oracle's density n(x_q) = sum_k f_k |psi_k(x_q)|^2 at every point
    (``oracle.assemble.density``, element ranges in parallel)."""
    pts, wts, off = rules
    nproc = nproc or _workers()
    jobs = [(wl, lo, hi, pts[off[lo]:off[hi]], C, f, off)
            for lo, hi in _chunks(len(off) - 1, 4 * nproc)]
    with _pool(nproc) as pool:
        parts = pool.map(_density_chunk, jobs)
    return np.concatenate(parts)
