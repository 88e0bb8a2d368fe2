"""Equation-of-state sweep and the fourth-order Birch-Murnaghan fit.

Sec. 6 computes the LiH energy-volume curve at a series of lattice constants
and fits a fourth-order Birch-Murnaghan form to it (Table 2: V_0, a_0, B_0).
Here one self-consistent field (Sec. 3) runs per lattice constant on the GPU:
every iteration replays the H/S assemblies of all cells (and of all their
k-points, Sec. 4 eqs. bloch, strong) from one captured CUDA graph, takes each
cell's lowest states from a host FP64 generalized eigensolve (LAPACK; the
eigensolver is not part of the library), and calls pufe_scf_step (or
pufe_scf_step_bloch) for the occupations, output density, energy terms, Pulay
mixing and the next potential.  The fit is host arithmetic on the converged
energies.
"""
from __future__ import annotations

import numpy as np
import numpy.polynomial.polynomial as P
import scipy.linalg as sla
import scipy.sparse as sp

from . import pufe

HA_PER_BOHR3_IN_GPA = 29421.02648438959

# The 1/4-shifted 2x2x2 Monkhorst-Pack grid reduced by time reversal (k and
# -k carry the same density and eigenvalues): four k-points in units of
# 2 pi / a per axis, equal weights.
MP2_SHIFTED = ([(0.25, 0.25, 0.25), (0.25, 0.25, -0.25), (0.25, -0.25, 0.25),
                (-0.25, 0.25, 0.25)], [0.25, 0.25, 0.25, 0.25])


def birch_murnaghan4_fit(V, E):
    """Least-squares fourth-order Birch-Murnaghan fit of E(V).

    The n-th order form is a polynomial of degree n in the Eulerian strain
    f = ((V_0/V)^(2/3) - 1) / 2, which is affine in t = V^(-2/3); the fit is
    therefore E = sum_{k<=4} c_k t^k.  Returns dict(V0, E0, B0, B0p, coeffs,
    rms): the minimum of the fitted curve nearest the samples, the bulk modulus
    B0 = V d2E/dV2 (Ha/bohr^3) and its pressure derivative B0' there."""
    V = np.asarray(V, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    if V.shape != E.shape or V.size < 5:
        raise ValueError("need at least 5 (V, E) samples of the same shape")
    t = V ** (-2.0 / 3.0)
    c, *_ = np.linalg.lstsq(np.vander(t, 5, increasing=True), E, rcond=None)
    d1, d2, d3 = P.polyder(c, 1), P.polyder(c, 2), P.polyder(c, 3)
    roots = P.polyroots(d1)
    span = t.max() - t.min()
    cand = [r.real for r in roots if abs(r.imag) <= 1e-12 * abs(r.real)
            and t.min() - span <= r.real <= t.max() + span and P.polyval(r.real, d2) > 0]
    if not cand:
        raise ValueError("the fitted curve has no minimum near the sampled volumes")
    t0 = min(cand, key=lambda r: abs(r - t.mean()))
    V0 = t0 ** -1.5
    Et, Ett, Ettt = P.polyval(t0, d1), P.polyval(t0, d2), P.polyval(t0, d3)
    tV = -2.0 / 3.0 * V0 ** (-5.0 / 3.0)
    tVV = 10.0 / 9.0 * V0 ** (-8.0 / 3.0)
    tVVV = -80.0 / 27.0 * V0 ** (-11.0 / 3.0)
    EVV = Ett * tV * tV + Et * tVV
    EVVV = Ettt * tV ** 3 + 3.0 * Ett * tV * tVV + Et * tVVV
    rms = float(np.sqrt(np.mean((P.polyval(t, c) - E) ** 2)))
    return dict(V0=V0, E0=float(P.polyval(t0, c)), B0=V0 * EVV, B0p=-1.0 - V0 * EVVV / EVV,
                coeffs=c, rms=rms)


def _atoms(wl):
    tau = np.array([t for _, t in wl["atoms"]], dtype=np.float64).reshape(-1, 3)
    Z = np.array([wl["species"][s]["Z"] for s, _ in wl["atoms"]], dtype=np.float64)
    sig = np.array([wl["species"][s]["sigma"] for s, _ in wl["atoms"]], dtype=np.float64)
    return tau, Z, sig


class _Cell:
    """Device state of one cell's self-consistent field (at the Gamma point,
    or at the k-points `kpoints` = (fractions of 2 pi / a, weights))."""

    def __init__(self, wl, prec, dev, kpoints=None):
        import torch
        self.wl, self.prec = wl, prec
        self.kpts = self.wk = None
        if kpoints is not None:
            kf, w = kpoints
            self.kpts = [2.0 * np.pi / float(wl["a"]) * np.asarray(k, dtype=np.float64)
                         for k in kf]
            self.wk = np.asarray(w, dtype=np.float64)
        self.ctx = pufe.pufe_build_mesh(wl)
        c = self.ctx
        c.pufe_tabulate(pufe.PUFE_FP64)
        if prec != pufe.PUFE_FP64:
            c.pufe_tabulate(prec)
        f64 = dict(dtype=torch.float64, device=dev)
        self.rho_I = torch.empty(c.n_q, **f64)
        c.pufe_ion_density(*_atoms(wl), self.rho_I)
        vol = float(wl["a"]) ** 3
        self.n = torch.full((c.n_q,), float(wl["nelec"]) / vol, **f64)
        self.V_in = torch.empty(c.n_q, **f64)
        self.V_out = torch.empty(c.n_q, **f64)
        c.pufe_effective_potential(self.n, self.rho_I, self.V_in)
        self.H = torch.empty(c.nnz, **f64)
        self.S = torch.empty(c.nnz, **f64)
        if self.kpts is not None:   # H(k), S(k) as (re, im) pairs
            mk = lambda: (torch.empty(c.nnz, **f64), torch.empty(c.nnz, **f64))
            self.Hk = [mk() for _ in self.kpts]
            self.Sk = [mk() for _ in self.kpts]
        rowptr, col = c.pattern()
        self.pattern = (rowptr, col)
        c.pufe_scf_reset()
        self.energies, self.info, self.converged = [], None, False

    def assemble(self):
        if self.kpts is None:
            self.ctx.pufe_assemble_HS(self.V_in, self.H, self.S, prec=self.prec)
            return
        for k, Hk, Sk in zip(self.kpts, self.Hk, self.Sk):
            self.ctx.pufe_assemble_HS_bloch(k, self.V_in, Hk, Sk, prec=self.prec)

    def _dense(self, re, im=None):
        rowptr, col = self.pattern
        N = self.ctx.n_dof
        v = re.cpu().numpy() if im is None else re.cpu().numpy() + 1j * im.cpu().numpy()
        return sp.csr_matrix((v, col, rowptr), shape=(N, N)).toarray()

    def step(self, nstates, kT, alpha, pulay, tol):
        import torch
        dev = self.H.device
        if self.kpts is None:
            eps, C = sla.eigh(self._dense(self.H), self._dense(self.S),
                              subset_by_index=[0, nstates - 1])
            Cd = torch.tensor(np.ascontiguousarray(C), device=dev)
            _, info = self.ctx.pufe_scf_step(eps, Cd, float(self.wl["nelec"]), kT, alpha,
                                             self.rho_I, self.V_in, self.n, self.V_out,
                                             prec=self.prec, pulay=pulay)
        else:
            eps, Cs = [], []
            for Hk, Sk in zip(self.Hk, self.Sk):
                e, C = sla.eigh(self._dense(*Hk), self._dense(*Sk),
                                subset_by_index=[0, nstates - 1])
                eps.append(e)
                Cs.append((torch.tensor(np.ascontiguousarray(C.real), device=dev),
                           torch.tensor(np.ascontiguousarray(C.imag), device=dev)))
            _, info = self.ctx.pufe_scf_step_bloch(np.array(self.kpts), self.wk, np.array(eps),
                                                   Cs, float(self.wl["nelec"]), kT, alpha,
                                                   self.rho_I, self.V_in, self.n, self.V_out,
                                                   prec=self.prec, pulay=pulay)
        self.V_in.copy_(self.V_out)
        self.info = info
        self.energies.append(info["e_total"])
        self.converged = len(self.energies) > 1 and abs(self.energies[-1] - self.energies[-2]) < tol


def scf_sweep(workloads, prec=pufe.PUFE_FP64, nstates=None, kT=0.01, alpha=0.5, pulay=4,
              tol=1e-6, max_iter=80, use_graph=True, kpoints=None):
    """Self-consistent total energies of several cells (one workload dict
    each), iterated together until every cell's total energy changes by less
    than `tol` Ha between iterations.  At the Gamma point, or with `kpoints`
    = (list of k in units of 2 pi / a per axis, weights summing to 1) at those
    Bloch wavevectors (H(k), S(k) of every k and cell in the one graph; the
    complex states of each k from a host FP64 eigensolve; pufe_scf_step_bloch).
    Returns a list of dicts (e_total, iterations, the final info of the step)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    cells = [_Cell(wl, prec, dev, kpoints) for wl in workloads]
    ns = [nstates or max(4, int(np.ceil(float(wl["nelec"]) / 2.0)) + 4) for wl in workloads]
    graph = None
    if use_graph:
        # one graph replays the assemblies of all cells (their V_in, H, S
        # buffers stay in place between iterations)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for c in cells:
                c.assemble()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for c in cells:
                c.assemble()
        torch.cuda.synchronize()
    for _ in range(max_iter):
        if graph is not None:
            graph.replay()
        else:
            for c in cells:
                c.assemble()
        torch.cuda.synchronize()
        for c, k in zip(cells, ns):
            if not c.converged:
                c.step(k, kT, alpha, pulay, tol)
        if all(c.converged for c in cells):
            break
    for c in cells:
        c.ctx.pufe_sync_status()
    return [dict(e_total=c.energies[-1], iterations=len(c.energies), converged=c.converged,
                 info=c.info, a=float(c.wl["a"])) for c in cells]
