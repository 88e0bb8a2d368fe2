"""Thin Python binding of the ``libpufe.so`` C ABI (see ``include/pufe.h``).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  The binding
raises if the library cannot be loaded; there is no fallback.

Functions carry the C names: ``pufe_build_mesh`` returns a :class:`Context`
whose methods ``pufe_tabulate``, ``pufe_assemble_HS``, ``pufe_density``,
``pufe_assemble_HV_adjoint`` and ``pufe_sync_status`` wrap the calls of the
same name on that context.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

PUFE_FP64, PUFE_TF32X3 = 0, 1
PUFE_WANT_H, PUFE_WANT_S = 1, 2
PUFE_FE_LAGRANGE64, PUFE_FE_SERENDIPITY32 = 0, 1
STATUS = {0: "PUFE_OK", 1: "PUFE_EINVAL", 2: "PUFE_ENOMEM", 3: "PUFE_ECUDA",
          4: "PUFE_ENOTSPD", 5: "PUFE_ENOTCONV", 6: "PUFE_ETIMEOUT",
          7: "PUFE_EDEVICE", 8: "PUFE_ESTATE"}

# every symbol that include/pufe.h declares
EXPORTS = ["pufe_build_mesh", "pufe_get_sizes", "pufe_get_quadrature", "pufe_get_pattern",
           "pufe_get_element_basis", "pufe_tabulate", "pufe_assemble_HS", "pufe_density",
           "pufe_assemble_HV_adjoint", "pufe_sync_status", "pufe_destroy", "pufe_last_error",
           "pufe_assemble_HS_static", "pufe_ion_density", "pufe_effective_potential",
           "pufe_scf_step", "pufe_scf_reset", "pufe_assemble_HS_bloch", "pufe_density_bloch",
           "pufe_assemble_HV_adjoint_bloch", "pufe_nonlocal_projections",
           "pufe_nonlocal_projections_bloch", "pufe_get_element_slots",
           "pufe_profile_assembly", "pufe_profile_read", "pufe_selftest_timeout",
           "pufe_autotune", "pufe_scf_step_bloch"]


def _projector_array(projs):
    arr = (Projector * len(projs))()
    for i, p in enumerate(projs):
        arr[i].tau = (C.c_double * 3)(*[float(t) for t in p["tau"]])
        arr[i].l, arr[i].m, arr[i].r_p = int(p["l"]), int(p["m"]), float(p["rp"])
    return arr


class PufeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Cell(C.Structure):
    _fields_ = [("a", C.c_double * 3), ("nel", C.c_int * 3), ("natoms", C.c_int),
                ("tau", C.POINTER(C.c_double)), ("species", C.POINTER(C.c_int)),
                ("lattice", C.POINTER(C.c_double)), ("fe_space", C.c_int)]


class _Species(C.Structure):
    _fields_ = [("norb", C.c_int), ("n", C.POINTER(C.c_int)), ("l", C.POINTER(C.c_int)),
                ("m", C.POINTER(C.c_int)), ("zeta", C.POINTER(C.c_double)),
                ("r_c", C.c_double), ("r_e", C.c_double)]


class _Quad(C.Structure):
    _fields_ = [("mode", C.c_int), ("p_far", C.c_int), ("p_near", C.c_int),
                ("p_min", C.c_int), ("p_max", C.c_int), ("tol", C.c_double),
                ("max_depth", C.c_int), ("device_tests", C.c_int)]


class Projector(C.Structure):
    """pufe_projector: Gaussian projector centre, (l, m) and width."""
    _fields_ = [("tau", C.c_double * 3), ("l", C.c_int), ("m", C.c_int), ("r_p", C.c_double)]


class ScfInfo(C.Structure):
    """pufe_scf_info: energies (hartree) and residual of one SCF step."""
    _fields_ = [(k, C.c_double) for k in ("mu", "e_band", "e_dc", "e_es", "e_self", "e_xc",
                                          "e_ts", "e_total", "residual")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def library_path():
    from .build import LIBPATH
    return LIBPATH


def load_library(build_if_missing: bool = True):
    """Load libpufe.so (building it in-tree with nvcc if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path) and build_if_missing:
        from .build import build_library
        build_library()
    if not os.path.exists(path):
        raise ImportError(f"libpufe.so not found at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i64p, i32p, dp = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double)
    lib.pufe_build_mesh.argtypes = [C.POINTER(_Cell), C.POINTER(_Species), C.c_int,
                                    C.POINTER(_Quad), C.POINTER(vp)]
    lib.pufe_get_sizes.argtypes = [vp, i64p, i64p, i64p, i64p, i64p]
    lib.pufe_get_quadrature.argtypes = [vp, dp, dp, i64p]
    lib.pufe_get_pattern.argtypes = [vp, i64p, i32p]
    lib.pufe_get_element_basis.argtypes = [vp, i32p, i32p]
    lib.pufe_tabulate.argtypes = [vp, C.c_int, vp]
    lib.pufe_assemble_HS.argtypes = [vp, vp, C.c_int, C.c_int, vp, vp, vp]
    lib.pufe_assemble_HS_static.argtypes = [vp, vp, C.c_int, vp, vp, vp]
    lib.pufe_density.argtypes = [vp, vp, C.c_int64, vp, C.c_int, C.c_int, vp, vp]
    lib.pufe_assemble_HV_adjoint.argtypes = [vp, vp, C.c_int, vp, vp]
    lib.pufe_sync_status.argtypes = [vp, vp]
    lib.pufe_ion_density.argtypes = [vp, C.c_int, dp, dp, dp, vp, vp]
    lib.pufe_effective_potential.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.pufe_scf_step.argtypes = [vp, C.c_int, dp, vp, C.c_int64, C.c_double, C.c_double,
                                  C.c_double, C.c_int, C.c_int, vp, vp, vp, vp, dp,
                                  C.POINTER(ScfInfo), vp]
    lib.pufe_scf_step_bloch.argtypes = [vp, C.c_int, dp, dp, C.c_int, dp, C.POINTER(vp),
                                        C.POINTER(vp), C.c_int64, C.c_double, C.c_double,
                                        C.c_double, C.c_int, C.c_int, vp, vp, vp, vp, dp,
                                        C.POINTER(ScfInfo), vp]
    lib.pufe_scf_reset.argtypes = [vp]
    lib.pufe_nonlocal_projections.argtypes = [vp, C.c_int, C.POINTER(Projector), vp, vp]
    lib.pufe_nonlocal_projections_bloch.argtypes = [vp, dp, C.c_int, C.POINTER(Projector), vp,
                                                    vp, vp]
    lib.pufe_assemble_HS_bloch.argtypes = [vp, dp, vp, C.c_int, C.c_int, vp, vp, vp, vp, vp]
    lib.pufe_density_bloch.argtypes = [vp, dp, vp, vp, C.c_int64, vp, C.c_int, C.c_int, vp, vp]
    lib.pufe_assemble_HV_adjoint_bloch.argtypes = [vp, dp, vp, vp, C.c_int, vp, vp]
    lib.pufe_get_element_slots.argtypes = [vp, i32p]
    lib.pufe_profile_assembly.argtypes = [vp, C.c_int]
    lib.pufe_profile_read.argtypes = [vp, dp]
    lib.pufe_selftest_timeout.argtypes = [vp, C.c_uint64, vp]
    lib.pufe_autotune.argtypes = [vp, C.POINTER(C.c_int), vp]
    lib.pufe_destroy.argtypes = [vp]
    lib.pufe_destroy.restype = None
    lib.pufe_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("pufe_destroy", "pufe_last_error"):
            getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


def _check(st):
    if st != 0:
        raise PufeError(st, _LIB.pufe_last_error().decode())


def _ptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """Owns a pufe_ctx; methods wrap the C calls on it."""

    def __init__(self, handle, wl):
        self._h = handle
        self.wl = wl
        n, nnz, nq, ne, mb = (C.c_int64() for _ in range(5))
        _check(_LIB.pufe_get_sizes(self._h, C.byref(n), C.byref(nnz), C.byref(nq),
                                   C.byref(ne), C.byref(mb)))
        self.n_dof, self.nnz, self.n_q = n.value, nnz.value, nq.value
        self.n_elem, self.max_basis = ne.value, mb.value

    # -- getters ---------------------------------------------------------------
    def quadrature(self):
        x = np.empty((self.n_q, 3))
        w = np.empty(self.n_q)
        off = np.empty(self.n_elem + 1, dtype=np.int64)
        _check(_LIB.pufe_get_quadrature(self._h, x.ctypes.data_as(C.POINTER(C.c_double)),
                                        w.ctypes.data_as(C.POINTER(C.c_double)),
                                        off.ctypes.data_as(C.POINTER(C.c_int64))))
        return x, w, off

    def pattern(self):
        rowptr = np.empty(self.n_dof + 1, dtype=np.int64)
        col = np.empty(self.nnz, dtype=np.int32)
        _check(_LIB.pufe_get_pattern(self._h, rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                                     col.ctypes.data_as(C.POINTER(C.c_int32))))
        return rowptr, col

    def element_basis(self):
        n_e = np.empty(self.n_elem, dtype=np.int32)
        _check(_LIB.pufe_get_element_basis(self._h, n_e.ctypes.data_as(C.POINTER(C.c_int32)), None))
        dofs = np.empty(int(n_e.sum()), dtype=np.int32)
        _check(_LIB.pufe_get_element_basis(self._h, None, dofs.ctypes.data_as(C.POINTER(C.c_int32))))
        return n_e, dofs

    def element_slots(self):
        """Enrichment functions (slots) in each element's basis."""
        a = np.empty(self.n_elem, dtype=np.int32)
        _check(_LIB.pufe_get_element_slots(self._h, a.ctypes.data_as(C.POINTER(C.c_int32))))
        return a

    def pufe_autotune(self, stream=None):
        """Pick the strip's E x E form per element class by timing (see the
        header); returns the number of classes set."""
        n = C.c_int(0)
        _check(_LIB.pufe_autotune(self._h, C.byref(n), _stream(stream)))
        return n.value

    # -- diagnostics and instrumentation -------------------------------------
    def pufe_selftest_timeout(self, wait_ns=100_000_000, stream=None):
        _check(_LIB.pufe_selftest_timeout(self._h, int(wait_ns), _stream(stream)))

    def pufe_profile_assembly(self, enable=True):
        _check(_LIB.pufe_profile_assembly(self._h, int(bool(enable))))

    def pufe_profile_read(self):
        """ms of the last instrumented mixed assembly: call, FE-FE kernels,
        E-E kernel of S, tensor-core tile, strip (0 for kernels that did not run)."""
        ms = np.zeros(5, dtype=np.float64)
        _check(_LIB.pufe_profile_read(self._h, ms.ctypes.data_as(C.POINTER(C.c_double))))
        return dict(zip(("call", "fefe", "see", "tc", "strip"), ms.tolist()))

    # -- compute calls --------------------------------------------------------
    def pufe_tabulate(self, prec=PUFE_FP64, stream=None):
        _check(_LIB.pufe_tabulate(self._h, int(prec), _stream(stream)))

    def pufe_assemble_HS(self, V, H=None, S=None, prec=PUFE_FP64, what=None, stream=None):
        import torch
        if what is None:
            what = (PUFE_WANT_H if H is not None else 0) | (PUFE_WANT_S if S is not None else 0)
        _check(_LIB.pufe_assemble_HS(self._h, _ptr(V, torch.float64), int(prec), int(what),
                                     _ptr(H, torch.float64), _ptr(S, torch.float64),
                                     _stream(stream)))

    def pufe_assemble_HS_static(self, V, H=None, S=None, what=None, stream=None):
        """TF32X3 assembly whose V scratch is a library-owned static array (no allocation)."""
        import torch
        if what is None:
            what = (PUFE_WANT_H if H is not None else 0) | (PUFE_WANT_S if S is not None else 0)
        _check(_LIB.pufe_assemble_HS_static(self._h, _ptr(V, torch.float64), int(what),
                                            _ptr(H, torch.float64), _ptr(S, torch.float64),
                                            _stream(stream)))

    def pufe_density(self, Cmat, f, rho, prec=PUFE_FP64, stream=None):
        import torch
        nocc = Cmat.shape[1]
        _check(_LIB.pufe_density(self._h, _ptr(Cmat, torch.float64), int(Cmat.stride(0)),
                                 _ptr(f, torch.float64), int(nocc), int(prec),
                                 _ptr(rho, torch.float64), _stream(stream)))

    def pufe_assemble_HV_adjoint(self, Hbar, Vbar, prec=PUFE_FP64, stream=None):
        import torch
        _check(_LIB.pufe_assemble_HV_adjoint(self._h, _ptr(Hbar, torch.float64), int(prec),
                                             _ptr(Vbar, torch.float64), _stream(stream)))

    def pufe_ion_density(self, tau, Z, sigma, rho_I, stream=None):
        """Gaussian ionic charges (host arrays) at the quadrature points."""
        import numpy as np
        import torch
        tau = np.ascontiguousarray(tau, dtype=np.float64).reshape(-1, 3)
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        dp = C.POINTER(C.c_double)
        _check(_LIB.pufe_ion_density(self._h, int(len(Z)), tau.ctypes.data_as(dp),
                                     Z.ctypes.data_as(dp), sigma.ctypes.data_as(dp),
                                     _ptr(rho_I, torch.float64), _stream(stream)))

    def pufe_effective_potential(self, n, rho_I, V_eff, V_C=None, eps_xc=None, stream=None):
        import torch
        _check(_LIB.pufe_effective_potential(self._h, _ptr(n, torch.float64),
                                             _ptr(rho_I, torch.float64), _ptr(V_eff, torch.float64),
                                             _ptr(V_C, torch.float64), _ptr(eps_xc, torch.float64),
                                             _stream(stream)))

    def pufe_scf_step(self, eps, Cmat, nelec, kT, alpha, rho_I, V_eff_in, n, V_eff_out,
                      prec=PUFE_FP64, pulay=0, stream=None):
        """One SCF step; returns (occupations, info dict).  Blocking."""
        import numpy as np
        import torch
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        f = np.zeros(len(eps))
        info = ScfInfo()
        dp = C.POINTER(C.c_double)
        _check(_LIB.pufe_scf_step(self._h, int(len(eps)), eps.ctypes.data_as(dp),
                                  _ptr(Cmat, torch.float64), int(Cmat.stride(0)), float(nelec),
                                  float(kT), float(alpha), int(pulay), int(prec),
                                  _ptr(rho_I, torch.float64),
                                  _ptr(V_eff_in, torch.float64), _ptr(n, torch.float64),
                                  _ptr(V_eff_out, torch.float64), f.ctypes.data_as(dp),
                                  C.byref(info), _stream(stream)))
        return f, info.as_dict()

    def pufe_scf_step_bloch(self, kpts, wk, eps, Cs, nelec, kT, alpha, rho_I, V_eff_in, n,
                            V_eff_out, prec=PUFE_FP64, pulay=0, stream=None):
        """One SCF step with k-points: kpts (nk, 3) Cartesian 1/bohr, wk (nk),
        eps (nk, nstates), Cs a list of nk (C_re, C_im) pairs of N x nstates
        device tensors with one stride.  Returns (occupations (nk, nstates),
        info dict).  Blocking."""
        import numpy as np
        import torch
        kp = np.ascontiguousarray(kpts, dtype=np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(wk, dtype=np.float64).reshape(-1)
        eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(len(w), -1)
        nk, ns = eps.shape
        if len(kp) != nk or len(Cs) != nk:
            raise ValueError("kpts, wk, eps and Cs must have one entry per k-point")
        ld = int(Cs[0][0].stride(0))
        for cr, ci in Cs:
            if cr.stride(0) != ld or ci.stride(0) != ld or cr.shape[1] < ns or ci.shape != cr.shape:
                raise ValueError("every C_re, C_im must be N x nstates with one row stride")
        pre = (C.c_void_p * nk)(*[_ptr(cr, torch.float64).value for cr, _ in Cs])
        pim = (C.c_void_p * nk)(*[_ptr(ci, torch.float64).value for _, ci in Cs])
        f = np.zeros((nk, ns))
        info = ScfInfo()
        dp = C.POINTER(C.c_double)
        _check(_LIB.pufe_scf_step_bloch(self._h, nk, kp.ctypes.data_as(dp), w.ctypes.data_as(dp),
                                        ns, eps.ctypes.data_as(dp), pre, pim, ld, float(nelec),
                                        float(kT), float(alpha), int(pulay), int(prec),
                                        _ptr(rho_I, torch.float64),
                                        _ptr(V_eff_in, torch.float64), _ptr(n, torch.float64),
                                        _ptr(V_eff_out, torch.float64), f.ctypes.data_as(dp),
                                        C.byref(info), _stream(stream)))
        return f, info.as_dict()

    def pufe_assemble_HS_bloch(self, k, V, H=None, S=None, what=None, stream=None,
                               prec=PUFE_FP64):
        """H(k), S(k) at wavevector k: H and S are (re, im) pairs of nnz tensors."""
        import torch
        kk = (C.c_double * 3)(*[float(x) for x in k])
        if what is None:
            what = (PUFE_WANT_H if H is not None else 0) | (PUFE_WANT_S if S is not None else 0)
        Hr, Hi = H if H is not None else (None, None)
        Sr, Si = S if S is not None else (None, None)
        f64 = torch.float64
        _check(_LIB.pufe_assemble_HS_bloch(self._h, kk, _ptr(V, f64), int(prec), int(what),
                                           _ptr(Hr, f64),
                                           _ptr(Hi, f64), _ptr(Sr, f64), _ptr(Si, f64),
                                           _stream(stream)))

    def pufe_density_bloch(self, k, Cre, Cim, f, rho, stream=None, prec=PUFE_FP64):
        import torch
        kk = (C.c_double * 3)(*[float(x) for x in k])
        if Cre.shape != Cim.shape or Cre.stride() != Cim.stride():
            raise ValueError("C_re and C_im must have the same shape and strides")
        f64 = torch.float64
        _check(_LIB.pufe_density_bloch(self._h, kk, _ptr(Cre, f64), _ptr(Cim, f64),
                                       int(Cre.stride(0)), _ptr(f, f64), int(Cre.shape[1]),
                                       int(prec), _ptr(rho, f64), _stream(stream)))

    def pufe_assemble_HV_adjoint_bloch(self, k, Hbar_re, Hbar_im, Vbar, stream=None,
                                       prec=PUFE_FP64):
        import torch
        kk = (C.c_double * 3)(*[float(x) for x in k])
        f64 = torch.float64
        _check(_LIB.pufe_assemble_HV_adjoint_bloch(self._h, kk, _ptr(Hbar_re, f64),
                                                   _ptr(Hbar_im, f64), int(prec), _ptr(Vbar, f64),
                                                   _stream(stream)))

    def pufe_nonlocal_projections(self, projs, F, stream=None):
        """F (N x P device tensor) <- projections onto projs: list of
        dict(tau, l, m, rp)."""
        import torch
        arr = _projector_array(projs)
        _check(_LIB.pufe_nonlocal_projections(self._h, len(projs), arr, _ptr(F, torch.float64),
                                              _stream(stream)))

    def pufe_nonlocal_projections_bloch(self, k, projs, F, stream=None):
        """F = (F_re, F_im) (N x P device tensors) <- projections onto the
        Bloch sums of projs at wavevector k."""
        import torch
        kk = (C.c_double * 3)(*[float(x) for x in k])
        arr = _projector_array(projs)
        f64 = torch.float64
        _check(_LIB.pufe_nonlocal_projections_bloch(self._h, kk, len(projs), arr,
                                                    _ptr(F[0], f64), _ptr(F[1], f64),
                                                    _stream(stream)))

    def pufe_scf_reset(self):
        _check(_LIB.pufe_scf_reset(self._h))

    def pufe_sync_status(self, stream=None):
        _check(_LIB.pufe_sync_status(self._h, _stream(stream)))

    def close(self):
        if self._h:
            _LIB.pufe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pufe_build_mesh(wl: dict) -> Context:
    """Build a context from a workload dict (see workloads.workload)."""
    lib = load_library()
    natoms = len(wl["atoms"])
    tau = (C.c_double * max(1, 3 * natoms))(*[c for _, t in wl["atoms"] for c in t])
    spec = (C.c_int * max(1, natoms))(*[int(s) for s, _ in wl["atoms"]])
    nel = int(wl["nel"])
    fe_space = {"lagrange64": PUFE_FE_LAGRANGE64,
                "serendipity32": PUFE_FE_SERENDIPITY32}[wl.get("fe", "lagrange64")]
    if wl.get("lattice") is not None:   # a general cell: rows a_1, a_2, a_3
        lat = (C.c_double * 9)(*[float(c) for row in wl["lattice"] for c in row])
        cell = _Cell((C.c_double * 3)(0.0, 0.0, 0.0), (C.c_int * 3)(nel, nel, nel), natoms, tau,
                     spec, lat, fe_space)
    else:
        a = float(wl["a"])
        lat = None
        cell = _Cell((C.c_double * 3)(a, a, a), (C.c_int * 3)(nel, nel, nel), natoms, tau, spec,
                     None, fe_space)
    keep = []
    sp = (_Species * max(1, len(wl["species"])))()
    for i, s in enumerate(wl["species"]):
        orbs = s["orbitals"]
        n = (C.c_int * max(1, len(orbs)))(*[o[0] for o in orbs])
        l = (C.c_int * max(1, len(orbs)))(*[o[1] for o in orbs])
        m = (C.c_int * max(1, len(orbs)))(*[o[2] for o in orbs])
        z = (C.c_double * max(1, len(orbs)))(*[o[3] for o in orbs])
        keep += [n, l, m, z]
        sp[i] = _Species(len(orbs), n, l, m, z, float(s["r_c"]), float(s["r_e"]))
    q = wl["quad"]
    quad = _Quad(int(q["mode"]), int(q["p_far"]), int(q["p_near"]), int(q["p_min"]),
                 int(q["p_max"]), float(q["tol"]), int(q["max_depth"]),
                 int(q.get("device_tests", 0)))
    h = C.c_void_p()
    _check(lib.pufe_build_mesh(C.byref(cell), sp, len(wl["species"]), C.byref(quad), C.byref(h)))
    del lat
    return Context(h, wl)


def pufe_workload(name: str) -> Context:
    return pufe_build_mesh(W.workload(name))
