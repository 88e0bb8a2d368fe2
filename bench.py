"""Benchmark of the PUFE hot path on one GB300 (replicas across GPUs).

One step = one pass of the whole hot path over the workload's quadrature
points: K0 tabulation, H+S assembly (K1-K3), density (K4) and the adjoint of
V -> H (K5).  The metric is quadrature-point contractions per second: the
number of quadrature points that went through the step, divided by its time.

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas of
the same workload (no collective on the data path; a barrier brackets the
timed region) and report the aggregate rate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec tf32x3|fp64]
                  [--workload c2_rocksalt_12cube] [--impl pufe|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "quadrature-point contractions/s for H/S assembly + density"
UNIT = "QPC/s"
L2_BYTES = 129 * 1024 * 1024
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
TF32_PER_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 tensor rates
# DRAM bytes (read + write) per launch of the assembly call's kernels (the
# strip, the FE-FE block and the E-E block of S) and of the strip alone, from
# the one-kernel ncu captures summarised under profiles/ (absent: not
# captured for that workload)
ASM_TRAFFIC = {("c2_rocksalt_12cube", "tf32x3"): 318.8e6}
STRIP_TRAFFIC = {("c2_rocksalt_12cube", "tf32x3"): 168.0e6}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(vals, device):
    """Each value's maximum over the ranks of the process group (the job's
    time is its slowest rank's); the values themselves on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def _job_rate(ws, units_per_rank, steps, ms):
    """Whole-job throughput: the units every rank processed over `steps`
    steps, divided by the (slowest rank's) time in milliseconds."""
    return ws * units_per_rank * steps / (ms * 1e-3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def scf_timing(ctx, wl, prec, dev, reps=10):
    """Times of the SCF calls on the same workload (Sec. 3): the effective
    potential of a density (ionic charge + FE Poisson + LDA) and one SCF step
    (occupations, output density, energies, mixing, new potential) with
    synthetic states; CUDA events on the launching stream."""
    import numpy as np
    import torch

    from paper_1611_00731_gb300 import workloads as W

    tau = np.array([t for _, t in wl["atoms"]], dtype=np.float64).reshape(-1, 3)
    Z = np.array([wl["species"][s]["Z"] for s, _ in wl["atoms"]], dtype=np.float64)
    sig = np.array([wl["species"][s]["sigma"] for s, _ in wl["atoms"]], dtype=np.float64)
    rho_I = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    ctx.pufe_ion_density(tau, Z, sig, rho_I)
    nelec = float(wl["nelec"])
    n = torch.full((ctx.n_q,), nelec / wl["a"] ** 3, dtype=torch.float64, device=dev)
    V = torch.empty_like(n)
    V2 = torch.empty_like(n)
    nst = int(wl["nocc"])
    eps = np.sort(np.random.default_rng(7).uniform(-1.0, 0.0, nst))
    Cm = torch.tensor(W.random_coefficients(ctx.n_dof, nst, seed=7), device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    t_pot = timed(lambda: ctx.pufe_effective_potential(n, rho_I, V))
    n0 = n.clone()

    def one_step():
        n.copy_(n0)
        ctx.pufe_scf_step(eps, Cm, nelec, 0.01, 0.5, rho_I, V, n, V2, prec=prec)

    t_step = timed(one_step)
    ctx.pufe_sync_status()
    return {"effective_potential_ms": t_pot, "scf_step_ms": t_step, "states": nst,
            "note": "ionic charge + FE Poisson (fast diagonalization) + PZ81; the step adds "
                    "occupations, output density, energies, mixing and the new potential"}


def bloch_timing(ctx, wl, V, dev, reps=3, prec=None):
    """Time of the Bloch assembly H(k), S(k) (real and imaginary parts) at
    k = (1/4, 1/4, 1/4) 2 pi / a on the same workload (FP64 unless `prec`)."""
    import math

    import torch

    from paper_1611_00731_gb300 import pufe

    prec = pufe.PUFE_FP64 if prec is None else prec
    ctx.pufe_tabulate(prec)
    k = [0.25 * 2.0 * math.pi / wl["a"]] * 3
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    H, S = (mk(), mk()), (mk(), mk())
    ctx.pufe_assemble_HS_bloch(k, V, H, S, prec=prec)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.pufe_assemble_HS_bloch(k, V, H, S, prec=prec)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ctx.pufe_sync_status()
    return statistics.median(ts)


def fp64_step_timing(ctx, V, Cm, f, H, S, rho, vbar, flush, stream, reps=3):
    """The same step (tabulation, H/S assembly, density, adjoint) on the plain
    FP64 GPU path, L2 flushed before each timed step, median of `reps`."""
    import torch

    from paper_1611_00731_gb300 import pufe

    fp = pufe.PUFE_FP64

    def step():
        ctx.pufe_tabulate(fp)
        ctx.pufe_assemble_HS(V, H, S, prec=fp)
        ctx.pufe_density(Cm, f, rho, prec=fp)
        ctx.pufe_assemble_HV_adjoint(H, vbar, prec=fp)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ctx.pufe_sync_status()
    return statistics.median(ts)


def c3_timing(dev, flush, stream, reps=5):
    """The uneven CsCl-like 16^3 cell (element classes from 64 to 184 basis
    functions and 64 to 4,096 points, h-adaptive rules): the same step in
    both precisions, L2 flushed before each timed step, and the assembly call
    alone with the mixed path's per-kernel times."""
    import numpy as np
    import torch

    from paper_1611_00731_gb300 import pufe, workloads as W

    wl = W.workload("c3_cscl_16cube")
    ctx = pufe.pufe_build_mesh(wl)
    n_e, _ = ctx.element_basis()
    _, _, qoff = ctx.quadrature()
    Qe = np.diff(qoff)
    flops = float(5.0 * (Qe * n_e * (n_e + 1.0)).sum())
    nocc = int(wl["nocc"])
    V = torch.tensor(W.random_potential(ctx.n_q, seed=3), device=dev)
    Cm = torch.tensor(W.random_coefficients(ctx.n_dof, nocc, seed=3), device=dev)
    f = torch.tensor(W.random_occupations(nocc, seed=3), device=dev)
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    vbar = torch.empty_like(rho)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = {"workload": "c3_cscl_16cube", "n_q": ctx.n_q, "n_dof": ctx.n_dof,
           "elements_above_128": int((n_e > 128).sum()), "flops_per_assembly": flops}
    for name, prec in (("tf32x3", pufe.PUFE_TF32X3), ("fp64", pufe.PUFE_FP64)):
        ctx.pufe_tabulate(prec)

        def step():
            ctx.pufe_tabulate(prec)
            ctx.pufe_assemble_HS(V, H, S, prec=prec)
            ctx.pufe_density(Cm, f, rho, prec=prec)
            ctx.pufe_assemble_HV_adjoint(H, vbar, prec=prec)

        out[f"{name}_step_ms"] = timed(step)
        out[f"{name}_assemble_ms"] = timed(lambda: ctx.pufe_assemble_HS(V, H, S, prec=prec))
        if name == "tf32x3":
            ctx.pufe_profile_assembly(True)
            ctx.pufe_assemble_HS(V, H, S, prec=prec)
            out["tf32x3_kernel_ms"] = ctx.pufe_profile_read()
            ctx.pufe_profile_assembly(False)
    ctx.pufe_sync_status()
    out["fp64_over_tf32x3_step"] = out["fp64_step_ms"] / out["tf32x3_step_ms"]
    return out


def c5_timing(dev, flush, stream, reps=3):
    """The equation-of-state configuration's hot path at its full size: the
    2x2x2 supercell of the rocksalt cube (64 atoms, 16^3 elements per cube,
    32^3 in all) at the four k-points of the 1/4-shifted 2x2x2 grid reduced
    by time reversal: per k-point the mixed-precision H(k), S(k) and the
    density of 64 complex states, L2 flushed before each timed 4-k step; one
    FP64 k-point beside it.  (The self-consistent sweep at this size needs an
    iterative complex eigensolver, which the library does not provide.)"""
    import numpy as np
    import torch

    from paper_1611_00731_gb300 import eos, pufe, workloads as W

    name = "c5_rocksalt_2x2x2_16cube"
    wl = W.workload(name)
    t0 = time.time()
    ctx = pufe.pufe_build_mesh(wl)
    build_s = time.time() - t0
    nocc = int(wl["nocc"])
    a = float(wl["a"])
    ks = [2.0 * np.pi / a * np.asarray(k) for k in eos.MP2_SHIFTED[0]]
    wk = eos.MP2_SHIFTED[1]
    V = torch.tensor(W.random_potential(ctx.n_q, seed=5), device=dev)
    rng = np.random.default_rng(5)
    Cr = torch.tensor(rng.standard_normal((ctx.n_dof, nocc)), device=dev)
    Ci = torch.tensor(rng.standard_normal((ctx.n_dof, nocc)), device=dev)
    f = torch.tensor(W.random_occupations(nocc, seed=5), device=dev)
    mk = lambda: torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    H, S = (mk(), mk()), (mk(), mk())
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    nk = torch.empty_like(rho)

    def timed(fn, n=reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def kstep(prec, kl):
        for i, k in enumerate(kl):
            ctx.pufe_assemble_HS_bloch(k, V, H, S, prec=prec)
            ctx.pufe_density_bloch(k, Cr, Ci, f, rho if i == 0 else nk, prec=prec)
            if i:
                rho.add_(nk, alpha=wk[i] / wk[0])

    ctx.pufe_tabulate(pufe.PUFE_TF32X3)
    ms = timed(lambda: kstep(pufe.PUFE_TF32X3, ks))
    asm = timed(lambda: ctx.pufe_assemble_HS_bloch(ks[0], V, H, S, prec=pufe.PUFE_TF32X3))
    den = timed(lambda: ctx.pufe_density_bloch(ks[0], Cr, Ci, f, rho, prec=pufe.PUFE_TF32X3))
    ctx.pufe_tabulate(pufe.PUFE_FP64)
    ms64 = timed(lambda: kstep(pufe.PUFE_FP64, ks[:1]), n=1)
    ctx.pufe_sync_status()
    return {"workload": name, "atoms": len(wl["atoms"]), "n_elem": ctx.n_elem, "n_q": ctx.n_q,
            "n_dof": ctx.n_dof, "nnz": ctx.nnz, "states": nocc, "kpoints": len(ks),
            "build_s": round(build_s, 2), "tf32x3_4k_step_ms": ms,
            "value": len(ks) * ctx.n_q / (ms * 1e-3), "unit": "QPC/s",
            "tf32x3_assemble_bloch_ms": asm, "tf32x3_density_bloch_ms": den,
            "fp64_1k_step_ms": ms64, "fp64_over_tf32x3_per_k": ms64 / (ms / len(ks)),
            "note": "per k-point: mixed H(k), S(k) (FP32 element blocks, FP64 accumulation) "
                    "and the density of 64 complex states; random V and C"}


def projection_timing(ctx, wl, dev, reps=3):
    """Time of the projections onto s + p Gaussian projectors (r_p = 0.8) on
    every atom of the workload (FP64, Gamma point)."""
    import torch

    from paper_1611_00731_gb300 import pufe

    ctx.pufe_tabulate(pufe.PUFE_FP64)
    ps = []
    for _, tau in wl["atoms"]:
        ps.append(dict(tau=tau, l=0, m=0, rp=0.8))
        ps += [dict(tau=tau, l=1, m=m, rp=0.8) for m in (-1, 0, 1)]
    F = torch.empty(ctx.n_dof, len(ps), dtype=torch.float64, device=dev)
    ctx.pufe_nonlocal_projections(ps, F)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.pufe_nonlocal_projections(ps, F)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    # the same projectors at k = (1/4, 1/4, 1/4) 2 pi / a (complex F)
    k = [0.5 * math.pi / wl["a"]] * 3
    Fi = torch.empty_like(F)
    ctx.pufe_nonlocal_projections_bloch(k, ps, (F, Fi))
    torch.cuda.synchronize()
    tk = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.pufe_nonlocal_projections_bloch(k, ps, (F, Fi))
        b.record()
        b.synchronize()
        tk.append(a.elapsed_time(b))
    ctx.pufe_sync_status()
    return {"projections_ms": statistics.median(ts), "projections_bloch_ms": statistics.median(tk),
            "projectors": len(ps), "prec": "fp64", "k_bloch": "(1/4, 1/4, 1/4) 2 pi / a"}


def run_pufe(args):
    import numpy as np
    import torch

    from paper_1611_00731_gb300 import pufe, workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = {"fp64": pufe.PUFE_FP64, "tf32x3": pufe.PUFE_TF32X3}[args.prec]

    wl = W.workload(args.workload)
    t0 = time.time()
    ctx = pufe.pufe_build_mesh(wl)
    build_s = time.time() - t0
    n_e, _ = ctx.element_basis()
    _, _, qoff = ctx.quadrature()
    Qe = np.diff(qoff)
    nocc = int(wl["nocc"])
    flops_asm = float(5.0 * (Qe * n_e * (n_e + 1.0)).sum())
    # the strip's share of the direct count: every pair with an enrichment
    # column, on the elements the CUDA-core strip takes (64 < n_e <= 128)
    strip = (n_e > 64) & (n_e <= 128)
    flops_strip = float(5.0 * (Qe[strip] * (n_e[strip] * (n_e[strip] + 1.0) - 64 * 65)).sum())
    # algorithmic bytes of the recompute form: per point the
    # weight, V and 4 values per enrichment slot in FP32, plus H and S once
    slots = ctx.element_slots()
    rowptr, col = ctx.pattern()
    bytes_in = float((Qe * (2.0 + 4.0 * slots)).sum() * 4.0)
    bytes_out = 2.0 * ctx.nnz * 8.0
    n_fe = (3 * int(wl["nel"])) ** 3
    row = np.repeat(np.arange(ctx.n_dof), np.diff(rowptr))
    nnz_e = int(((row >= n_fe) | (col >= n_fe)).sum())
    bytes_strip = float((Qe[strip] * (2.0 + 4.0 * slots[strip])).sum() * 4.0) + 2.0 * nnz_e * 8.0

    V_h = torch.tensor(W.random_potential(ctx.n_q, seed=rank), dtype=torch.float64).pin_memory()
    C_h = torch.tensor(W.random_coefficients(ctx.n_dof, nocc, seed=rank)).pin_memory()
    f_h = torch.tensor(W.random_occupations(nocc, seed=rank)).pin_memory()
    V = V_h.to(dev)
    Cm = C_h.to(dev)
    f = f_h.to(dev)
    H = torch.empty(ctx.nnz, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    rho = torch.empty(ctx.n_q, dtype=torch.float64, device=dev)
    vbar = torch.empty_like(rho)
    rho_h = torch.empty(ctx.n_q, dtype=torch.float64).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    ev_a = torch.cuda.Event(enable_timing=True)
    ev_b = torch.cuda.Event(enable_timing=True)

    side = torch.cuda.Stream() if args.density_stream == "side" else None

    def step():
        ctx.pufe_tabulate(prec)
        if side is not None:
            # the density needs only the table and C: run it on a second
            # stream, concurrently with the assembly, and join before the end
            cur = torch.cuda.current_stream()
            side.wait_stream(cur)
            ctx.pufe_density(Cm, f, rho, prec=prec, stream=side)
            ctx.pufe_assemble_HS(V, H, S, prec=prec)
            cur.wait_stream(side)
        else:
            ctx.pufe_assemble_HS(V, H, S, prec=prec)
            ctx.pufe_density(Cm, f, rho, prec=prec)
        ctx.pufe_assemble_HV_adjoint(H, vbar, prec=prec)

    tune = None
    if prec == pufe.PUFE_TF32X3 and args.autotune:
        # pick the strip's E x E form per element class by timing, once per
        # geometry, before the warm-up (cached in PUFE_AUTOTUNE_CACHE if set)
        ctx.pufe_tabulate(prec)
        t_tune = time.time()
        tune = {"classes": ctx.pufe_autotune(), "s": round(time.time() - t_tune, 3)}
    for _ in range(args.warmup):
        step()
    ctx.pufe_sync_status()
    graph = None
    if args.launch == "graph":
        # the whole step captured once into a CUDA graph and replayed: same
        # kernels, same arguments, no per-launch host overhead
        graph = torch.cuda.CUDAGraph()
        warm = torch.cuda.Stream()
        warm.wait_stream(stream)
        with torch.cuda.stream(warm):
            step()
        stream.wait_stream(warm)
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        ctx.pufe_sync_status()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # device-resident timing: each step bracketed by events, L2 flushed between
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    step_ms, asm_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if graph is not None:
            graph.replay()
        else:
            step()
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    # the assembly call on its own (stream launches), for the roofline
    for _ in range(max(3, min(args.steps, 10))):
        flush.fill_(1.0)
        ka = torch.cuda.Event(enable_timing=True)
        kb = torch.cuda.Event(enable_timing=True)
        ka.record(stream)
        ctx.pufe_assemble_HS(V, H, S, prec=prec)
        kb.record(stream)
        kb.synchronize()
        asm_ms.append(ka.elapsed_time(kb))
    # per-kernel times of the mixed assembly (events around each kernel, on
    # the stream it runs on; separate calls, so the step timing above is not
    # instrumented)
    kern_ms = []
    if args.prec == "tf32x3":
        ctx.pufe_profile_assembly(True)
        for _ in range(max(3, min(args.steps, 10))):
            flush.fill_(1.0)
            ctx.pufe_assemble_HS(V, H, S, prec=prec)
            kern_ms.append(ctx.pufe_profile_read())
        ctx.pufe_profile_assembly(False)
    barrier()
    clocks = sampler.stop()
    ctx.pufe_sync_status()
    total_ms = sum(step_ms)

    # end to end through the C ABI with host buffers: H2D of V and C, the
    # step, D2H of the density
    barrier()
    ev_a.record(stream)
    for _ in range(args.steps):
        V.copy_(V_h, non_blocking=True)
        Cm.copy_(C_h, non_blocking=True)
        f.copy_(f_h, non_blocking=True)
        step()
        rho_h.copy_(rho, non_blocking=True)
    ev_b.record(stream)
    ev_b.synchronize()
    e2e_ms = ev_a.elapsed_time(ev_b)
    ctx.pufe_sync_status()
    barrier()

    scf = scf_timing(ctx, wl, prec, dev) if args.scf else None
    bloch = None
    if args.scf:
        bloch = {"assemble_HS_ms": bloch_timing(ctx, wl, V, dev), "prec": "fp64",
                 "k": "(1/4, 1/4, 1/4) 2 pi / a"}
        if args.prec == "tf32x3" and int((n_e > 128).sum()) == 0:
            bloch["assemble_HS_tf32x3_ms"] = bloch_timing(ctx, wl, V, dev, prec=prec)
            ctx.pufe_tabulate(prec)
    nonlocal_ = projection_timing(ctx, wl, dev) if args.scf else None
    fp64_ms = (fp64_step_timing(ctx, V, Cm, f, H, S, rho, vbar, flush, stream)
               if args.scf and args.prec != "fp64" else None)
    c3 = (c3_timing(dev, flush, stream)
          if args.scf and args.workload == "c2_rocksalt_12cube" else None)
    c5 = (c5_timing(dev, flush, stream)
          if args.scf and args.workload == "c2_rocksalt_12cube" else None)

    if ws > 1:
        total_ms, e2e_ms = _max_over_ranks([total_ms, e2e_ms], dev)
    if rank != 0:
        return None

    ms_per_step = total_ms / args.steps
    value = _job_rate(ws, ctx.n_q, args.steps, total_ms)
    peaks, src = _peaks()
    asm_avg = statistics.mean(asm_ms)
    achieved = flops_asm / (asm_avg * 1e-3) / 1e12
    n_big = int((n_e > 128).sum())
    hbm = peaks["hbm_gbs"] * 1e9
    if args.prec == "fp64":
        # FP64 contraction: the recipe's nominal FP64 rate scaled like the
        # measured bf16 figure (measured bf16 x nominal FP64/bf16 ratio)
        peak = peaks["bf16_tflops"] * (1.25 / 2250.0)
        bound, dtype = "alu", "f64"
        peak_source = f"{src} bf16 x nominal FP64/bf16 ratio"
        kernels = "k_assemble_fp64"
        launches_per_step = 4
        prec_label = "fp64"
    else:
        # the binding roof of the recompute form: the tensor
        # pipe at three TF32 products per product, or the algorithmic bytes
        # at the measured HBM rate, whichever is lower
        tf32x3 = peaks["bf16_tflops"] * TF32_PER_BF16 / 3.0
        ai = flops_asm / (bytes_in + bytes_out)
        peak = min(tf32x3, ai * hbm / 1e12)
        bound = "tensor" if tf32x3 <= ai * hbm / 1e12 else "hbm"
        dtype = "f32+f64"
        peak_source = (f"min(TF32x3 = {src} bf16 burst x nominal TF32/bf16 / 3 = {tf32x3:.1f}, "
                       f"AI x {src} HBM = {ai * hbm / 1e12:.1f}) TFLOP/s")
        if n_big == 0:
            kernels = "memset H + S0 copy + k_fefe_sumfac + k_see + k_strip_sf"
            # tabulate, FE-FE block, E-E block of S, strip, density,
            # adjoint_fefe, adjoint_strip
            launches_per_step = 7
            prec_label = ("fp32 (CUDA-core strip and FE-FE V block) + error-free fp32 "
                          "(E-E block of S, fp64-class sums)")
        else:
            kernels = ("memset H + S0 copy + k_fefe_sumfac + k_see + k_pack_v + "
                       "k_assemble_tc + k_strip_sf")
            launches_per_step = 10
            prec_label = ("tf32x3 tensor-core tile (n_e > 128) + fp32 CUDA-core strip + "
                          "error-free fp32 (E-E block of S, fp64-class sums)")
    roof = {"kernel": f"pufe_assemble_HS ({kernels})", "bound": bound, "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": ASM_TRAFFIC.get((args.workload, args.prec)),
            "peak_source": peak_source,
            "flops_per_launch": flops_asm, "flops_count": "sum_e 5 Q_e n_e (n_e + 1)",
            "algorithmic_bytes_per_launch": bytes_in + bytes_out,
            "bytes_count": "sum_e Q_e (2 + 4 A_e) 4 B in + 2 nnz 8 B out",
            "avg_launch_ms": asm_avg}
    if args.prec != "fp64":
        roof["fp32_cuda_core_frac"] = achieved / FP32_PEAK_TFLOPS
        roof["fp32_cuda_core_peak"] = FP32_PEAK_TFLOPS
    if kern_ms:
        km = {k: statistics.mean(d[k] for d in kern_ms) for k in kern_ms[0]}
        t_strip = km["strip"]
        if t_strip > 0:
            a_strip = flops_strip / (t_strip * 1e-3) / 1e12
            ai_s = flops_strip / bytes_strip
            peak_s = min(peaks["bf16_tflops"] * TF32_PER_BF16 / 3.0, ai_s * hbm / 1e12)
            roof["dominant_kernel"] = {
                "kernel": "k_strip_sf", "avg_launch_ms": t_strip, "achieved": a_strip,
                "peak": peak_s, "frac": a_strip / peak_s, "unit": "TFLOP/s",
                "fp32_cuda_core_frac": a_strip / FP32_PEAK_TFLOPS,
                "flops_per_launch": flops_strip,
                "flops_count": "sum over strip elements of 5 Q_e (n_e (n_e + 1) - 64 * 65)",
                "algorithmic_bytes_per_launch": bytes_strip,
                "traffic": STRIP_TRAFFIC.get((args.workload, args.prec))}
        roof["kernel_ms"] = km
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": args.workload, "n_dof": ctx.n_dof, "n_q": ctx.n_q,
                   "n_elem": ctx.n_elem, "nnz": ctx.nnz, "nocc": nocc, "prec": prec_label,
                   "l2": "flushed between steps (2x L2 buffer written)",
                   "launch": "cuda graph of the step" if graph is not None else "stream",
                   "density_stream": args.density_stream,
                   "autotune": tune,
                   "parallelism": f"replicas x{ws}", "build_s": round(build_s, 3)},
        "roofline": roof,
        "e2e": {"value": _job_rate(ws, ctx.n_q, args.steps, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": int(V_h.numel() * 8 + C_h.numel() * 8 + f_h.numel() * 8),
                "d2h_bytes_per_step": int(rho_h.numel() * 8)},
        "gpu_launches": launches_per_step * args.steps,
        "scf": scf,
        "bloch": bloch,
        "nonlocal": nonlocal_,
        "c3": c3,
        "c5": c5,
        "fp64_path": (None if fp64_ms is None else {
            "ms_per_step": fp64_ms, "speedup_of_this_path": fp64_ms / ms_per_step,
            "note": "same step on the plain FP64 kernels (direct element contraction, the "
                    "1e-12 reference path); the ratio includes the mixed path's sum "
                    "factorization as well as its precision. At equal eigenvalue "
                    "accuracy: on this cell the mixed path's 8 lowest eigenvalues are "
                    "within 6.5e-8 Ha of the FP64 oracle (tests/test_gpu_c2_full.py), "
                    "inside the 1e-5 Ha target"}),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_elems)
    return line


# --------------------------------------------------------------------------
# the oracle as the CPU baseline / reference arm
# --------------------------------------------------------------------------
_ORACLE_SCRIPT = r"""
import json, multiprocessing as mp, sys, time
import numpy as np


def setup(root, workload, elems):
    sys.path.insert(0, root)
    from paper_1611_00731_gb300 import workloads as W
    from oracle import mesh as omesh, quadrature as oq
    wl = W.workload(workload)
    m = omesh.Mesh(wl)
    rules = {e: oq.element_rule(m, e) for e in elems}
    C = W.random_coefficients(m.n_dof, wl["nocc"])
    f = W.random_occupations(wl["nocc"])
    return m, rules, C, f


def one_pass(m, elems, rules, C, f):
    from paper_1611_00731_gb300 import workloads as W
    from oracle import assemble as oasm
    nq = 0
    for e in elems:
        p, w = rules[e]
        V = W.random_potential(len(w), seed=e)
        He, Se = oasm.element_HS(m, e, p, w, V)             # tabulation + basis + H/S
        B, _ = oasm.element_basis(m, e, p)
        Y = B @ C[m.elem_dofs(e)]
        rho = (Y * Y) @ f                                    # density
        vbar = w * np.einsum("qi,ij,qj->q", B, He, B)        # adjoint
        nq += len(w)
    return nq


def worker(root, workload, elems, reps, barrier, queue):
    m, rules, C, f = setup(root, workload, elems)
    out = []
    for _ in range(reps):
        barrier.wait()                                       # every worker starts together
        t0 = time.perf_counter()
        nq = one_pass(m, elems, rules, C, f)
        out.append((nq, time.perf_counter() - t0))
    queue.put(out)


if __name__ == "__main__":
    root, workload = sys.argv[1], sys.argv[2]
    nel, reps, nproc = int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[5])
    sys.path.insert(0, root)
    from paper_1611_00731_gb300 import workloads as W
    from oracle import mesh as omesh
    nelem = omesh.Mesh(W.workload(workload)).nelem
    rng = np.random.default_rng(0)
    elems = [int(e) for e in rng.choice(nelem, size=min(nel * nproc, nelem), replace=False)]
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(nproc), ctx.Queue()
    parts = [elems[i::nproc] for i in range(nproc)]
    procs = [ctx.Process(target=worker, args=(root, workload, parts[i], reps, barrier, queue))
             for i in range(nproc)]
    for p in procs:
        p.start()
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    # per repetition: points of all workers over the slowest worker's time
    print(json.dumps([(sum(r[k][0] for r in res), max(r[k][1] for r in res))
                      for k in range(reps)]))
"""


def _oracle_steps(workload, nelem, steps, nproc=1):
    """Runs the oracle's element loop (element H/S, density, adjoint) on
    `nelem` random elements per process in `nproc` processes (one thread
    each), `steps` repetitions; returns (points, seconds) per repetition."""
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.NamedTemporaryFile("w", suffix=".py", delete=False) as fh:
        fh.write(_ORACLE_SCRIPT)
        script = fh.name
    try:
        r = subprocess.run([sys.executable, script, ROOT, workload, str(nelem), str(steps),
                            str(nproc)], capture_output=True, text=True, env=env)
    finally:
        os.unlink(script)
    if r.returncode != 0:
        raise RuntimeError(r.stderr.strip()[-400:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(workload, nelem, reps=5):
    """The oracle on the host cores, as it stands: one thread, and one
    single-threaded process per core; best of `reps` repetitions each."""
    cores = os.cpu_count() or 1
    out = {"unit": UNIT, "kind": "oracle", "host_cpu_count": cores}
    try:
        one = max(nq / sec for nq, sec in _oracle_steps(workload, nelem, reps, 1))
        allc = max(nq / sec for nq, sec in _oracle_steps(workload, nelem, reps, cores))
    except RuntimeError as ex:
        out.update(value=None, cores=1, sample=f"failed: {ex}")
        return out
    out.update(value=allc, cores=cores, value_1_thread=one,
               sample=f"{nelem} random elements of {workload} (seed 0) per process: tabulation "
                      "and basis, element H/S, density, adjoint; best of "
                      f"{reps}; {cores} single-threaded processes ({cores * nelem} elements) "
                      f"and separately 1 thread ({nelem} elements)")
    return out


def run_reference(args):
    """The oracle as the reference arm: each step is the bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    res = _oracle_steps(args.workload, args.ref_elems, args.warmup + args.steps,
                        cores)[args.warmup:]
    nq = sum(r[0] for r in res)
    sec = sum(r[1] for r in res)
    value = nq / sec
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / len(res),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "prec": "fp64 oracle (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_elems} random elements of {args.workload} "
                                       f"(seed 0) per process and step, {cores} "
                                       "single-threaded processes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pufe", choices=["pufe", "reference"])
    ap.add_argument("--prec", default="tf32x3", choices=["tf32x3", "fp64"])
    ap.add_argument("--no-scf", dest="scf", action="store_false",
                    help="skip the timing of the SCF, Bloch and projector calls")
    ap.add_argument("--density-stream", default="side", choices=["same", "side"],
                    help="run the density on the step's stream or concurrently on a second one")
    ap.add_argument("--launch", default="stream", choices=["graph", "stream"],
                    help="replay the step as a captured CUDA graph, or launch call by call")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the strip's operation-count choice of the E x E form")
    ap.add_argument("--workload", default="c2_rocksalt_12cube")
    ap.add_argument("--cpu-elems", type=int, default=96)
    ap.add_argument("--ref-elems", type=int, default=24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "pufe" else max(args.warmup, 0)
    line = run_reference(args) if args.impl == "reference" else run_pufe(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
