"""Benchmark of the SEM pressure-Poisson hot path on GB300.

One step = one FP64 Jacobi-PCG solve to relative residual 1e-8 of the channel
workload: 32 x 32 x 32 hexahedra, N = 7 (16.8 M element-local points,
n = E N^3 = 11.2 M), tanh wall-normal stretching (beta = 2), periodic in x and
z, Dirichlet walls in y, right-hand side i.i.d. U[-1, 1] on the global nodes,
zero-mean.  Per iteration: the fused FP64 operator (p update, A_L p, <p,Ap>),
the gather-scatter and the fused vector update.  The mesh, its geometric
factors and the right-hand side are resident in HBM before the timed region;
every step solves from x0 = 0.

value  = n * CG iterations / step time   (FP64 operator applications, GDOF/s)
e2e    = the same through sem_pcg_solve_host: b copied host->device and x
         device->host inside the timed region.
roofline = the fused FP64 operator kernel (the step's dominant kernel).  On
         GB300 it is bound by the FP64 pipe, not by HBM: achieved = its
         algorithmic FP64 flops per launch / its mean duration from CUDA
         events recorded on the launching stream inside the timed solves,
         against the FP64 peak from the unit counts and the clock; its HBM
         fraction is stated beside it.
pcg    = plain FP64 time to 1e-8 against the chosen solver (the fastest
         whose FP64 true residual the oracle confirms: FP64 refinement around
         flexible FP32 CG with the hybrid Schwarz preconditioner), and the
         other solvers on the same mesh and right-hand side.

`--impl reference` times the FP64 CPU oracle on this machine's host cores on
a bounded sample of the same workload (a few CG iterations per step).
Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun every rank solves its own replica (weak scaling, no collective on
the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Ax GDOF/s (% HBM roofline); PCG time-to-1e-8 residual, plain FP64 vs chosen"
UNIT = "GDOF/s"
WORKLOAD = "channel 32x32x32 hex, N=7, tanh beta=2 in y, periodic x/z, Dirichlet y, random mean-zero RHS"


def channel_workload(nel, order):
    """The channel workload's name at the sizes a run uses (WORKLOAD at 32^3, N = 7)."""
    return WORKLOAD.replace("32x32x32", f"{nel}x{nel}x{nel}").replace("N=7", f"N={order}")
TOL = 1e-8
AX_BYTES_PER_POINT = {"f64": 64}

# DRAM traffic per launch of the operator kernels from one ncu capture
# (bytes), keyed by the SHA-256 of the kernel source it was taken on; the
# bench reports null once the source changes.
NCU_TRAFFIC = {"ax64_cg": {"bytes_per_launch": 1408.6e6, "src_sha": "21f1d46784359222",
                           "from": "profiles/ax64_cg_n7_nel20_ncu_full.md (20^3 case scaled x4.096)"}}


def _src_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--nel", type=int, default=32)
    p.add_argument("--order", type=int, default=7)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-iters", type=int, default=3, help="oracle CG iterations in the CPU sample")
    p.add_argument("--plain-steps", type=int, default=2, help="plain FP64 solves timed for comparison")
    p.add_argument("--op", choices=["ax-f64", "ax-f32", "ax-f64pair", "dssum-f64", "dssum-f32", "schwarz", "pcg-f64",
                                    "gemm"],
                   default=None, help="time one entry point alone instead of the solve")
    p.add_argument("--workload", choices=["channel", "tgv-learned", "batched", "deformed", "tgv-steps", "schwarz",
                                          "tgv-long"],
                   default="channel")
    p.add_argument("--coarse-iters", type=int, default=3, help="Schwarz: coarse-level CG iterations per application")
    p.add_argument("--mid", type=int, default=0,
                   help="Schwarz: order of the intermediate multigrid level (0: two levels)")
    p.add_argument("--mid-weight", type=float, default=0.15, help="Schwarz: weight of the intermediate level")
    p.add_argument("--krylov", choices=["cg", "fgmres"], default="cg",
                   help="schwarz: inner Krylov method (flexible CG or flexible restarted GMRES)")
    p.add_argument("--gmres-restart", type=int, default=30, help="schwarz: GMRES cycle length")
    p.add_argument("--inner-tol", type=float, default=1e-5, help="schwarz: inner relative tolerance of a round")
    p.add_argument("--outer-pair", action="store_true",
                   help="Schwarz workload: outer residual with the double-float (FP32-pair) operator")
    p.add_argument("--nsolve", type=int, default=64)
    p.add_argument("--t-end", type=float, default=10.0, help="tgv-long: final time")
    p.add_argument("--dt", type=float, default=2e-3, help="tgv-long: time step")
    p.add_argument("--sample-every", type=int, default=25, help="tgv-long: steps between energy samples")
    p.add_argument("--round-iters", type=int, default=16)
    p.add_argument("--batched-schwarz", action="store_true",
                   help="batched workload: hybrid Schwarz inner preconditioner per solve")
    p.add_argument("--train-steps", type=int, default=100)
    p.add_argument("--eval-steps", type=int, default=100)
    p.add_argument("--epochs", type=int, default=30)
    p.add_argument("--variant", choices=["p1", "d3"], default="p1")
    p.add_argument("--tol", type=float, default=1e-8, help="tgv-learned: relative tolerance of the pressure solves")
    p.add_argument("--loss", choices=["mse", "energy", "energy_avg"], default="energy_avg",
                   help="tgv-learned: training loss")
    p.add_argument("--lam", type=float, default=1.0, help="tgv-learned: mass weight of the energy-norm loss")
    p.add_argument("--methods", default="", help="tgv-learned: comma-separated subset of the methods")
    p.add_argument("--fp64-residual", action="store_true",
                   help="tgv-learned: residual feature with the FP64 operator (default: FP32-pair)")
    p.add_argument("--bf16", action="store_true",
                   help="channel variant: the FP32 inner operator reads BF16 geometric factors (32 B/point)")
    p.add_argument("--affine", action="store_true",
                   help="channel variant: the affine-element FP32 operator (3 scalars per element, 20 B/point)")
    return p.parse_args(argv)


# ------------------------------------------------------------------ distributed plumbing


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ peaks


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# ------------------------------------------------------------------ CPU oracle samples


def cpu_oracle_sample(case, iters, verts=None):
    """Time the oracle's Jacobi-PCG for `iters` CG iterations on the full
    workload (FP64, 1 thread).  The oracle forms r = b - A x0 before its
    first iteration, so the sample makes iters + 1 operator applications;
    GDOF/s counts those.  Returns (GDOF/s, seconds, description, mesh, b)."""
    import oracle
    V = case.vertices() if verts is None else verts
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    t0 = time.perf_counter()
    _, it, _, _ = om.pcg(b, tol=1e-30, max_iter=iters)
    dt = time.perf_counter() - t0
    gdofs = case.n_paper * (it + 1) / dt / 1e9
    return (gdofs, dt, f"{it} FP64 oracle CG iterations ({it + 1} operator applications incl. the initial "
                       f"residual) on the full {case.E}-element workload, 1 thread ({dt:.1f} s)", om, b)


def _cpu_ax_worker(N, verts, reps, seed, barrier, out):
    import numpy as np

    import oracle
    _, G, _, st = oracle.geometry(N, verts)
    D = oracle.deriv(N)
    u = np.random.default_rng(seed).standard_normal((verts.shape[0], (N + 1) ** 3))
    oracle.ax_local(N, D, G, u)  # warm
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.ax_local(N, D, G, u)
    out.put(((time.perf_counter() - t0) / reps, verts.shape[0]))


def cpu_oracle_allcores(case, verts, elems_per_core=512, reps=5):
    """The oracle's local operator on every host core at once: one process
    per core (spawned, so no CUDA state is inherited) applies oracle.ax_local
    to its own block of elements; throughput = the elements of all blocks /
    the slowest block's time.  Operator only (no gather-scatter, no vector
    updates).  Returns (GDOF/s, cores, description)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(cores), ctx.Queue()
    procs = []
    for c in range(cores):
        lo = (c * elems_per_core) % max(case.E - elems_per_core, 1)
        procs.append(ctx.Process(target=_cpu_ax_worker,
                                 args=(case.N, verts[lo:lo + elems_per_core], reps, c, barrier, q)))
    for pr in procs:
        pr.start()
    res = [q.get(timeout=600) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    t = max(r[0] for r in res)
    ne = sum(r[1] for r in res)
    gdofs = ne * case.N ** 3 / t / 1e9
    return gdofs, cores, (f"oracle local operator (ax_local, FP64) on {cores} processes x {elems_per_core} "
                          f"elements of the workload, {reps} applications each, slowest process {t * 1e3:.1f} ms")


# ------------------------------------------------------------------ our arm

# Algorithmic bytes per local point of the operator kernels:
#   fused FP64 CG operator: reads r, dinv, p (8 B each) and G (6 x 8 B),
#     writes p and w (8 B each) = 88 B;
#   FP64 operator: reads u (8 B) and G (6 x 8 B), writes w (8 B) = 64 B;
#   fused FP32 CG operator: reads r, dinv, p (4 B each) and G (6 x 4 B),
#     writes p and w (4 B each) = 44 B.
OP_BYTES = {"f32_cg": 44, "f64": 64, "f64_cg": 88,
            # affine-element form: r, dinv, p read, p, w written; 16 B of scalars per element
            "f32_cg_aff": 20,
            # BF16 factors: r, dinv, p read (4 B each), G (6 x 2 B), p, w written
            "f32_cg_bf16": 32}
# Algorithmic FP64 flops per local point of the even/odd operator at order N
# (FMA = 2, add or multiply = 1): per line of N+1 points the even/odd split
# (N+1 adds), two H x H coefficient blocks (H = (N+1)/2, 2 H^2 FMAs) and the
# recombination (N+1 adds), three forward and three backward directions; the
# geometric factors 3 multiplies + 6 FMAs; the three directions summed (2
# adds).  Fused CG form: p = dinv r + beta p (multiply + FMA) and <p, Ap>
# (FMA).  FP64 pipe operations count every instruction once.
def f64_op_counts(N, cg):
    n1 = N + 1
    H = n1 // 2
    line_flops = 2 * n1 + 2 * 2 * H * H + (2 * H if n1 % 2 else 0)
    line_ops = 2 * n1 + 2 * H * H + (H if n1 % 2 else 0)
    flops = 6 * line_flops / n1 + 15 + 2 + (5 if cg else 0)
    ops = 6 * line_ops / n1 + 9 + 2 + (3 if cg else 0)
    return flops, ops


# FP64 peak of GB300 from the unit counts and the clock: 152 SMs x 2 FP64
# FMA lanes per clock x 2 flops x 2.07 GHz (an FMA-chain probe measures
# 1.20 TFLOP/s, 95 % of it).
F64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
F64_PEAK_OPS = 152 * 2 * 2.07e9
MID_WEIGHT = 0.15  # weight of the intermediate Schwarz level (oracle and GPU measurements on the channel)
# theta of the adaptive inner tolerance: a refinement round stops once half
# the outer target is within reach (the FP64 residual still decides)
INNER_ADAPT = 0.5
# inner tolerance of the Schwarz solves: 1e-5 (two refinement rounds; Jacobi-PCG keeps 1e-2, its long FP32
# runs lose orthogonality)
SCHWARZ_INNER_TOL = 1e-5
CHOSEN_SCHWARZ = dict(precision=1, inner_tol=SCHWARZ_INNER_TOL, coarse_iters=3, coarse_tol=1e-2, check_every=8,
                      inner_adapt=INNER_ADAPT)
JACOBI_MIXED = dict(precision=1, inner_tol=1e-2, inner_adapt=INNER_ADAPT)  # FP64 refinement around FP32 Jacobi-PCG
GMRES_RESTART = 30  # cycle length of flexible GMRES (one cycle per refinement round)
PLAIN = dict(precision=0)


def _solve_series(gm, b, scratch, steps, opts, profile=True, stream=None):
    """`steps` solves; per-solve device times from CUDA events on `stream`."""
    import torch
    iters, ax_ms, ax_n, launches, outer_ms, outer_n = 0, 0.0, 0, 0, 0.0, 0
    stats, times = None, []
    for _ in range(steps):
        if stream is not None:
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        _, stats = gm.pcg(b, scratch=scratch, profile=profile, **opts)
        if stream is not None:
            z.record(stream)
            times.append((a, z))
        iters += stats["iters"]
        ax_ms += stats["ax_ms"]
        ax_n += stats["ax_launches"]
        launches += stats["kernel_launches"]
        outer_ms += stats["outer_ax_ms"]
        outer_n += stats["outer_ax_launches"]
    if times:
        torch.cuda.synchronize()
        times = [a.elapsed_time(z) for a, z in times]
    return dict(iters=iters, ax_ms=ax_ms, ax_n=ax_n, launches=launches, outer_ms=outer_ms, outer_n=outer_n,
                last=stats, times=times)


def median_ci(xs):
    """Median and a 95 % confidence interval of the mean (normal
    approximation, as the paper's measurement protocol) of a sample."""
    if not xs:
        return None
    m = statistics.mean(xs)
    h = 1.96 * statistics.stdev(xs) / math.sqrt(len(xs)) if len(xs) > 1 else 0.0
    return {"median": round(statistics.median(xs), 3), "mean": round(m, 3),
            "ci95": [round(m - h, 3), round(m + h, 3)], "n": len(xs)}


def perf_model_block(case, gm, scratch, ms_per_step, iters, cpu_gdofs, om):
    """The paper's performance model (section 4.1) applied to this GPU and
    its host: cost = element-iterations of one solve; P_opt(GPU) from the
    timed solves, P_opt(CPU) from the oracle's single-core rate times the
    host's cores (linear scaling: as optimistic as the model); capacities =
    device memory / bytes per element of each side."""
    import numpy as np
    import torch

    from paper_2405_05640_gb300 import binding
    E = case.E
    C = E * iters
    P_gpu = C / (ms_per_step / 1e3)
    cores = os.cpu_count() or 1
    P_cpu = cpu_gdofs * 1e9 / case.N ** 3 * cores
    _, total = torch.cuda.mem_get_info()
    # the FP64 solver's footprint: mesh workspace without the FP32 and
    # FP32-pair factor copies this benchmark adds for its other solvers
    # (24 + 48 B per point), plus the solver scratch
    gpu_bpe = (gm.info.workspace_bytes - 72 * case.nloc + scratch.numel()) / E
    cpu_bpe = sum(v.nbytes for v in vars(om).values() if isinstance(v, np.ndarray)) / E
    host = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    emax_gpu, emax_cpu = 0.95 * total / gpu_bpe, 0.8 * host / cpu_bpe
    T, split = binding.perf_model([P_gpu, P_cpu], C, [emax_gpu * iters, emax_cpu * iters])
    out = {"unit": "element-iterations/s", "P_opt_gpu": round(P_gpu, 1), "P_opt_cpu": round(P_cpu, 1),
           "host_cores": cores, "cost": C, "T_gpu_alone_ms": round(ms_per_step, 3),
           "T_min_gpu_plus_cpu_ms": round(T * 1e3, 3), "predicted_gain": round(ms_per_step / (T * 1e3) - 1.0, 5),
           "elements_gpu_cpu": [round(split[0] / iters, 1), round(split[1] / iters, 1)],
           "capacity_elements_gpu_cpu": [int(emax_gpu), int(emax_cpu)],
           "bytes_per_element_gpu_cpu": [int(gpu_bpe), int(cpu_bpe)]}
    # the capacity-bound regime: a problem larger than the GPU holds (half as
    # much again, within what GPU + host hold together), same iterations
    Eb = emax_gpu + 0.5 * min(emax_gpu, emax_cpu)
    if Eb <= emax_gpu + emax_cpu:
        Tb, sb = binding.perf_model([P_gpu, P_cpu], Eb * iters, [emax_gpu * iters, emax_cpu * iters])
        Tc = Eb * iters / P_cpu if Eb <= emax_cpu else float("inf")
        out["capacity_case"] = {"elements": int(Eb), "T_min_ms": round(Tb * 1e3, 1),
                                "cpu_alone_ms": round(Tc * 1e3, 1) if Tc != float("inf") else None,
                                "elements_gpu_cpu": [round(sb[0] / iters, 1), round(sb[1] / iters, 1)],
                                "gpu_alone": "does not fit"}
    return out


def _timed_solves(gm, b, scratch, opts, steps, stream):
    """One untimed solve, then `steps` timed ones (CUDA events around the
    series on `stream`); returns (ms per solve, series)."""
    import torch
    gm.pcg(b, scratch=scratch, **opts)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    ser = _solve_series(gm, b, scratch, steps, opts)
    p1.record(stream)
    torch.cuda.synchronize()
    return p0.elapsed_time(p1) / steps, ser


def run_ours(args):
    import torch

    from paper_2405_05640_gb300 import binding, inputs
    from paper_2405_05640_gb300 import build as _build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist_init("nccl")
    _build.build()
    case = inputs.channel(args.nel, args.order)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_pair=True,
                      geom_affine=args.affine, geom_bf16=args.bf16)
    bg = torch.from_numpy(case.rhs_global()).cuda()
    b = gm.scatter(bg)
    base = dict(tol=TOL, max_iter=50000, check_every=32)
    plain = dict(base, **PLAIN)
    mixed = dict(base, **JACOBI_MIXED)
    scratch = gm.pcg_scratch(gm.pcg_opts(**mixed))  # the larger of the two
    stream = torch.cuda.current_stream()

    # ---- the headline: K plain FP64 Jacobi-PCG solves
    for _ in range(args.warmup):
        gm.pcg(b, scratch=scratch, **plain)
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ser = _solve_series(gm, b, scratch, args.steps, plain, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    barrier()
    t_max = max_over_ranks(elapsed_ms / 1e3, device="cuda")
    tot_iters = sum_over_ranks(float(ser["iters"]), device="cuda")
    value = case.n_paper * tot_iters / t_max / 1e9
    ms_per_step = t_max * 1e3 / args.steps
    it_per_solve = ser["iters"] / args.steps
    step_stats = median_ci(ser["times"])
    value_stats = {k: (round(case.n_paper * it_per_solve / (v * 1e-3) / 1e9, 4) if k in ("median", "mean") else
                       [round(case.n_paper * it_per_solve / (x * 1e-3) / 1e9, 4) for x in v[::-1]] if k == "ci95"
                       else v) for k, v in step_stats.items()}

    # ---- the other solvers on the same mesh and right-hand side
    ps = args.plain_steps
    mixed_ms, mser = _timed_solves(gm, b, scratch, mixed, ps, stream)
    pair_ms, qser = _timed_solves(gm, b, scratch, dict(base, precision=2), ps, stream)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    t_sw = time.perf_counter()
    sw = binding.Schwarz(gm, gc)
    sw_setup_s = time.perf_counter() - t_sw
    sw_opts = dict(base, **CHOSEN_SCHWARZ, schwarz=sw)
    sw_scratch = gm.pcg_scratch(gm.pcg_opts(**sw_opts))
    sw_ms, wser = _timed_solves(gm, b, sw_scratch, sw_opts, ps, stream)
    swp_ms, vser = _timed_solves(gm, b, sw_scratch, dict(sw_opts, outer_pair=True), ps, stream)
    # the three-level Schwarz multigrid: an intermediate order-3 level
    gmid = binding.Mesh(3, case.nel, case.periodic, case.faces, V, geom_f32=True)
    swmid = binding.Schwarz(gmid, gc)
    sw3_opts = dict(sw_opts, schwarz_mid=swmid, mid_weight=MID_WEIGHT)
    sw3_scratch = gm.pcg_scratch(gm.pcg_opts(**sw3_opts))
    sw3_ms, tser = _timed_solves(gm, b, sw3_scratch, sw3_opts, ps, stream)
    sw3p_ms, user_ = _timed_solves(gm, b, sw3_scratch, dict(sw3_opts, outer_pair=True), ps, stream)
    # the paper's Krylov method: flexible restarted GMRES with the same preconditioners
    # (inner tolerance 1e-2: a cycle is capped at GMRES_RESTART iterations, and longer
    # cycles cost more Gram-Schmidt than the rounds they save)
    gm_opts = dict(krylov=binding.SEM_KRYLOV_FGMRES, gmres_restart=GMRES_RESTART, inner_tol=1e-2)
    gm2_scratch = gm.pcg_scratch(gm.pcg_opts(**dict(sw_opts, **gm_opts)))
    gm2_ms, g2ser = _timed_solves(gm, b, gm2_scratch, dict(sw_opts, **gm_opts), ps, stream)
    del gm2_scratch
    gm3_scratch = gm.pcg_scratch(gm.pcg_opts(**dict(sw3_opts, **gm_opts)))
    gm3_ms, g3ser = _timed_solves(gm, b, gm3_scratch, dict(sw3_opts, **gm_opts), ps, stream)
    del gm3_scratch

    # ---- end to end through the host-buffer entry point (the headline solve)
    e2e = None
    if not args.no_e2e:
        hb = torch.empty(case.nloc, dtype=torch.float64, pin_memory=True)
        hb.copy_(b.cpu())
        hx = torch.empty(case.nloc, dtype=torch.float64, pin_memory=True)
        hscr = gm.pcg_host_scratch(gm.pcg_opts(**plain))
        gm.pcg_host(hb, hx, scratch=hscr, **plain)
        torch.cuda.synchronize()
        barrier()
        nsteps = min(args.steps, 3)
        te_list, e_iters = [], 0
        for _ in range(nsteps):
            t0 = time.perf_counter()
            _, s2 = gm.pcg_host(hb, hx, scratch=hscr, **plain)
            torch.cuda.synchronize()
            te_list.append(time.perf_counter() - t0)
            e_iters += s2["iters"]
        te = max_over_ranks(sum(te_list), device="cuda")
        e_iters = sum_over_ranks(float(e_iters), device="cuda")
        e2e = {"value": round(case.n_paper * e_iters / te / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": int(hb.numel() * 8), "d2h_bytes_per_step": int(hx.numel() * 8),
               "ms_per_step": round(te * 1e3 / nsteps, 3), "steps": nsteps,
               "ms_per_step_stats": median_ci([t * 1e3 for t in te_list])}

    peaks = measured_peaks()
    hbm = peaks["hbm_gbs"]
    # ---- roofline of the dominant kernel: the fused FP64 operator
    f64_ms = ser["ax_ms"] / max(ser["ax_n"], 1)
    flops_pt, ops_pt = f64_op_counts(case.N, cg=True)
    f64_flops = flops_pt * case.nloc
    f64_bytes = OP_BYTES["f64_cg"] * case.nloc
    achieved = f64_flops / (f64_ms * 1e-3) / 1e12
    sha = _src_sha(os.path.join(ROOT, "paper_2405_05640_gb300", "csrc", "sem_ax64.cu"))
    tr = NCU_TRAFFIC.get("ax64_cg")
    traffic = tr["bytes_per_launch"] if tr and tr.get("src_sha") == sha else None
    roofline = {"kernel": f"ax64_kernel<{case.N},CG> (fused FP64 operator: p update, A_L p, <p,Ap>; "
                          "even/odd contractions)",
                "bound": "alu", "achieved": round(achieved, 4), "peak": round(F64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(achieved / F64_PEAK_TFLOPS, 4), "traffic": traffic,
                "peak_source": "FP64 peak from unit counts and clock (152 SMs x 2 FMA/clk x 2.07 GHz); "
                               "an FMA-chain probe reaches 1.20 TFLOP/s",
                "algorithmic_flops_per_launch": int(f64_flops), "flops_per_point": flops_pt,
                "fp64_pipe_ops_per_point": ops_pt,
                "fp64_pipe_frac": round(ops_pt * case.nloc / (f64_ms * 1e-3) / F64_PEAK_OPS, 4),
                "mean_launch_ms": round(f64_ms, 4),
                "algorithmic_bytes_per_launch": int(f64_bytes),
                "hbm_achieved_gbs": round(f64_bytes / (f64_ms * 1e-3) / 1e9, 1), "hbm_peak_gbs": hbm,
                "hbm_frac": round(f64_bytes / (f64_ms * 1e-3) / 1e9 / hbm, 4),
                "attainable": "min(HBM, FP64 pipe): FP64 pipe (the HBM bound would allow "
                              f"{round(f64_bytes / (hbm * 1e9) * 1e3, 4)} ms)"}
    # ---- secondary kernels: the plain FP64 operator, the double-float operator,
    # the fused FP32 operator of the mixed solvers
    u = torch.randn(case.nloc, dtype=torch.float64, device="cuda")
    w = torch.empty_like(u)

    def _op_ms(pair, reps=20):
        for _ in range(3):
            gm.ax(u, w, pair=pair)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        q0.record(stream)
        for _ in range(reps):
            gm.ax(u, w, pair=pair)
        q1.record(stream)
        torch.cuda.synchronize()
        return q0.elapsed_time(q1) / reps

    pair_op_ms, plain64_ms = _op_ms(True), _op_ms(False)
    fl_plain, op_plain = f64_op_counts(case.N, cg=False)
    roofline_f64_plain = {"kernel": f"ax64_kernel<{case.N}> (FP64 operator, sem_ax)", "bound": "alu",
                          "mean_launch_ms": round(plain64_ms, 4),
                          "achieved_tflops": round(fl_plain * case.nloc / (plain64_ms * 1e-3) / 1e12, 4),
                          "frac": round(fl_plain * case.nloc / (plain64_ms * 1e-3) / 1e12 / F64_PEAK_TFLOPS, 4),
                          "fp64_pipe_frac": round(op_plain * case.nloc / (plain64_ms * 1e-3) / F64_PEAK_OPS, 4),
                          "hbm_frac": round(64 * case.nloc / (plain64_ms * 1e-3) / 1e9 / hbm, 4),
                          "gdofs": round(case.n_paper / (plain64_ms * 1e-3) / 1e9, 3)}
    pair_bytes = OP_BYTES["f64"] * case.nloc
    roofline_pair = {"kernel": f"ax_pair_kernel<{case.N}> (FP64 in/out, double-float arithmetic on the FP32 pipes, "
                               "~48 significant bits)", "bound": "issue (fp32 alu)",
                     "mean_launch_ms": round(pair_op_ms, 4),
                     "achieved_gbs": round(pair_bytes / (pair_op_ms * 1e-3) / 1e9, 1),
                     "hbm_frac": round(pair_bytes / (pair_op_ms * 1e-3) / 1e9 / hbm, 4),
                     "gdofs": round(case.n_paper / (pair_op_ms * 1e-3) / 1e9, 3),
                     "speedup_vs_fp64_operator": round(plain64_ms / pair_op_ms, 3)}
    f32_ms = mser["ax_ms"] / max(mser["ax_n"], 1)
    f32_bytes = ((OP_BYTES["f32_cg_aff"] * case.nloc + 16 * case.E) if args.affine else
                 OP_BYTES["f32_cg_bf16"] * case.nloc if args.bf16 else OP_BYTES["f32_cg"] * case.nloc)
    tr32 = NCU_TRAFFIC.get("ax_f32_cg")
    sha32 = _src_sha(os.path.join(ROOT, "paper_2405_05640_gb300", "csrc", "sem_ax.cu"))
    roofline_f32 = {"kernel": "ax_kernel<7,float,CG> (fused FP32 operator of the mixed solvers' inner loop)",
                    "bound": "hbm", "mean_launch_ms": round(f32_ms, 4),
                    "achieved": round(f32_bytes / (f32_ms * 1e-3) / 1e9, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(f32_bytes / (f32_ms * 1e-3) / 1e9 / hbm, 4),
                    "traffic": tr32["bytes_per_launch"] if tr32 and tr32.get("src_sha") == sha32 and
                    not (args.affine or args.bf16) else None,
                    "algorithmic_bytes_per_launch": int(f32_bytes),
                    "gdofs": round(case.n_paper / (f32_ms * 1e-3) / 1e9, 3)}

    def _sol(ms, sr, steps):
        st = sr["last"]
        return {"time_to_1e-8_ms": round(ms, 3), "iters": sr["iters"] / steps,
                "outer_iters": st["outer_iters"] if st else None,
                "rel_res_fp64": st["rel_res"] if st else None, "status": st["status"] if st else None,
                "speedup_vs_plain_fp64": round(ms_per_step / ms, 3)}

    two, three = _sol(sw_ms, wser, ps), _sol(sw3_ms, tser, ps)
    chosen3 = three["time_to_1e-8_ms"] < two["time_to_1e-8_ms"]
    chosen = three if chosen3 else two
    rec = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": channel_workload(args.nel, args.order), "E": case.E, "N": case.N,
                   "n_paper": case.n_paper,
                   "nloc": case.nloc, "nglob": gm.nglob, "tol": TOL,
                   "precision": "FP64 Jacobi-PCG (FP64 operator, gather-scatter, vectors and dot products)",
                   "geometry": "general: 6 geometric factors per point (FP64)",
                   "l2": "inputs larger than L2 (FP64 G 805 MB, fields 134 MB each)",
                   "parallelism": f"replicas x{world}"},
        "value_stats": value_stats, "ms_per_step_stats": step_stats,
        "pcg": {"plain_fp64_time_to_1e-8_ms": round(ms_per_step, 3), "plain_fp64_iters": it_per_solve,
                "plain_fp64_rel_res": ser["last"]["rel_res"], "plain_fp64_status": ser["last"]["status"],
                "chosen": "FP64 refinement around flexible FP32 CG with the hybrid Schwarz multigrid "
                          + ("(three levels: N = 7, 3, trilinear coarse)" if chosen3 else "(two levels)")
                          + ", FP64 outer residual",
                "chosen_time_to_1e-8_ms": chosen["time_to_1e-8_ms"],
                "chosen_speedup_vs_plain_fp64": chosen["speedup_vs_plain_fp64"],
                "solvers": {"schwarz_mixed": two,
                            "schwarz_mixed_pair_outer": _sol(swp_ms, vser, ps),
                            "schwarz3_mixed": three,
                            "schwarz3_mixed_pair_outer": _sol(sw3p_ms, user_, ps),
                            "schwarz_fgmres": _sol(gm2_ms, g2ser, ps),
                            "schwarz3_fgmres": _sol(gm3_ms, g3ser, ps),
                            "jacobi_mixed": _sol(mixed_ms, mser, ps),
                            "fp64_vectors_double_float_operator": _sol(pair_ms, qser, ps)},
                "schwarz_setup_s": round(sw_setup_s, 3), "schwarz_subdomain_problems": sw.problems,
                "schwarz_launches_per_solve": wser["launches"] / ps},
        "ax_kernel_gdofs": round(case.n_paper / (f64_ms * 1e-3) / 1e9, 3),
        "roofline": roofline,
        "roofline_fp64_plain_operator": roofline_f64_plain,
        "roofline_fp32_operator": roofline_f32,
        "roofline_double_float_operator": roofline_pair,
        "gpu_launches": ser["launches"],
        "e2e": e2e,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        g, dt, desc, om, _ = cpu_oracle_sample(case, args.cpu_iters, V)
        rec["cpu_baseline"] = {"value": round(g, 5), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        try:
            ga, cores, desca = cpu_oracle_allcores(case, V)
            rec["cpu_baseline_all_cores"] = {"value": round(ga, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                                             "sample": desca}
        except Exception as exc:  # a host without spawn support or memory: report, do not fail the bench
            rec["cpu_baseline_all_cores"] = {"unavailable": f"{type(exc).__name__}: {exc}"}
        rec["perf_model"] = perf_model_block(case, gm, scratch, ms_per_step, it_per_solve, g, om)
    if rank == 0:
        print(json.dumps(rec), flush=True)


# ------------------------------------------------------------------ reference arm


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2405_05640_gb300 import inputs
    case = inputs.channel(args.nel, args.order)
    import oracle
    V = case.vertices()
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    per_step = args.cpu_iters  # CG iterations per timed step (bounded sample of one solve)
    for _ in range(args.warmup):
        om.pcg(b, tol=1e-30, max_iter=per_step)
    times, apps = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, it, _, _ = om.pcg(b, tol=1e-30, max_iter=per_step)
        times.append(time.perf_counter() - t0)
        apps += it + 1
    dt = sum(times)
    value = case.n_paper * apps / dt / 1e9
    desc = (f"{per_step} FP64 oracle CG iterations per step ({per_step + 1} operator applications incl. the "
            f"initial residual) on the full {case.E}-element workload, 1 thread")
    rec = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": channel_workload(args.nel, args.order), "E": case.E,
                                           "N": case.N,
                                           "n_paper": case.n_paper, "tol": TOL, "precision": "FP64 oracle"},
           "ms_per_step_stats": median_ci([t * 1e3 for t in times]),
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(rec), flush=True)


def run_op(args):
    """Time one entry point alone: K launches of sem_ax / sem_dssum on the
    channel mesh, CUDA events on the launching stream (inputs > L2)."""
    import torch

    from paper_2405_05640_gb300 import binding, inputs
    from paper_2405_05640_gb300 import build as _build
    _build.build()
    if args.op == "gemm":
        return run_op_gemm(args)
    case = inputs.channel(args.nel, args.order)
    if args.op == "schwarz":
        return run_op_schwarz(args, case)
    if args.op == "pcg-f64":
        return run_op_pcg_f64(args, case)
    kind, dt = args.op.split("-")
    pair = dt == "f64pair"
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices(), geom_f32=not pair,
                      geom_pair=pair)
    tdt = torch.float32 if dt == "f32" else torch.float64
    u = torch.randn(case.nloc, dtype=tdt, device="cuda")
    w = torch.empty_like(u)
    if kind == "ax":
        # algorithmic bytes per local point: u in, w out, six factors (FP64 or FP32-pair: 8 B each)
        fn, nbytes = (lambda: gm.ax(u, w, pair=pair)), (32 if dt == "f32" else 64) * case.nloc
    else:
        fn = lambda: gm.dssum(w, mask=True)
        nbytes = 2 * gm.info.n_shared_points * (8 if dt == "f64" else 4)
    for _ in range(args.warmup):
        fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    peak = measured_peaks()["hbm_gbs"]
    print(json.dumps({"op": args.op, "nel": args.nel, "N": case.N, "ms_per_launch": round(ms, 4),
                      "gdofs": round(case.n_paper / (ms * 1e-3) / 1e9, 3), "algorithmic_bytes": nbytes,
                      "achieved_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                      "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4)}), flush=True)


def run_op_gemm(args):
    """The tcgen05 BF16 GEMM (sem_gemm_bf16: C = act(A B^T + bias), FP32
    accumulation in TMEM) on the guess network's shapes at the 32^3 TGV mesh
    (32768 element rows; 2048-256-256-512 layers): the three forward layers
    and the five backward products, plus one 8192^3 product for the peak;
    TFLOP/s = 2 M N K / mean launch time (CUDA events, `steps` launches after
    `warmup`), against the measured cuBLAS BF16 burst peak."""
    import torch

    from paper_2405_05640_gb300 import binding
    from paper_2405_05640_gb300 import build as _build
    _build.build()
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peak = float(json.load(f)["bf16_tflops"])
    src = "measured bf16_tflops (burst)" if peak else "fallback"
    peak = peak or 1900.0
    R, I, H, O = 32768, 2048, 256, 512
    shapes = [("fwd W1", R, H, I, 1), ("fwd W2", R, H, H, 1), ("fwd W3", R, O, H, 0),
              ("bwd dW3", O, H, R, 0), ("bwd dH2", R, H, O, 0), ("bwd dW2", H, H, R, 0),
              ("bwd dH1", R, H, H, 0), ("bwd dW1", H, I, R, 0), ("square 8192", 8192, 8192, 8192, 0)]
    s = torch.cuda.current_stream()
    g = torch.Generator(device="cuda").manual_seed(0)
    rows = []
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for name, M, N, K, act in shapes:
        A = torch.randn((M, K), generator=g, device="cuda").to(torch.bfloat16)
        B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16)
        bias = torch.zeros(N, dtype=torch.float32, device="cuda")
        # the weight gradients (small outputs, K = the rows) with split-K, as the network runs them
        work = binding.gemm_splitk_work(M, N, K) if name.startswith("bwd dW") else None
        for _ in range(args.warmup):
            binding.gemm_bf16(A, B, bias, act, err=err, work=work)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(args.steps):
            binding.gemm_bf16(A, B, bias, act, err=err, work=work)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        rows.append({"gemm": name, "M": M, "N": N, "K": K, "ms": round(ms, 4), "tflops": round(tf, 1),
                     "frac": round(tf / peak, 4), "split_k": work is not None})
    assert int(err.item()) == 0, "a bounded wait of the GEMM gave up"
    fwd = [r for r in rows if r["gemm"].startswith("fwd")]
    bwd = [r for r in rows if r["gemm"].startswith("bwd")]
    f_fl = sum(2.0 * r["M"] * r["N"] * r["K"] for r in fwd)
    b_fl = sum(2.0 * r["M"] * r["N"] * r["K"] for r in bwd)
    print(json.dumps({"op": "gemm", "kernel": "gemm_tn_bf16_kernel (tcgen05.mma kind::f16, TMA, TMEM accumulator)",
                      "peak_tflops": peak, "peak_source": src, "shapes": rows,
                      "forward_pass": {"ms": round(sum(r["ms"] for r in fwd), 4),
                                       "tflops": round(f_fl / (sum(r["ms"] for r in fwd) * 1e-3) / 1e12, 1)},
                      "backward_pass": {"ms": round(sum(r["ms"] for r in bwd), 4),
                                        "tflops": round(b_fl / (sum(r["ms"] for r in bwd) * 1e-3) / 1e12, 1)}}),
          flush=True)


def run_op_pcg_f64(args, case):
    """W + K plain FP64 Jacobi-PCG solves of the channel workload at --nel
    (for launch lists and kernel captures: only the solver's own kernels)."""
    import torch

    from paper_2405_05640_gb300 import binding
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices())
    b = gm.scatter(torch.from_numpy(case.rhs_global()).cuda())
    opts = dict(tol=TOL, max_iter=50000, check_every=32, precision=binding.SEM_PCG_F64)
    scratch = gm.pcg_scratch(gm.pcg_opts(**opts))
    for _ in range(args.warmup):
        gm.pcg(b, scratch=scratch, **opts)
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    ser = _solve_series(gm, b, scratch, args.steps, opts, profile=False, stream=s)
    print(json.dumps({"op": "pcg-f64", "nel": args.nel, "N": case.N, "iters": ser["iters"] / args.steps,
                      "ms_per_solve": median_ci(ser["times"]), "kernel_launches": ser["launches"]}), flush=True)


def _schwarz_setup(case, pair=False):
    from paper_2405_05640_gb300 import binding
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_pair=pair)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    return gm, binding.Schwarz(gm, gc)


def run_op_schwarz(args, case):
    """K applications of sem_schwarz_apply (local solves, coarse CG, overlap
    sums) on the channel residual in FP32; algorithmic bytes per local point:
    r read, the extended solutions written and read back ((N+3)^3/(N+1)^3 x
    4 B each), z written."""
    import torch
    gm, sw = _schwarz_setup(case)
    r = gm.scatter(torch.from_numpy(case.rhs_global()).cuda()).float()
    z = torch.empty_like(r)
    fn = lambda: sw.apply(r, coarse_iters=args.coarse_iters, coarse_tol=1e-2, z=z)
    for _ in range(args.warmup):
        fn()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ext = ((case.N + 3) / (case.N + 1)) ** 3
    nbytes = int((4 + 8 * ext + 4) * case.nloc)
    peak = measured_peaks()["hbm_gbs"]
    # the local solves' six 1-D contractions: (N+3)^4 multiply-adds each per element
    flops = 2 * 6 * (case.N + 3) ** 4 * case.E
    print(json.dumps({"op": "schwarz", "nel": args.nel, "N": case.N, "coarse_iters": args.coarse_iters,
                      "subdomain_problems": sw.problems, "ms_per_launch": round(ms, 4),
                      "algorithmic_bytes": nbytes, "achieved_gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                      "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
                      "contraction_flops": flops, "achieved_tflops": round(flops / (ms * 1e-3) / 1e12, 2),
                      "fp32_peak_tflops": 73.5, "peak_source": "measured FMA-chain probe on GB300 (FP32)",
                      "fp32_frac": round(flops / (ms * 1e-3) / 1e12 / 73.5, 4)}), flush=True)


def run_schwarz(args):
    """The channel solved to 1e-8 by FP64 refinement around flexible FP32 CG
    with the hybrid Schwarz preconditioner (K timed solves)."""
    import torch

    from paper_2405_05640_gb300 import binding, inputs
    from paper_2405_05640_gb300 import build as _build
    _build.build()
    case = inputs.channel(args.nel, args.order)
    gm, sw = _schwarz_setup(case, pair=args.outer_pair)
    b = gm.scatter(torch.from_numpy(case.rhs_global()).cuda())
    opts = dict(tol=TOL, max_iter=50000, precision=binding.SEM_PCG_MIXED, inner_tol=args.inner_tol, check_every=8,
                schwarz=sw, coarse_iters=args.coarse_iters, coarse_tol=1e-2, outer_pair=args.outer_pair,
                inner_adapt=INNER_ADAPT)
    if args.krylov == "fgmres":
        opts.update(krylov=binding.SEM_KRYLOV_FGMRES, gmres_restart=args.gmres_restart)
    if args.mid:
        V = case.vertices()
        gmid = binding.Mesh(args.mid, case.nel, case.periodic, case.faces, V, geom_f32=True)
        gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
        smid = binding.Schwarz(gmid, gc)
        opts.update(schwarz_mid=smid, mid_weight=args.mid_weight)
    scratch = gm.pcg_scratch(gm.pcg_opts(**opts))
    for _ in range(args.warmup):
        gm.pcg(b, scratch=scratch, **opts)
    stream = torch.cuda.current_stream()
    with ClockSampler(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ser = _solve_series(gm, b, scratch, args.steps, opts, profile=False)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    st = ser["last"]
    method = "flexible GMRES" if args.krylov == "fgmres" else "flexible CG"
    print(json.dumps({"metric": f"pressure solve time to 1e-8, hybrid Schwarz {method} inside FP64 refinement",
                      "value": round(ms, 3), "unit": "ms", "higher_is_better": False, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
                      "dtype": "f32 inner / f64 refinement",
                      "config": {"workload": channel_workload(args.nel, args.order),
                                 "coarse_iters": args.coarse_iters, "krylov": args.krylov,
                                 "inner_tol": args.inner_tol,
                                 "gmres_restart": args.gmres_restart if args.krylov == "fgmres" else None,
                                 "levels": 3 if args.mid else 2, "mid_order": args.mid or None,
                                 "mid_weight": args.mid_weight if args.mid else None,
                                 "outer_residual": "double-float operator" if args.outer_pair else "FP64 operator"},
                      "inner_iters": ser["iters"] / args.steps, "outer_iters": st["outer_iters"],
                      "rel_res_fp64": st["rel_res"], "status": st["status"], "gpu_launches": ser["launches"],
                      "subdomain_problems": sw.problems, "clocks": clk.summary()}), flush=True)


def run_tgv_learned(args):
    """The learned-initial-guess workload: TGV Re=1600, 32^3, N=7, dt=1e-3,
    network trained on steps 1-100, pressure solves of steps 101-200 timed
    per method: plain FP64 from p^{n-1}; FP64 refinement around FP32
    Jacobi-PCG and around flexible FP32 CG with the hybrid Schwarz
    preconditioner, each from p^{n-1}, from the cubic extrapolation and from
    the learned guess.  value = speedup of the fastest method over plain
    FP64; the learned guess's gain is reported over each solver's own
    extrapolation start."""
    from paper_2405_05640_gb300 import build as _build
    from paper_2405_05640_gb300 import tgv_learned
    _build.build()
    out = tgv_learned.run(nel=args.nel, N=args.order, train_steps=args.train_steps, eval_steps=args.eval_steps,
                          schwarz_inner_tol=SCHWARZ_INNER_TOL,
                          epochs=args.epochs, variant=args.variant, inner_adapt=INNER_ADAPT, tol=args.tol,
                          loss=args.loss, lam=args.lam,
                          pair=not args.fp64_residual,
                          **({"methods": tuple(args.methods.split(","))} if args.methods else {}))
    m = out["methods"]
    best = min((k for k in m if k != "plain_f64_prev"), key=lambda k: m[k]["pressure_ms_total"])
    gain = {}
    for solver in ("chosen", "schwarz", "schwarz3", "schwarz_fixed"):
        base, fx = solver.split("_")[0], "_fixed" if solver.endswith("_fixed") else ""
        a, b = m.get(f"{base}_learned{fx}"), m.get(f"{base}_extrap{fx}")
        if a and b:
            gain[solver] = {"iters_learned": a["iters_mean"], "iters_extrap": b["iters_mean"],
                            "iter_gain": round(1.0 - a["iters_mean"] / b["iters_mean"], 4),
                            "time_gain": round(1.0 - a["pressure_ms_total"] / b["pressure_ms_total"], 4)}
    rec = {"metric": f"pressure-solve wall time to {args.tol:g} over the evaluated TGV steps, fastest method vs plain "
                     "FP64 (x0 = previous pressure)",
           "value": m[best].get("speedup_vs_plain_f64_prev"), "unit": "x (speedup)", "best_method": best,
           "higher_is_better": True, "n_gpus": 1, "dtype": "bf16 network / f32 inner / f64 refinement",
           "data": "synthetic", "config": {"workload": out["workload"]}, "inner_adapt": INNER_ADAPT,
           "learned_gain": gain, **out}
    print(json.dumps(rec), flush=True)


def run_batched(args):
    """Batched serving: independent deformed-box Poisson solves of uneven
    size (E ~ U{8^3..40^3}, N ~ U{5, 7, 9}, seed 0), solved together by
    sem_pcg_solve_batched (one CUDA graph per round) after the operator
    launch shape has been autotuned per order.  Reports aggregate GDOF/s and
    the p50 / p99 per-solve completion latency."""
    import torch

    from paper_2405_05640_gb300 import binding, inputs
    from paper_2405_05640_gb300 import build as _build
    _build.build()
    cases = inputs.batched_cases(args.nsolve, seed=0)
    # device memory per local point: mesh (G64 48, G32 24, B/mult/minv/dinv 32,
    # dinv32/minv32 8, groups ~3) + batched scratch (FP64 r, w 16 + FP32 x4 16)
    # (+ Schwarz: extended local solutions ~8 B, tables and coarse level ~17 B)
    bpp = 147 + (25 if args.batched_schwarz else 0)
    need = sum(c.nloc for c in cases) * bpp
    free, total = torch.cuda.mem_get_info()
    used = list(cases)
    while used and sum(c.nloc for c in used) * bpp > 0.85 * free:
        used.pop()
    meshes, bs = [], []
    for c in used:
        m = binding.Mesh(c.N, c.nel, c.periodic, c.faces, c.vertices(), geom_f32=True)
        meshes.append(m)
        bs.append(m.scatter(torch.from_numpy(c.rhs_global()).cuda()))
    tune = {}
    for N in sorted({c.N for c in used}):
        i = next(k for k, c in enumerate(used) if c.N == N)
        tune[N] = meshes[i].autotune(binding.SEM_F32, True)
    kw = dict(tol=TOL, max_iter=50000, inner_tol=SCHWARZ_INNER_TOL if args.batched_schwarz else 1e-2,
              check_every=args.round_iters, inner_adapt=INNER_ADAPT)
    keep = []
    if args.batched_schwarz:
        sws = []
        for c, m in zip(used, meshes):
            gc = binding.Mesh(1, c.nel, c.periodic, c.faces, c.vertices(), geom_f32=True)
            keep.append(gc)
            sws.append(binding.Schwarz(m, gc))
        kw.update(schwarz=sws, coarse_iters=3, coarse_tol=1e-2)
    xs, _ = binding.pcg_solve_batched(meshes, bs, **kw)  # warm-up (graph capture, instantiation)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        xs, stats = binding.pcg_solve_batched(meshes, bs, xs=xs, **kw)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    lat = sorted(s["wall_ms"] for s in stats)
    gdof = sum(c.n_paper * s["iters"] for c, s in zip(used, stats))
    rec = {"metric": "batched Poisson solves to 1e-8: aggregate GDOF/s, p50/p99 per-solve latency",
           "value": round(gdof / wall / 1e9, 3), "unit": "GDOF/s", "higher_is_better": True, "n_gpus": 1,
           "dtype": "f32 inner / f64 refinement", "data": "synthetic",
           "preconditioner": "hybrid Schwarz (two levels) per solve" if args.batched_schwarz else "Jacobi",
           "config": {"workload": f"{len(used)} of {len(cases)} deformed boxes (memory bound {need / 1e9:.0f} GB)",
                      "solves": len(used), "orders": {str(N): sum(1 for c in used if c.N == N) for N in tune},
                      "local_points": sum(c.nloc for c in used), "round_iters": args.round_iters},
           "wall_s": round(wall, 3), "latency_ms": {"p50": lat[len(lat) // 2],
                                                      "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                                                      "max": lat[-1]},
           "status": [s["status"] for s in stats].count(0), "iters_total": sum(s["iters"] for s in stats),
           "autotune": {str(N): {k: v for k, v in t.items() if k != "table"} for N, t in tune.items()},
           "clocks": clk.summary()}
    print(json.dumps(rec), flush=True)


def run_deformed(args):
    """Mixed precision on the deformed cube (64^3 elements, N = 7, vertices
    moved by 0.05 h, Dirichlet walls, random right-hand side): time to 1e-8
    of plain FP64 PCG, of FP64 refinement around FP32 Jacobi-PCG and around
    flexible FP32 CG with the hybrid Schwarz preconditioner (its local solves
    use the elements' mean edge lengths, approximate on deformed elements),
    and each mixed solution's error against the FP64 solution, all converged
    to 1e-11."""
    import torch

    from paper_2405_05640_gb300 import binding, inputs
    from paper_2405_05640_gb300 import build as _build
    _build.build()
    case = inputs.deformed_cube(args.nel, args.order)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_bf16=args.bf16)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    sw = binding.Schwarz(gm, gc)
    gmid = binding.Mesh(3, case.nel, case.periodic, case.faces, V, geom_f32=True)
    swmid = binding.Schwarz(gmid, gc)
    b = gm.scatter(torch.from_numpy(case.rhs_global()).cuda())
    solvers = {"plain_fp64": dict(precision=binding.SEM_PCG_F64),
               "jacobi_mixed": dict(JACOBI_MIXED),
               "schwarz_mixed": dict(CHOSEN_SCHWARZ, schwarz=sw),
               "schwarz3_mixed": dict(CHOSEN_SCHWARZ, schwarz=sw, schwarz_mid=swmid, mid_weight=MID_WEIGHT),
               "schwarz_fgmres": dict(CHOSEN_SCHWARZ, schwarz=sw, krylov=binding.SEM_KRYLOV_FGMRES,
                                      gmres_restart=GMRES_RESTART, inner_tol=1e-2)}
    scratch = gm.pcg_scratch(gm.pcg_opts(precision=binding.SEM_PCG_MIXED, schwarz=sw, schwarz_mid=swmid,
                                         krylov=binding.SEM_KRYLOV_FGMRES, gmres_restart=GMRES_RESTART))
    out = {}
    for name, kw in solvers.items():
        kw = dict(kw, tol=TOL, max_iter=100000, check_every=8 if "schwarz" in kw else 32)
        gm.pcg(b, scratch=scratch, **kw)  # warm-up
        torch.cuda.synchronize()
        times = []
        for _ in range(max(1, min(args.steps, 3))):
            t0 = time.perf_counter()
            x, st = gm.pcg(b, scratch=scratch, **kw)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
        out[name] = {"time_to_1e-8_ms": round(statistics.median(times), 1), "iters": st["iters"],
                     "outer": st["outer_iters"], "rel_res": st["rel_res"], "status": st["status"]}
    xs = {}
    for name, kw in solvers.items():
        kw = dict(kw, tol=1e-11, max_iter=100000, check_every=8 if "schwarz" in kw else 32)
        xs[name], _ = gm.pcg(b, scratch=scratch, **kw)
    ref = xs["plain_fp64"]
    mixed = [k for k in solvers if k != "plain_fp64"]
    for name in mixed:
        d = xs[name] - ref
        out[name]["rel_err_vs_fp64_at_1e-11"] = (gm.glsc3(d, d) / gm.glsc3(ref, ref)) ** 0.5
        out[name]["speedup_vs_plain_fp64"] = round(out["plain_fp64"]["time_to_1e-8_ms"] /
                                                   out[name]["time_to_1e-8_ms"], 3)
    best = max(mixed, key=lambda k: out[k]["speedup_vs_plain_fp64"])
    rec = {"metric": "PCG time-to-1e-8, plain FP64 vs the fastest mixed solver",
           "value": out[best]["speedup_vs_plain_fp64"], "best": best,
           "unit": "x (speedup)", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
           "dtype": "f32 inner / f64 refinement",
           "config": {"workload": f"deformed cube {args.nel}^3 elements, N={case.N}, amplitude 0.05 h, seed 0",
                      "nloc": case.nloc, "n_paper": case.n_paper, "schwarz_subdomain_problems": sw.problems},
           "solves": out}
    print(json.dumps(rec), flush=True)


def run_tgv_steps(args):
    """Navier-Stokes steps of the Taylor-Green vortex (Re = 1600, dt = 1e-3,
    [0, 2pi]^3, nel^3 elements, N = 7): the default scheme (BDF2/EXT2,
    collocated advection) against BDF3/EXT3 with dealiased advection
    (3/2 rule); milliseconds per step (pressure and velocity solves to 1e-8 /
    1e-10, mixed-precision pressure from the previous pressure) and the
    advection alone (CUDA events on the launching stream)."""
    import numpy as np
    import torch

    from paper_2405_05640_gb300 import binding, inputs
    from paper_2405_05640_gb300 import build as _build
    _build.build()
    case = inputs.tgv_box(args.nel, args.order)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_rx=True, geom_f32=True)
    xyz = gm.coords().cpu().numpy()
    u0 = torch.from_numpy(np.stack([c.reshape(-1) for c in inputs.tgv_velocity(*xyz)])).cuda()
    po = gm.pcg_opts(tol=1e-8, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2,
                     use_initial_guess=True, inner_adapt=INNER_ADAPT)
    vo = gm.pcg_opts(tol=1e-10, max_iter=20000)
    stream = torch.cuda.current_stream()
    out = {}
    for name, order, dealias in (("bdf2_collocation", 2, False), ("bdf3_dealiased", 3, True)):
        st = binding.NSState(gm, 1600.0)
        st.set_scheme(order, dealias=dealias)
        st.set_velocity(u0)
        for _ in range(args.warmup):
            st.step(1e-3, po, vo)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        pit = 0
        for _ in range(args.steps):
            ps, _ = st.step(1e-3, po, vo)
            pit += ps["iters"]
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / args.steps
        u = torch.stack([st.get(c) for c in range(3)])
        e0.record(stream)
        for _ in range(5):
            st.advect(u)
        e1.record(stream)
        torch.cuda.synchronize()
        adv_ms = e0.elapsed_time(e1) / 5
        out[name] = {"ms_per_step": round(step_ms, 3), "pressure_iters_per_step": pit / args.steps,
                     "advection_ms": round(adv_ms, 3), "kinetic_energy": st.kinetic_energy()}
        del st
    # FP64 work of the dealiased advection per element (N = 7, M = 12): ~0.45 M FMA
    M = (3 * (case.N + 1) + 1) // 2
    n1 = case.N + 1
    fma = (3 * (n1 * n1 * M * n1 + n1 * M * M * n1 + M ** 3 * n1) + 9 * M ** 3 +
           3 * (2 * n1 * n1 * M * n1 + 3 * n1 * M * M * n1 + 3 * M ** 3 * n1 + 3 * M ** 3 +
                n1 * M * M * M + n1 * n1 * M * M + n1 ** 3 * M))
    tf = 2 * fma * case.E / (out["bdf3_dealiased"]["advection_ms"] * 1e-3) / 1e12
    rec = {"metric": "Navier-Stokes step time, TGV Re=1600: BDF2 collocation vs BDF3 dealiased",
           "value": out["bdf3_dealiased"]["ms_per_step"], "unit": "ms/step", "higher_is_better": False,
           "n_gpus": 1, "data": "synthetic", "dtype": "f64 (pressure: f32 inner / f64 refinement)",
           "config": {"workload": f"TGV {args.nel}^3 elements, N={case.N}, dt=1e-3", "steps": args.steps,
                      "warmup": args.warmup},
           "schemes": out,
           "dealiased_advection_fp64": {"fma_per_element": fma, "achieved_tflops": round(tf, 3),
                                        "peak_tflops": 1.257, "frac": round(tf / 1.257, 3)}}
    print(json.dumps(rec), flush=True)


def run_tgv_long(args):
    """A long Taylor-Green vortex run: Re = 1600, [0, 2 pi]^3, nel^3
    elements, N = 7, BDF3 / EXT3 with dealiased (3/2-rule) advection, the
    pressure solved by FP64 refinement around flexible FP32 CG with the
    hybrid Schwarz preconditioner from the cubic extrapolation, the velocity
    by FP64 Jacobi-CG, to t_end.  Every `sample_every` steps: the kinetic
    energy E_k = <|u|^2> / 2 and the enstrophy Omega = <|w|^2> / 2 (w = curl u
    from the library's collocation gradient, integrated element by element
    with the GLL mass).  Self-consistency of the run: E_k must decrease, and
    the dissipation -dE_k/dt (central differences of the samples) must match
    2 nu Omega; both series are reported.  The reference data of the
    benchmark case are not available here."""
    import numpy as np
    import torch

    from paper_2405_05640_gb300 import binding, inputs
    from paper_2405_05640_gb300 import build as _build
    _build.build()
    Re, dt, nu = 1600.0, args.dt, 1.0 / 1600.0
    case = inputs.tgv_box(args.nel, args.order)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_rx=True, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    sw = binding.Schwarz(gm, gc)
    xyz = gm.coords().cpu().numpy()
    u0 = torch.from_numpy(np.stack([c.reshape(-1) for c in inputs.tgv_velocity(*xyz)])).cuda()
    ns = binding.NSState(gm, Re)
    ns.set_scheme(3, dealias=True)
    ns.set_velocity(u0)
    po = gm.pcg_opts(tol=1e-8, max_iter=50000, precision=binding.SEM_PCG_MIXED, inner_tol=SCHWARZ_INNER_TOL,
                     check_every=8,
                     schwarz=sw, coarse_iters=3, coarse_tol=1e-2, use_initial_guess=True, inner_adapt=INNER_ADAPT)
    vo = gm.pcg_opts(tol=1e-8, max_iter=50000, check_every=8)
    Bm = gm.field(0)
    vol = float(Bm.sum())
    zero = torch.zeros((gm.E, gm.npt), dtype=torch.float32, device="cuda")
    guess = torch.empty(gm.nloc, dtype=torch.float64, device="cuda")

    def enstrophy():
        g = [gm.gradient(ns.get(c)) for c in range(3)]  # g[c][m] = d u_c / d x_m
        wx, wy, wz = g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]
        return 0.5 * float((Bm * (wx * wx + wy * wy + wz * wz)).sum()) / vol

    nsteps = int(round(args.t_end / dt))
    t, E, Om, piters, viters = [0.0], [ns.kinetic_energy()], [enstrophy()], [], []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    t_wall = time.perf_counter()
    for n in range(1, nsteps + 1):
        ns.step_begin(dt)
        pg = None
        if n > 3:  # cubic extrapolation of the last three pressures, no correction
            binding.guess_apply(gm, zero, ns.get(3), ns.get(4), ns.get(5), 0.0, guess)
            pg = guess
        ps, vs = ns.step_finish(po, vo, p_guess=pg)
        piters.append(ps["iters"])
        viters.append(sum(v["iters"] for v in vs))
        if ps["status"] != 0 or any(v["status"] != 0 for v in vs):
            raise RuntimeError(f"step {n}: solver status {ps['status']} / {[v['status'] for v in vs]}")
        if n % args.sample_every == 0 or n == nsteps:
            t.append(n * dt)
            E.append(ns.kinetic_energy())
            Om.append(enstrophy())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    wall = time.perf_counter() - t_wall
    t, E, Om = np.array(t), np.array(E), np.array(Om)
    eps_num = -np.gradient(E, t)      # -dE_k/dt from the samples
    eps_ens = 2.0 * nu * Om           # 2 nu Omega
    inner = slice(1, len(t) - 1)
    mism = np.abs(eps_num[inner] - eps_ens[inner]) / np.maximum(eps_ens[inner], 1e-30)
    k_peak = int(np.argmax(eps_ens))
    rec = {"metric": "long TGV run: dissipation self-consistency (-dE_k/dt vs 2 nu Omega) and time per step",
           "value": round(ms / nsteps, 3), "unit": "ms/step", "higher_is_better": False, "n_gpus": 1,
           "data": "synthetic", "dtype": "f64 (pressure: f32 inner / f64 refinement)",
           "config": {"workload": f"TGV Re=1600, {args.nel}^3 elements, N={case.N}, dt={dt:g}, t_end={args.t_end:g}, "
                                  "BDF3/EXT3, 3/2-rule dealiasing, Schwarz pressure from the cubic extrapolation",
                      "steps": nsteps, "sample_every": args.sample_every},
           "wall_s": round(wall, 1),
           "pressure_iters_mean": round(float(np.mean(piters)), 2),
           "velocity_iters_mean": round(float(np.mean(viters)) / 3, 2),
           "energy_monotone": bool(np.all(np.diff(E) < 0)),
           "E_k0": E[0], "E_k_end": E[-1],
           "dissipation_peak": {"t": float(t[k_peak]), "2nu_Omega": float(eps_ens[k_peak]),
                                "minus_dEdt": float(eps_num[k_peak])},
           "identity_rel_mismatch": {"median": float(np.median(mism)), "max": float(np.max(mism)),
                                     "at_peak": float(abs(eps_num[k_peak] - eps_ens[k_peak]) / eps_ens[k_peak])},
           "series": {"t": [round(float(x), 4) for x in t], "E_k": [float(x) for x in E],
                      "2nu_Omega": [float(x) for x in eps_ens], "minus_dEdt": [float(x) for x in eps_num]}}
    print(json.dumps(rec), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.workload == "deformed":
        run_deformed(args)
    elif args.workload == "tgv-learned":
        run_tgv_learned(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "tgv-steps":
        run_tgv_steps(args)
    elif args.workload == "schwarz":
        run_schwarz(args)
    elif args.workload == "tgv-long":
        run_tgv_long(args)
    elif args.op:
        run_op(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
