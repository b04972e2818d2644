"""Benchmark of the Leja exponential-integrator hot path on one GB300 per rank.

Workload (default): 2D linear advection-diffusion u_t = nu (u_xx + u_yy) +
a (u_x + u_y) on the periodic unit square, 4096 x 4096, nu = 1e-2, a = 1,
second-order central differences, FP64, seeded sum-of-three-Gaussians initial
state, exponential Rosenbrock-Euler steps with h = 50 dt_CFL, tolerance 1e-10,
spectral bound from 10 power-iteration passes (once, before the timed steps).
A bench "step" is one Rosenbrock-Euler step: h f(u), one phi_1 Leja loop of
fused iterations, and u + p.

Metric: GDOF * Leja-iterations per second = sum over steps of
nx*ny*iters / time / 1e9, the whole job over all ranks.  Multi-GPU runs are
independent replicas (the path has no exchange step), so scaling is weak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference   # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "GDOF*Leja-iter/s"
UNIT = "GDOF*iter/s"
NX = NY = 4096
NU, ADV = 1e-2, 1.0
CFL_MULT = 50.0
TOL = 1e-10
ALG_BYTES = {"fp64": 32, "mixed": 24, "df64": 32}  # algorithmic bytes per point per fused Leja iteration
FP64_OPS_PER_POINT_ITER = 8  # FP64 FMA-class instructions per point per Leja iteration (native FP64 kernel)
FP64_FMA_PEAK_G = 625.0  # GB300 nominal FP64 1.25 TFLOP/s = 625 G fused multiply-adds per second


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="lexgb", choices=["lexgb", "reference"])
    p.add_argument("--precision", default="df64", choices=["fp64", "mixed", "df64"])
    p.add_argument("--n", type=int, default=NX)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-plain", action="store_true", help="skip the plain-form (native FP64) comparison")
    p.add_argument("--tol", type=float, default=TOL, help="default workload: Leja tolerance (rtol = atol)")
    p.add_argument("--kernel", default=None, help="force a fused-iteration kernel (name) instead of autotuning "
                   "(burgers2048: for its float-float forms)")
    p.add_argument("--forms", default=None,
                   help="burgers2048: comma-separated subset of fp64,mixed,df64,epirk4s3a_fp64,epirk4s3a_df64")
    p.add_argument("--strip-h", type=int, default=8)
    p.add_argument("--unroll", type=int, default=None, help="fused-iteration launches per graph-loop pass")
    p.add_argument("--source", action="store_true",
                   help="diffusion-advection with a time-independent source S (u' = A u + S)")
    p.add_argument("--workload", default="advdiff4096",
                   choices=["advdiff4096", "batch256", "burgers2048", "vertical4096", "paper1", "paper2",
                            "paper3", "rhs4096", "learned2048"])
    p.add_argument("--cfl", type=float, default=100.0, help="paper workloads: step size in units of dt_CFL")
    p.add_argument("--tf", type=float, default=None,
                   help="paper workloads: integrate to this final time and report the end-to-end time")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(dist, t_local, units_local, device="cuda"):
    """Whole-job numbers of independent replicas: the slowest rank's time and
    the units all ranks processed (one all-reduce each, not on the data path)."""
    if dist is None:
        return t_local, units_local
    import torch

    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for rel in ("paper_2310_08344_gb300/csrc/leja_kernels.cuh", "paper_2310_08344_gb300/csrc/leja_df64.cuh",
                "paper_2310_08344_gb300/csrc/leja_df64_2step.cuh", "paper_2310_08344_gb300/csrc/leja_df64_2step_x.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name: str, n_points: int):
    """DRAM bytes per launch of the fused kernel from the committed ncu
    summary, or None when the summary is for other kernel sources or another
    grid size (the L2-resident share depends on the size)."""
    path = os.path.join(ROOT, "profiles", "leja_iter_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    ent = rec.get(kernel_name)
    if not ent or ent.get("source_sha") != kernel_source_sha() or int(ent.get("points", 0)) != n_points:
        return None
    return float(ent["dram_bytes_per_point"]) * n_points


def host_cpu():
    """CPU model of this host (lscpu's model name, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def oracle_steps(n: int, steps: int, warmup: int, parallel: bool):
    """The oracle, as it stands, on the benchmark's recipe at n x n: the
    10-pass power bound, then `warmup` untimed and `steps` timed
    Rosenbrock-Euler steps.  Returns (GDOF*iter/s, seconds, iterations)."""
    import oracle

    u = synth.gaussians_ic(n, n, seed=1)
    h = CFL_MULT * synth.cfl_step(n, n, NU, ADV)
    v0 = synth.power_start(n * n, seed=5)
    rho, _, _ = oracle.power_iteration(oracle.ADVDIFF, n, n, NU, ADV, None, v0, 10, parallel=parallel)
    c, g = oracle.spectral_interval(rho)
    xi = oracle.leja_points(1000)
    for _ in range(warmup):
        u, it, st = oracle.ros_eu(oracle.ADVDIFF, n, n, NU, ADV, u, c, g, h, TOL, TOL, xi, parallel=parallel)
    total = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        u, it, st = oracle.ros_eu(oracle.ADVDIFF, n, n, NU, ADV, u, c, g, h, TOL, TOL, xi, parallel=parallel)
        total += it
    dt = time.perf_counter() - t0
    return n * n * total / dt / 1e9, dt, total


def cpu_baseline(n: int, steps: int):
    """The oracle's OpenMP build on all host cores, on the benchmark's own
    workload (a bounded number of steps), plus its single-threaded parity
    build on one step at half the grid size."""
    import oracle

    try:
        cores = oracle.threads(True)
        par = True
    except Exception:  # no OpenMP on this host: the parity build, one core
        cores, par = 1, False
    val, dt, its = oracle_steps(n, steps, 0, par)
    val1, dt1, its1 = oracle_steps(n // 2, 1, 0, False)
    build = "-O3 -fopenmp build" if par else "single-threaded build (no OpenMP on this host)"
    return {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"{steps} Ros-Eu steps at {n}x{n} ({its} Leja iterations, {dt:.2f} s) with the oracle's "
                      f"{build}, after its 10-pass power bound",
            "single_thread": {"value": val1, "unit": UNIT, "cores": 1,
                              "sample": f"one Ros-Eu step at {n // 2}x{n // 2} ({its1} Leja iterations, "
                                        f"{dt1:.2f} s), the single-threaded parity build"}}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle

    val, dt, its = oracle_steps(NX, args.steps, args.warmup, True)
    cores = oracle.threads(True)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "advdiff-4096x4096-rosenbrock-euler", "nx": NX, "ny": NX, "nu": NU,
                       "a": ADV, "h_over_dt_cfl": CFL_MULT, "tol": TOL,
                       "note": "the CPU oracle, as it stands, built with -O3 -fopenmp, on all host cores"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": host_cpu(),
                             "sample": f"{args.steps} Ros-Eu steps at {NX}x{NX} ({its} Leja iterations)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def symbol_radius(n, nu, a):
    """Largest |lambda| of the periodic central-difference operator (its
    discrete Fourier symbol): the spectral bound given to each batched
    instance as an input."""
    t = 2 * np.pi * np.fft.fftfreq(n)
    re = nu * (2 * np.cos(t) - 2) * n * n
    im = a * np.sin(t) * n
    return float(np.max(np.abs((re[:, None] + re[None, :]) + 1j * (im[:, None] + im[None, :]))))


def run_batch(args, rank, world, local):
    """Batched workload: 256 instances, n ~ U{128..1024}, nu log-U[1e-3, 1e-1],
    a ~ U[0, 2], one exp(hA)v per instance per step, h = 50 dt_CFL each.
    Compares the batched launch with the plain per-instance path."""
    import torch

    import paper_2310_08344_gb300 as lx

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    inst = synth.batch_instances(256, seed=7)
    probs = [(d["n"], d["n"], d["nu"], d["a"]) for d in inst]
    ws, outs, cs, gs, hs = [], [], [], [], []
    for d in inst:
        n = d["n"]
        ws.append(torch.from_numpy(synth.gaussians_ic(n, n, seed=d["seed"])).cuda())
        outs.append(torch.empty(n * n, dtype=torch.float64, device="cuda"))
        c, g = lx.spectral_interval(symbol_radius(n, d["nu"], d["a"]))
        cs.append(c)
        gs.append(g)
        hs.append(CFL_MULT * synth.cfl_step(n, n, d["nu"], d["a"]))
    npts = np.array([d["n"] ** 2 for d in inst], dtype=np.float64)
    b = lx.batch_setup(probs, 1000, stream)
    for _ in range(args.warmup):
        lx.batch_step(b, 0, ws, outs, cs, gs, hs, TOL, TOL)
    lx.batch_stats(b, reset=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    units = 0.0
    statuses = None
    for _ in range(args.steps):
        st, its, sts = lx.batch_step(b, 0, ws, outs, cs, gs, hs, TOL, TOL)
        units += float(np.dot(npts, its))
        statuses = sts
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stats = lx.batch_stats(b, reset=True)
    value = units / (ms / 1e3) / 1e9
    # the same batch in float-float (every n here is a multiple of 128)
    bd = lx.batch_setup(probs, 1000, stream, precision=lx.DF64)
    for _ in range(args.warmup):
        lx.batch_step(bd, 0, ws, outs, cs, gs, hs, TOL, TOL)
    torch.cuda.synchronize()
    e0.record(stream)
    dunits = 0.0
    for _ in range(args.steps):
        st, its_d, sts_d = lx.batch_step(bd, 0, ws, outs, cs, gs, hs, TOL, TOL)
        dunits += float(np.dot(npts, its_d))
    e1.record(stream)
    torch.cuda.synchronize()
    dms = e0.elapsed_time(e1)
    dvalue = dunits / (dms / 1e3) / 1e9
    bd.close()
    # plain form: one context and one phi_l_apply (one graph loop) per instance
    ctxs = [lx.leja_setup(n, n, nu, a, lx.ADVDIFF, lx.FP64, lx.ROS_EU, 1000, stream) for (n, _, nu, a) in probs]
    for _ in range(max(1, args.warmup)):
        for k, ctx in enumerate(ctxs):
            lx.phi_l_apply(ctx, 0, None, ws[k], outs[k], cs[k], gs[k], hs[k], TOL, TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    punits = 0.0
    plain_steps = max(1, args.steps // 2)
    for _ in range(plain_steps):
        for k, ctx in enumerate(ctxs):
            st, it = lx.phi_l_apply(ctx, 0, None, ws[k], outs[k], cs[k], gs[k], hs[k], TOL, TOL)
            punits += npts[k] * it
    torch.cuda.synchronize()
    pdt = time.perf_counter() - t0
    pvalue = punits / pdt / 1e9
    ok = sum(1 for s_ in statuses if s_ == 0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch-256-advdiff-128..1024", "instances": 256, "points": int(npts.sum()),
                       "h_over_dt_cfl": CFL_MULT, "tol": TOL, "converged_instances": ok,
                       "failed_instances_note": "advection-dominated instances (4 nu n / a < ~2) diverge with real "
                                                "Leja points and report a failure status",
                       "batch_launches_per_step": stats["loop_iterations"] / max(args.steps, 1)},
            "plain": {"value": pvalue, "unit": UNIT, "ms_per_step": pdt * 1e3 / plain_steps,
                      "path": "one phi_l_apply (graph loop) per instance"},
            "speedup_vs_plain": (pdt / plain_steps) / (ms / 1e3 / args.steps),
            "float_float_batch": {"value": dvalue, "unit": UNIT, "ms_per_step": dms / args.steps,
                                  "converged_instances": sum(1 for s_ in sts_d if s_ == 0),
                                  "speedup_vs_plain": (pdt / plain_steps) / (dms / 1e3 / args.steps)}}
    if rank == 0:
        print(json.dumps(line))
    for ctx in ctxs:
        ctx.close()
    b.close()
    return 0


def run_paper(args, rank, world, local):
    """The paper's own test problems (Sec. 3) on periodic [-1,1)^2 with the
    third-order upwind gradient and the central Laplacian, diffusion 1 and
    advection / flux coefficient 10, tolerance 1e-12:
      paper1: u_t = A u, one exp(h A) u per step (Leja exponential),
      paper2: u_t = A u + S, Rosenbrock-Euler (phi_1 of A u + S),
      paper3: u_t = Lap u + 5 ((u^2)_x + (u^2)_y), EXPRB32 with a power
              bound before every step.
    Grid --n (the paper uses 8192 and 16384), h = --cfl x dt_CFL.  With --tf
    the run integrates from t = 0 to that final time (the last step shortened)
    and reports the device time of the whole integration, for comparison with
    the paper's end-to-end runtimes (16384^2, T_f = 2e-6, 100 dt_CFL)."""
    import torch

    import paper_2310_08344_gb300 as lx

    if args.tf is not None:
        return run_paper_tf(args, rank, world, local)

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n = args.n
    N = n * n
    nu, a, tol = 1.0, 10.0, 1e-12
    which = args.workload
    prec_name = args.precision
    prec = {"fp64": lx.FP64, "mixed": lx.MIXED, "df64": lx.DF64}[prec_name]
    kind = lx.BURGERS_UP3 if which == "paper3" else lx.ADVDIFF_UP3
    integ = lx.EXPRB32 if which == "paper3" else lx.ROS_EU
    ctx = lx.leja_setup(n, n, nu, a, kind, prec, integ, 1000, stream)
    if args.kernel and lx.lx_ctx_select_kernel(ctx, args.kernel, args.strip_h) != 0:
        raise SystemExit(f"unknown kernel {args.kernel}")
    u0 = synth.problem3_ic(n, n) if which == "paper3" else synth.problem1_ic(n, n)
    ua = torch.from_numpy(u0).cuda()
    ub = torch.empty_like(ua)
    lo = torch.empty_like(ua)
    v0 = torch.from_numpy(synth.power_start(N, seed=5)).cuda()
    amax = a * (float(np.abs(u0).max()) if which == "paper3" else 1.0)
    h = args.cfl * synth.cfl_step_pm1(n, n, nu, amax)
    src = None
    if which == "paper2":
        src = torch.from_numpy(synth.problem2_source(n, n)).cuda()
        lx.lx_ctx_set_source(ctx, src)
    st, rho, _ = lx.power_bound(ctx, ua if which == "paper3" else None, v0, 10)
    c, g = lx.spectral_interval(rho)

    def step(x, y):
        nonlocal c, g
        if which == "paper1":
            st, it = lx.phi_l_apply(ctx, 0, None, x, y, c, g, h, tol, tol)
            return st, it
        if which == "paper3":
            st, r, _ = lx.power_bound(ctx, x, v0, 10)
            c, g = lx.spectral_interval(r)
            st2, err, it = lx.expint_step(ctx, x, lo, y, c, g, h, tol, tol)
            return st or st2, it
        st, err, it = lx.expint_step(ctx, x, None, y, c, g, h, tol, tol)
        return st, it

    cur, nxt = ua, ub
    for _ in range(max(args.warmup, 1)):
        st, it = step(cur, nxt)
        if st != 0:
            raise SystemExit(f"{which} step failed: {st}")
        cur, nxt = nxt, cur
    lx.lx_ctx_stats(ctx, reset=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        st, it = step(cur, nxt)
        if st != 0:
            raise SystemExit(f"{which} step failed: {st}")
        iters.append(it)
        cur, nxt = nxt, cur
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stats = lx.lx_ctx_stats(ctx, reset=True)
    value = float(N) * sum(iters) / (ms / 1e3) / 1e9
    ipl = lx.lx_ctx_iters_per_launch(ctx)
    avg_iter_s = stats["loop_ms"] / 1e3 / max(stats["loop_iterations"], 1)
    alg = (40 if which == "paper3" else 32) * N  # y, p read + write (+ u for J(u)) per iteration
    peaks, peak_src = measured_peaks()
    achieved = alg / avg_iter_s / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "df64": "f32x2 (float-float, FP64-accurate)"}[prec_name],
            "data": "synthetic",
            "config": {"workload": f"{which}-{n}x{n}-upwind3-[-1,1]^2", "diffusion": nu, "advection": a,
                       "h_over_dt_cfl": args.cfl, "tol": tol, "precision": prec_name,
                       "leja_iters_per_step": iters, "kernel": lx.lx_ctx_kernel_name(ctx)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None, "iterations_per_launch": ipl,
                         "alg_bytes_per_iteration": alg, "avg_iteration_us": avg_iter_s * 1e6,
                         "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst copy)"},
            "gpu_launches": int(stats["kernels"])}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


# The paper's end-to-end runtimes on one A100 for 16384^2, T_f = 2e-6,
# dt = 100 dt_CFL, tol 1e-12 (its runtime table; context, another machine).
PAPER_A100_S = {"paper1": 4.76, "paper2": 4.14, "paper3": 15.5}


def run_paper_tf(args, rank, world, local):
    import torch

    import paper_2310_08344_gb300 as lx

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n = args.n
    N = n * n
    nu, a, tol = 1.0, 10.0, 1e-12
    which = args.workload
    prec = {"fp64": lx.FP64, "mixed": lx.MIXED, "df64": lx.DF64}[args.precision]
    kind = lx.BURGERS_UP3 if which == "paper3" else lx.ADVDIFF_UP3
    integ = lx.EXPRB32 if which == "paper3" else lx.ROS_EU
    ctx = lx.leja_setup(n, n, nu, a, kind, prec, integ, 1000, stream)
    if args.kernel and lx.lx_ctx_select_kernel(ctx, args.kernel, args.strip_h) != 0:
        raise SystemExit(f"unknown kernel {args.kernel}")
    u0 = synth.problem3_ic(n, n) if which == "paper3" else synth.problem1_ic(n, n)
    amax = a * (float(np.abs(u0).max()) if which == "paper3" else 1.0)
    h = args.cfl * synth.cfl_step_pm1(n, n, nu, amax)
    v0 = torch.from_numpy(synth.power_start(N, seed=5)).cuda()
    src = torch.from_numpy(synth.problem2_source(n, n)).cuda() if which == "paper2" else None
    if src is not None:
        lx.lx_ctx_set_source(ctx, src)
    ua = torch.from_numpy(u0).cuda()
    ub, lo = torch.empty_like(ua), torch.empty_like(ua)

    def integrate(u, v):
        t, steps, iters = 0.0, 0, 0
        st, rho, _ = lx.power_bound(ctx, u if which == "paper3" else None, v0, 10)
        c, g = lx.spectral_interval(rho)
        while t < args.tf * (1 - 1e-12):
            hh = min(h, args.tf - t)
            if which == "paper3":
                st, rho, _ = lx.power_bound(ctx, u, v0, 10)
                c, g = lx.spectral_interval(rho)
                st, err, it = lx.expint_step(ctx, u, lo, v, c, g, hh, tol, tol)
            elif which == "paper1":
                st, it = lx.phi_l_apply(ctx, 0, None, u, v, c, g, hh, tol, tol)
            else:
                st, err, it = lx.expint_step(ctx, u, None, v, c, g, hh, tol, tol)
            if st != 0:
                raise SystemExit(f"{which} step failed: {st}")
            u, v = v, u
            t += hh
            steps += 1
            iters += it
        return steps, iters

    integrate(ua.clone(), ub)  # warm-up run (graphs, coefficients)
    u = ua.clone()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps, iters = integrate(u, ub)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    ref = PAPER_A100_S.get(which) if (n == 16384 and abs(args.tf - 2e-6) < 1e-18 and args.cfl == 100.0) else None
    line = {"metric": "s to T_f (end to end, device time)", "value": sec, "unit": "s", "n_gpus": world,
            "steps": steps, "warmup": 1, "ms_per_step": sec * 1e3 / max(steps, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": (sec / ref) if ref else None,
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "df64": "f32x2 (float-float, FP64-accurate)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{which}-{n}x{n}-upwind3-[-1,1]^2-tf{args.tf:g}", "tf": args.tf,
                       "h_over_dt_cfl": args.cfl, "tol": tol, "leja_iters_total": iters,
                       "gdof_leja_iter_per_s": N * iters / sec / 1e9, "kernel": lx.lx_ctx_kernel_name(ctx),
                       "paper_a100_s": ref,
                       "note": "vs_baseline = this time / the paper's A100 time for the same workload (context: "
                               "another machine, and dt_CFL read as min(dx^2/4nu, dx/2a))"}}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def run_vertical(args, rank, world, local):
    """Vertical interpolation at 4096^2 (diffusion-advection, nu = 1e-2, a = 1,
    h = 50 dt_CFL): phi_1(alpha_j h A) w for alpha = 1/4, 1/2, 3/4, 1 from one
    Newton basis, against four separate phi_l_apply calls, each form in FP64
    and float-float; also the largest difference between the two forms."""
    import torch

    import paper_2310_08344_gb300 as lx

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n = args.n
    N = n * n
    alphas = [0.25, 0.5, 0.75, 1.0]
    w = torch.from_numpy(synth.gaussians_ic(n, n, seed=1)).cuda()
    h = CFL_MULT * synth.cfl_step(n, n, NU, ADV)
    c, g = lx.spectral_interval(symbol_radius(n, NU, ADV))
    forms = {}
    for prec_name, prec in (("fp64", lx.FP64), ("df64", lx.DF64)):
        ctx = lx.leja_setup(n, n, NU, ADV, lx.ADVDIFF, prec, lx.ROS_EU, 1000, stream)
        outs_v = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in alphas]
        outs_s = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in alphas]

        def vertical():
            st, it = lx.phi_l_apply_vertical(ctx, 1, alphas, None, w, outs_v, c, g, h, TOL, TOL)
            if st != 0:
                raise SystemExit(f"phi_l_apply_vertical failed: {st}")
            return it

        def separate():
            its = []
            for j, al in enumerate(alphas):
                st, it = lx.phi_l_apply(ctx, 1, None, w, outs_s[j], c, g, h * al, TOL, TOL)
                if st != 0:
                    raise SystemExit(f"phi_l_apply failed: {st}")
                its.append(it)
            return its

        res = {}
        for name, fn in (("vertical", vertical), ("separate", separate)):
            for _ in range(max(args.warmup, 1)):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its = None
            for _ in range(args.steps):
                its = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = {"ms_per_call": e0.elapsed_time(e1) / args.steps, "leja_iters": its}
        diff = max(float(torch.linalg.norm(outs_v[j] - outs_s[j]) / torch.linalg.norm(outs_s[j]))
                   for j in range(len(alphas)))
        res["speedup_vs_separate"] = res["separate"]["ms_per_call"] / res["vertical"]["ms_per_call"]
        res["max_rel_l2_vertical_vs_separate"] = diff
        forms[prec_name] = res
        ctx.close()
    best = forms["df64"]["vertical"]
    line = {"metric": "ms per vertical phi call (4 step fractions)", "value": best["ms_per_call"],
            "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": best["ms_per_call"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2 (float-float, FP64-accurate)", "data": "synthetic",
            "config": {"workload": f"vertical-{n}x{n}-phi1-alpha4", "alphas": alphas, "nu": NU, "a": ADV,
                       "h_over_dt_cfl": CFL_MULT, "tol": TOL},
            "forms": forms}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_rhs(args, rank, world, local):
    """The unfused form (a caller's right-hand side, the Jacobian action by
    central differences) on the 4096^2 diffusion-advection Rosenbrock-Euler
    step (nu = 1e-2, a = 1, h = 50 dt_CFL, tol 1e-10): f from the engine's
    own FP64 right-hand side (lx_rhs_builtin) and from a Python/torch
    function, against the fused FP64 and float-float paths on the same step.
    Algorithmic bytes per point per Leja iteration of the unfused form:
    perturbation 32 (u, y in; x+, x- out), two calls of f 2 x 16, update 48
    (f(x+), f(x-), y, p in; y', p out) = 112."""
    import torch

    import paper_2310_08344_gb300 as lx

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n = args.n
    N = n * n
    u = torch.from_numpy(synth.gaussians_ic(n, n, seed=1)).cuda()
    h = CFL_MULT * synth.cfl_step(n, n, NU, ADV)
    c, g = lx.spectral_interval(symbol_radius(n, NU, ADV))
    prob = (n, n, NU, ADV, lx.ADVDIFF)

    def f_torch(x, out):
        X = x.view(n, n)
        L = (torch.roll(X, 1, 1) + torch.roll(X, -1, 1) - 2 * X) * (n * n) + \
            (torch.roll(X, 1, 0) + torch.roll(X, -1, 0) - 2 * X) * (n * n)
        G = (torch.roll(X, -1, 1) - torch.roll(X, 1, 1) + torch.roll(X, -1, 0) - torch.roll(X, 1, 0)) * (n / 2)
        out.copy_((NU * L + ADV * G).view(-1))

    out = torch.empty(N, dtype=torch.float64, device="cuda")
    forms = {}
    results = {}
    for name in ("unfused_builtin", "unfused_torch", "fused_fp64", "fused_df64"):
        if name.startswith("unfused"):
            ctx = lx.leja_setup_rhs(N, f=f_torch if name == "unfused_torch" else None,
                                    problem=None if name == "unfused_torch" else prob, stream=stream)

            def step():
                st, err, it = lx.expint_step_rhs(ctx, u, None, out, c, g, h, TOL, TOL)
                if st != 0:
                    raise SystemExit(f"expint_step_rhs failed: {st}")
                return it
        else:
            ctx = lx.leja_setup(n, n, NU, ADV, lx.ADVDIFF, lx.FP64 if name == "fused_fp64" else lx.DF64,
                                lx.ROS_EU, 1000, stream)
            if name == "fused_df64" and not args.no_autotune:
                lx.lx_ctx_autotune(ctx, iters=10)

            def step():
                st, err, it = lx.expint_step(ctx, u, None, out, c, g, h, TOL, TOL)
                if st != 0:
                    raise SystemExit(f"expint_step failed: {st}")
                return it
        for _ in range(max(args.warmup, 1)):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = 0
        for _ in range(args.steps):
            its += step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        rec = {"ms_per_step": ms, "leja_iters_per_step": its / args.steps,
               "gdof_iter_per_s": N * its / args.steps / (ms * 1e-3) / 1e9}
        if name.startswith("unfused"):
            rec["rhs_calls"] = lx.lx_rhs_ctx_stats(ctx)["rhs_calls"]
            rec["algorithmic_gbs"] = 112.0 * N * its / args.steps / (ms * 1e-3) / 1e9
        results[name] = out.clone()
        forms[name] = rec
        ctx.close()
    for name in ("unfused_builtin", "unfused_torch", "fused_df64"):
        forms[name]["rel_l2_vs_fused_fp64"] = float(torch.linalg.norm(results[name] - results["fused_fp64"]) /
                                                    torch.linalg.norm(results["fused_fp64"]))
    best = forms["unfused_builtin"]
    peaks, peak_src = measured_peaks()
    hbm = peaks["hbm_gbs"]
    line = {"metric": "GDOF*Leja-iter/s", "value": best["gdof_iter_per_s"], "unit": "GDOF*iter/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rhs-unfused-{n}x{n}-rosenbrock-euler", "nu": NU, "a": ADV,
                       "h_over_dt_cfl": CFL_MULT, "tol": TOL, "eps0": 2.0 ** -18,
                       "l2": "inputs larger than L2 (128 MiB per vector)"},
            "roofline": {"bound": "hbm", "achieved": best["algorithmic_gbs"], "peak": hbm, "unit": "GB/s",
                         "frac": best["algorithmic_gbs"] / hbm, "traffic": None, "peak_source": peak_src,
                         "note": "whole unfused Leja loop, 112 algorithmic bytes per point-iteration"},
            "forms": forms}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_learned(args, rank, world, local):
    """The learned step-size controller on its workload: the network shipped
    with the package (trained by paper_2310_08344_gb300/train_controller.py
    on Burgers trajectories at 256^2 and 512^2 with the library's
    tensor-core kernels) applied to Burgers at n^2 (default 2048^2,
    nu = 5e-3), adaptive EXPRB32 to T = 200 dt_CFL (the scope's test) and to
    T = 2000 dt_CFL (a run the ramp-up does not dominate), from a first step
    of 10 dt_CFL, against the classical controller from the same step; the
    embedded error test accepts or rejects every step in all runs.  Reported:
    Leja iterations, steps, rejections, wall time per simulated time unit
    (best of three runs) and the error of the final state against a
    tight-tolerance run."""
    import torch

    import paper_2310_08344_gb300 as lx
    from paper_2310_08344_gb300 import learned

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    tol, leja_tol = 1e-4, 1e-10
    model, meta = learned.load_model(stream=stream)
    n = args.n if args.n != NX else 2048
    nu = 5e-3
    N = n * n
    u0 = synth.burgers_ic(n, n, seed=12)
    dt = synth.cfl_step(n, n, nu, float(np.abs(u0).max()))
    v0 = torch.from_numpy(synth.power_start(N, seed=5)).cuda()
    prec = {"fp64": lx.FP64, "mixed": lx.MIXED, "df64": lx.DF64}[args.precision]
    ctx = lx.leja_setup(n, n, nu, 0.0, lx.BURGERS, prec, lx.EXPRB32, 1000, stream)
    h0 = 10 * dt
    horizons = {}
    for horizon in (200, 2000):
        T = horizon * dt
        ref = torch.from_numpy(u0).cuda()
        st, _ = lx.lx_integrate(ctx, ref, v0, T, 1e-9, leja_tol, 100000, 0.0, h0, 10)
        if st != 0:
            raise SystemExit(f"reference run failed: {st}")
        runs = {}
        for name in ("classical", "learned"):
            best = None
            for _ in range(3):
                u = torch.from_numpy(u0).cuda()
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                if name == "classical":
                    st, info = lx.lx_integrate(ctx, u, v0, T, tol, leja_tol, 100000, 0.0, h0, 10)
                else:
                    st, info = lx.lx_integrate_learned(ctx, u, v0, T, tol, leja_tol, model, dt, 100000, 0.0, h0, 10)
                torch.cuda.synchronize()
                wall = time.perf_counter() - t1
                if st != 0:
                    raise SystemExit(f"{name} run failed: {st}")
                if best is None or wall < best["wall_ms"] / 1e3:
                    best = {"leja_iters": info["leja_iters"], "steps": info["steps"], "rejected": info["rejected"],
                            "wall_ms": wall * 1e3, "wall_ms_per_unit_time": wall * 1e3 / T,
                            "rel_err_vs_tight": float((u - ref).norm().item() / ref.norm().item())}
            runs[name] = best
        c, l = runs["classical"], runs["learned"]
        horizons[f"T={horizon}dt_CFL"] = {"runs": runs, "gain_leja_iters": c["leja_iters"] / max(l["leja_iters"], 1),
                                          "gain_wall": c["wall_ms"] / l["wall_ms"]}
    main_h = horizons["T=200dt_CFL"]
    line = {"metric": "Leja iterations to T, classical / learned controller", "value": main_h["gain_leja_iters"],
            "unit": "ratio", "n_gpus": world, "steps": 1, "warmup": 0,
            "ms_per_step": main_h["runs"]["learned"]["wall_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "df64": "f32x2 (float-float, FP64-accurate)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"learned-controller-burgers-{n}x{n}", "nu": nu, "tol": tol, "leja_tol": leja_tol,
                       "first_step_over_dt_cfl": 10,
                       "network": {k: meta[k] for k in ("samples", "groups", "label", "candidates", "loss_last",
                                                        "epochs") if k in meta}},
            "horizons": horizons, "wall_gain": main_h["gain_wall"]}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def run_burgers(args, rank, world, local):
    """Viscous Burgers 2048^2, nu = 5e-3, EXPRB32 steps of h = 50 dt_CFL with
    a power-iteration bound before every step; FP64, mixed and float-float
    forms, and each form's difference from the FP64 path after the same
    steps; the same for EPIRK4s3A steps (FP64 and float-float)."""
    import torch

    import paper_2310_08344_gb300 as lx

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    n, nu = args.n if args.n != NX else 2048, 5e-3
    N = n * n
    u0 = synth.burgers_ic(n, n, seed=1)
    h = CFL_MULT * synth.cfl_step(n, n, nu, float(np.abs(u0).max()))
    v0 = torch.from_numpy(synth.power_start(N, seed=5)).cuda()
    results = {}
    finals = {}
    forms = (("fp64", lx.FP64, lx.EXPRB32), ("mixed", lx.MIXED, lx.EXPRB32), ("df64", lx.DF64, lx.EXPRB32),
             ("epirk4s3a_fp64", lx.FP64, lx.EPIRK4S3A), ("epirk4s3a_df64", lx.DF64, lx.EPIRK4S3A))
    if args.forms:
        want = set(args.forms.split(","))
        forms = tuple(f for f in forms if f[0] in want)
        if not forms:
            raise SystemExit(f"--forms: none of {sorted(want)} is a Burgers form")
    for prec_name, prec, integ in forms:
        ctx = lx.leja_setup(n, n, nu, 0.0, lx.BURGERS, prec, integ, 1000, stream)
        tune = None
        if args.kernel and prec == lx.DF64:
            if lx.lx_ctx_select_kernel(ctx, args.kernel, args.strip_h) != 0:
                raise SystemExit(f"--kernel {args.kernel} is not a float-float Burgers candidate")
        elif not args.no_autotune:
            _, tune = lx.lx_ctx_autotune(ctx, 10, None)
        u = torch.from_numpy(u0).cuda()
        lo, hi = torch.empty_like(u), torch.empty_like(u)

        def step():
            st, rho, _ = lx.power_bound(ctx, u, v0, 10)
            c, g = lx.spectral_interval(rho)
            st2, err, it = lx.expint_step(ctx, u, lo, hi, c, g, h, TOL, TOL)
            if st != 0 or st2 != 0:
                raise SystemExit(f"burgers step failed: {st} {st2}")
            u.copy_(hi)
            return it, err

        for _ in range(args.warmup):
            step()
        u.copy_(torch.from_numpy(u0))
        lx.lx_ctx_stats(ctx, reset=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its, errs = [], []
        for _ in range(args.steps):
            it, err = step()
            its.append(it)
            errs.append(err)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stt = lx.lx_ctx_stats(ctx, reset=True)
        results[prec_name] = {"value": N * sum(its) / (ms / 1e3) / 1e9, "ms_per_step": ms / args.steps,
                              "leja_iters": its, "err_estimates": errs,
                              "avg_iteration_us": 1e3 * stt["loop_ms"] / max(stt["loop_iterations"], 1),
                              "power_ms_per_step": stt["power_ms"] / args.steps,
                              "kernel": lx.lx_ctx_kernel_name(ctx),
                              "autotune_us_per_iteration": {f"{t['kernel']}/H{t['strip_h']}": round(t["us"], 2)
                                                            for t in (tune or {}).get("timings", [])}}
        finals[prec_name] = u.clone()
        ctx.close()
    def diff(a, b):
        if a not in finals or b not in finals:
            return None
        return float((finals[a] - finals[b]).norm().item() / finals[b].norm().item())

    head = results["fp64"] if "fp64" in results else next(iter(results.values()))
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if "fp64" in results else "f32x2 (float-float, FP64-accurate)", "data": "synthetic",
            "config": {"workload": f"burgers-{n}x{n}-exprb32", "nu": nu, "h_over_dt_cfl": CFL_MULT, "tol": TOL,
                       "power_iteration": "10 passes before every step", "forms": [f[0] for f in forms]},
            "forms": results, "mixed_vs_fp64_rel_l2_after_steps": diff("mixed", "fp64"),
            "df64_vs_fp64_rel_l2_after_steps": diff("df64", "fp64"),
            "epirk4s3a_df64_vs_fp64_rel_l2_after_steps": diff("epirk4s3a_df64", "epirk4s3a_fp64")}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch256":
        return run_batch(args, rank, world, local)
    if args.workload == "burgers2048":
        return run_burgers(args, rank, world, local)
    if args.workload == "vertical4096":
        return run_vertical(args, rank, world, local)
    if args.workload == "rhs4096":
        return run_rhs(args, rank, world, local)
    if args.workload == "learned2048":
        return run_learned(args, rank, world, local)
    if args.workload in ("paper1", "paper2", "paper3"):
        return run_paper(args, rank, world, local)
    import torch

    import paper_2310_08344_gb300 as lx

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    n = args.n
    N = n * n
    prec = {"fp64": lx.FP64, "mixed": lx.MIXED, "df64": lx.DF64}[args.precision]
    stream = torch.cuda.current_stream()
    ctx = lx.leja_setup(n, n, NU, ADV, lx.ADVDIFF, prec, lx.ROS_EU, 1000, stream)
    if args.unroll and lx.lx_ctx_set_graph_unroll(ctx, args.unroll) != 0:
        raise SystemExit(f"bad --unroll {args.unroll}")
    tune = None
    if args.kernel:
        if lx.lx_ctx_select_kernel(ctx, args.kernel, args.strip_h) != 0:
            raise SystemExit(f"unknown kernel {args.kernel}")
        tune = {"selected": {"kernel": args.kernel, "strip_h": args.strip_h, "forced": True}}
    elif not args.no_autotune:
        st, tune = lx.lx_ctx_autotune(ctx, 10, None)
        if st != 0:
            raise SystemExit(f"autotune failed: {st}")
    kname = lx.lx_ctx_kernel_name(ctx)
    u0 = synth.gaussians_ic(n, n, seed=1)
    h = CFL_MULT * synth.cfl_step(n, n, NU, ADV)
    ua = torch.from_numpy(u0).cuda()
    ub = torch.empty_like(ua)
    v0 = torch.from_numpy(synth.power_start(N, seed=5)).cuda()
    st, rho, _ = lx.power_bound(ctx, None, v0, 10)
    if st != 0:
        raise SystemExit(f"power_bound failed: {st}")
    c, g = lx.spectral_interval(rho)
    if args.source:
        src_field = torch.from_numpy(synth.source_field(n, n, seed=21)).cuda()
        if lx.lx_ctx_set_source(ctx, src_field) != 0:
            raise SystemExit("lx_ctx_set_source failed")

    def step(src, dst):
        st, err, it = lx.expint_step(ctx, src, None, dst, c, g, h, args.tol, args.tol)
        if st != 0:
            raise SystemExit(f"expint_step failed: {lx.STATUS.get(st, st)}")
        return it

    cur, nxt = ua, ub
    for _ in range(max(args.warmup, 0)):
        step(cur, nxt)
        cur, nxt = nxt, cur
    lx.lx_ctx_stats(ctx, reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        iters.append(step(cur, nxt))
        cur, nxt = nxt, cur
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stats = lx.lx_ctx_stats(ctx, reset=True)
    units = float(N) * sum(iters)
    t_local = ms / 1e3
    t_max, units_all = aggregate(pg, t_local, units)
    value = units_all / t_max / 1e9

    # dominant kernel: the fused Leja iteration, ipl iterations per launch
    # (2 for the two-step kernel).  Algorithmic bytes per launch = 32 B per
    # point-iteration x the point-iterations of one launch; the loop's event
    # time per iteration includes the launches that found the loop stopped.
    ipl = lx.lx_ctx_iters_per_launch(ctx)
    avg_iter_s = stats["loop_ms"] / 1e3 / max(stats["loop_iterations"], 1)
    avg_launch_s = avg_iter_s * ipl
    alg_bytes = ALG_BYTES[args.precision] * N * ipl
    peaks, peak_src = measured_peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    traffic = ncu_traffic(kname, N)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": kname, "iterations_per_launch": ipl, "alg_bytes_per_launch": alg_bytes,
                "avg_launch_us": avg_launch_s * 1e6,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst copy)"}
    if ipl > 1:
        # the kernel itself moves 32 B per point per launch (y_m, p_m in;
        # y_{m+ipl}, p_{m+ipl} out): report that share of HBM too
        own = ALG_BYTES[args.precision] * N
        roofline["min_dram_bytes_per_launch"] = own
        roofline["min_dram_frac"] = own / avg_launch_s / 1e9 / peaks["hbm_gbs"]
        roofline["note"] = ("temporal blocking: one launch performs ipl Leja iterations and moves the bytes of one, "
                            "so frac can exceed the kernel's own DRAM share (min_dram_frac)")
    launches = int(stats["kernels"])  # counted by the library on the context stream

    # the plain form (native FP64 kernels) on the same steps from the same
    # initial state: time per step and the difference of the final states
    plain = None
    if not args.no_plain and args.precision != "fp64":
        ctxp = lx.leja_setup(n, n, NU, ADV, lx.ADVDIFF, lx.FP64, lx.ROS_EU, 1000, stream)
        if args.source:
            lx.lx_ctx_set_source(ctxp, src_field)
        pc, pn = torch.from_numpy(u0).cuda(), torch.empty_like(ua)

        def pstep(s_, d_):
            st, err, it = lx.expint_step(ctxp, s_, None, d_, c, g, h, args.tol, args.tol)
            if st != 0:
                raise SystemExit(f"plain expint_step failed: {lx.STATUS.get(st, st)}")
            return it

        for _ in range(max(args.warmup, 0)):
            pstep(pc, pn)
            pc, pn = pn, pc
        lx.lx_ctx_stats(ctxp, reset=True)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        pits = []
        for _ in range(args.steps):
            pits.append(pstep(pc, pn))
            pc, pn = pn, pc
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1) / args.steps
        # the FP64 kernel against its two ceilings: the FP64 pipe (8 FP64
        # FMA-class instructions per point-iteration: 5 for the folded
        # stencil, 1 Newton update, 2 norms) and HBM (32 B per point-iteration)
        pst = lx.lx_ctx_stats(ctxp, reset=True)
        p_launch_s = pst["loop_ms"] / 1e3 / max(pst["loop_iterations"], 1)
        p_ach = FP64_OPS_PER_POINT_ITER * N / p_launch_s / 1e9
        p_hbm = ALG_BYTES["fp64"] * N / p_launch_s / 1e9
        plain_roofline = {"bound": "alu", "achieved": p_ach, "peak": FP64_FMA_PEAK_G, "unit": "G FP64 FMA/s",
                          "frac": p_ach / FP64_FMA_PEAK_G, "traffic": None,
                          "kernel": lx.lx_ctx_kernel_name(ctxp), "avg_launch_us": p_launch_s * 1e6,
                          "ops_per_point_iteration": FP64_OPS_PER_POINT_ITER,
                          "peak_source": "nominal GB300 FP64 1.25 TFLOP/s = 625 G FMA/s (no measured FP64 peak "
                                         "in MEASURED_PEAKS.json)",
                          "hbm": {"achieved": p_hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                  "frac": p_hbm / peaks["hbm_gbs"],
                                  "alu_ceiling_frac": FP64_FMA_PEAK_G * 1e9 / FP64_OPS_PER_POINT_ITER
                                  * ALG_BYTES["fp64"] / 1e9 / peaks["hbm_gbs"]}}
        plain = {"precision": "fp64 (native FP64 kernels)", "kernel": lx.lx_ctx_kernel_name(ctxp),
                 "roofline": plain_roofline,
                 "value": float(N) * sum(pits) / (pms * args.steps / 1e3) / 1e9, "ms_per_step": pms,
                 "leja_iters_per_step": pits, "chosen_speedup": pms / (ms / args.steps),
                 "rel_l2_final_chosen_vs_plain": float(torch.linalg.norm(cur - pc) / torch.linalg.norm(pc))}
        ctxp.close()

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        hin = torch.from_numpy(cur.cpu().numpy()).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        st, err, it = lx.expint_step_host(ctx, hin, None, hout, c, g, h, args.tol, args.tol)  # warm
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tot_it = 0
        for _ in range(args.steps):
            st, err, it = lx.expint_step_host(ctx, hin, None, hout, c, g, h, args.tol, args.tol)
            if st != 0:
                raise SystemExit(f"expint_step_host failed: {st}")
            tot_it += it
            hin, hout = hout, hin
        dt = time.perf_counter() - t0
        e_units = float(N) * tot_it
        dt, e_units = aggregate(pg, dt, e_units)
        e2e = {"value": e_units / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N,
               "path": "expint_step_host (pinned host buffers, copies inside the timed region)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, 2)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "df64": "f32x2 (float-float, FP64-accurate)"}[args.precision],
                "data": "synthetic",
                "config": {"workload": ("advdiff-4096x4096-rosenbrock-euler" if n == 4096 else f"advdiff-{n}x{n}")
                           + ("-source" if args.source else ""),
                           "nx": n, "ny": n, "nu": NU, "a": ADV, "h_over_dt_cfl": CFL_MULT, "tol": args.tol,
                           "precision": args.precision, "integrator": "ros_eu", "parallelism": f"replicas{world}",
                           "leja_iters_per_step": iters, "rho": rho,
                           "kernel_selected": (tune or {}).get("selected", {"kernel": kname}),
                           "l2": "inputs larger than L2 (128 MiB per vector, 512 MiB moved per Leja iteration)"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "plain": plain}
        print(json.dumps(line))
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
