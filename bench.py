#!/usr/bin/env python
"""Throughput of SIMPLE Krylov-vector solves on a 100^3 cosine-stretched grid.

One step = one Krylov-vector evaluation of Section 3 (Eqs. 8-10): the
momentum predictor w = J.v of Eq. 10 followed by the SIMPLE-like projection
loop (pressure-correction solve, velocity/pressure correction) until
||phi_k||_inf <= 1e-8 ||phi_1||_inf.  Workload: lid parallel to the x
sidewall, Re = 1900, 100^3 cosine-stretched grid, mixed precision (FP32
sweeps inside the FP64 defect-correction loop); right-hand sides are 16
seeded Gaussian velocity fields (seeds 1..16, 384 MB, more than the 126 MB
L2) used in rotation.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(plain definition: J.v + exact tensor-product projection) on the same
workload instead.  Under torchrun every rank runs its own replica (the path
has no exchange step): value = all ranks' solves / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 100
RE = 1900.0
ALPHA = 0.0
EPS = 1e-8
NRHS = 16
METRIC = "SIMPLE Krylov-vector solves/s (100^3, tol 1e-8)"
WORKLOAD = "100^3 cosine grid, lid parallel to the x sidewall (alpha=0), Re=1900: SIMPLE Krylov-vector solve to 1e-8"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-eigenpair", action="store_true",
                    help="skip the 16^3 time-to-leading-eigenpair measurement")
    ap.add_argument("--no-mg", action="store_true", help="skip the multigrid pressure-solve measurement")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            if len(s) >= 9:
                for nme, val in zip(names, s[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nme)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# algorithmic bytes (or flops) of one launch of each kernel class of the
# mixed path: float32 operands, float-float (8 B) SIMPLE state, float32
# pressure-correction transforms: per cell 4 n flop for the two 1-D transforms
# of a fused launch (2 n each)
def algorithmic(kind, n, prec):
    cells = n ** 3
    if prec != "mixed":
        f = 8
        table = {"momentum": 72, "correct": 24 + 8 + 16 + 24 + 8, "divergence": 32}
    else:
        f = 4
        table = {"momentum": 36,                 # read U, v (3 x 4 B each), write w (3 x 4 B)
                 "correct": 24 + 4 + 16 + 24 + 4,  # read v (ff), phi, r/w p (ff), write v (ff), r
                 "divergence": 16}               # read w (3 x 4 B), write r
    if kind in ("tpf_x", "tpf_xinv", "tpf_yz"):
        # fused tensor-core kernels (n <= 112) apply two 1-D transforms per
        # launch (2 n flop per cell each) and read + write the float32 field
        # once; the unfused ones apply one transform on the FP32 pipes
        k = 2 if n <= 112 else 1
        return {"flops": k * 2 * n * cells, "bytes": 2 * f * cells, "fused": n <= 112}
    return {"bytes": table.get(kind, 16) * cells}


def traffic_for(kind):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since that capture."""
    try:
        import hashlib
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        ent = t.get(kind)
        if not ent:
            return None
        src = open(os.path.join(ROOT, "paper_1704_08521_gb300", "csrc", ent["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest()[:16] != ent["sha"]:
            return None
        return ent["bytes_per_launch"]
    except Exception:
        return None


def run_ours(args):
    import torch
    import torch.distributed as dist
    import numpy as np

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1704_08521_gb300 as fv
    import synth

    n = args.n
    shape = (n, n, n)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    g = fv.Grid(n, n, n, "cosine", alpha=ALPHA, re=RE)
    U = torch.tensor(synth.vortex_base_flow(shape, "cosine", ALPHA), device=dev)
    # the base flow is registered once, as a Krylov method does for the
    # thousands of vectors it takes about one steady state
    g.set_base(U)
    V = [torch.tensor(synth.gaussian_velocity(shape, 1 + s + 1000 * rank), device=dev) for s in range(NRHS)]
    out = torch.empty(g.n_vel, dtype=torch.float64, device=dev)
    p = torch.empty(g.n_cell, dtype=torch.float64, device=dev)

    mixed = args.prec == "mixed"

    def step(s, prec=args.prec, async_=None):
        a = (prec == "mixed") if async_ is None else async_
        return fv.simple_krylov_solve(g, None, V[s % NRHS], out, p, eps=EPS, prec=prec, async_=a)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for s in range(args.warmup):
        step(s)
    st = step(0, async_=False)                  # one synchronised call: loop statistics
    passes = st["passes"]
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = fv.fv_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for s in range(args.steps):
        step(s)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    host_launches = fv.fv_launch_count() - l0
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = ws * args.steps / (ms_max / 1e3)
    # kernels per evaluation: graph = init, round, J.v, D w, pressure solve,
    # correct, decide (first pass) + solve, correct, decide per further pass
    # + join; the pressure solve is 3 fused kernels for n <= 128, else 6
    tpf_k = 3 if n <= 112 else 6
    kernels_per_solve = (7 + tpf_k + (tpf_k + 2) * (passes - 1)) if mixed else None
    gpu_launches = kernels_per_solve * args.steps if mixed else host_launches

    # same workload in the plain FP64 form, a few steps (context for the
    # mixed-precision speed-up; not the headline)
    fp64 = None
    if mixed:
        k64 = max(3, min(args.steps, 10))
        step(0, "fp64")
        barrier()
        e0.record(stream)
        for s in range(k64):
            step(s, "fp64")
        e1.record(stream)
        barrier()
        fp64 = k64 / (e0.elapsed_time(e1) / 1e3)

    # the float-float form (FP64-level accuracy on the FP32 pipes), a few steps
    ff_rate = None
    if mixed:
        kff = max(3, min(args.steps, 10))
        step(0, "ff", async_=False)
        barrier()
        e0.record(stream)
        for s in range(kff):
            step(s, "ff", async_=True)
        e1.record(stream)
        barrier()
        ff_rate = kff / (e0.elapsed_time(e1) / 1e3)

    # the multigrid pressure solve (the iterative alternative to the
    # tensor-product solve) on this grid: D G phi = D (L_U v) to a relative
    # residual of 1e-8, and the FP64 Krylov vector whose SIMPLE passes use it
    mg = None
    if mixed and not args.no_mg:
        mg = mg_measure(fv, torch, g, U, V[0], n, stream, barrier)

    # one Arnoldi cycle (Krylov dimension 60: 60 Krylov vectors + CGS2 in the
    # W-inner product + the Hessenberg step) on this base flow: time per
    # Arnoldi iteration, the unit the paper's eigenvalue times are made of
    arnoldi_ms = {}
    if mixed:
        for prec in ("mixed", "ff"):
            barrier()
            t0 = time.perf_counter()
            try:
                fv.arnoldi_leading(g, U, V[0], m=60, nev=10, max_restarts=1, prec=prec)
            except fv.FvError:
                pass                      # one cycle is not enough to converge
            torch.cuda.synchronize()
            arnoldi_ms[prec] = 1e3 * (time.perf_counter() - t0) / 60

    # per-kernel device time: back-to-back launches of each kernel class on
    # the grid's stream, timed with CUDA events (fv_bench_kernel)
    prof = {}
    if mixed:
        step(0, async_=False)
        if n <= 112:     # fused: tpf_x / tpf_xinv = forward / inverse x-y slab kernel,
                         # tpf_yz = one z-column kernel
            per_solve = {"momentum": 1, "divergence": 1, "correct": passes, "tpf_x": passes,
                         "tpf_xinv": passes, "tpf_yz": passes}
        else:
            per_solve = {"momentum": 1, "divergence": 1, "correct": passes, "tpf_x": 2 * passes,
                         "tpf_yz": 4 * passes}
        for kind, cnt in per_solve.items():
            prof[kind] = (fv.fv_bench_kernel(g, kind, reps=50), cnt)

    # end to end through the public API: each step copies its right-hand side
    # from pinned host memory, solves, and reads the result back to pinned host
    # memory.  Double-buffered pipeline: the input copy of step s + 1 (one copy
    # stream) and the read-back of step s - 1 (a second one, the link is full
    # duplex) overlap the solve of step s on the grid's stream; events keep
    # every buffer from being overwritten before its solve / read-back is done.
    hin = [V[s].cpu().pin_memory() for s in range(min(NRHS, 4))]
    hout = [torch.empty(g.n_vel, dtype=torch.float64).pin_memory() for _ in range(2)]
    vin = [torch.empty_like(out) for _ in range(2)]
    vout = [torch.empty_like(out) for _ in range(2)]
    cs_in, cs_out = torch.cuda.Stream(), torch.cuda.Stream()
    h2d_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    d2h_done = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(nsteps):
        with torch.cuda.stream(cs_in):
            vin[0].copy_(hin[0], non_blocking=True)
            h2d_done[0].record(cs_in)
        for s in range(nsteps):
            b = s & 1
            if s + 1 < nsteps:
                with torch.cuda.stream(cs_in):
                    if s >= 1:
                        cs_in.wait_event(comp_done[1 - b])    # solve s - 1 read vin[1 - b]
                    vin[1 - b].copy_(hin[(s + 1) % len(hin)], non_blocking=True)
                    h2d_done[1 - b].record(cs_in)
            stream.wait_event(h2d_done[b])
            if s >= 2:
                stream.wait_event(d2h_done[b])                # step s - 2 read vout[b] back
            fv.simple_krylov_solve(g, None, vin[b], vout[b], p, eps=EPS, prec=args.prec, async_=mixed)
            comp_done[b].record(stream)
            with torch.cuda.stream(cs_out):
                cs_out.wait_event(comp_done[b])
                hout[b].copy_(vout[b], non_blocking=True)
                d2h_done[b].record(cs_out)
        stream.wait_stream(cs_in)
        stream.wait_stream(cs_out)

    e2e_run(2)
    barrier()
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e = ws * args.steps / (float(t.item()) / 1e3)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    # roofline of the dominant kernel class (largest device time per solve)
    pk = peaks()
    roof = None
    breakdown = {}
    if prof:
        tot = sum(v[0] * v[1] for v in prof.values())
        breakdown = {k: {"ms_per_launch": v[0], "launches_per_solve": v[1],
                         "ms_per_solve": v[0] * v[1], "share": v[0] * v[1] / tot}
                     for k, v in prof.items()}
        kind = max(prof, key=lambda k: prof[k][0] * prof[k][1])
        per_launch_s = prof[kind][0] / 1e3
        alg = algorithmic(kind, n, args.prec)
        clock_mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
        if "flops" in alg and alg.get("fused"):
            # fused transforms: 4 n flop over 8 bytes per cell (50 flop/B at
            # n = 100) sit below the TF32 ridge point of the measured peaks, so
            # the byte floor binds: reported against HBM, with the tensor
            # fraction (three split-TF32 products per product) beside it
            peak = pk.get("hbm_gbs", 6800.0)
            achieved = alg["bytes"] / per_launch_s / 1e9
            tf32 = pk.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
            roof = {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "traffic": traffic_for(kind),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "tensor_tflops": alg["flops"] / per_launch_s / 1e12,
                    "tensor_frac": alg["flops"] / per_launch_s / 1e12 / tf32,
                    "tensor_peak_source": "MEASURED_PEAKS.json bf16_tflops x 1.1/2.25 (nominal TF32/BF16)",
                    "note": "tcgen05.mma kind::tf32 (TMEM accumulators), a*b = a_lo b_hi + a_hi b_lo + a_hi b_hi"}
        elif "flops" in alg:
            peak = 152 * 128 * 2 * clock_mhz * 1e6 / 1e12
            achieved = alg["flops"] / per_launch_s / 1e12
            roof = {"bound": "alu", "kernel": kind, "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic_for(kind),
                    "peak_source": f"FP32 FMA: 152 SM x 128 lanes x 2 flop x {clock_mhz:.0f} MHz "
                                   "(median SM clock under load)",
                    "hbm_frac": alg["bytes"] / per_launch_s / 1e9 / pk.get("hbm_gbs", 6800.0)}
        else:
            peak = pk.get("hbm_gbs", 6800.0)
            achieved = alg["bytes"] / per_launch_s / 1e9
            roof = {"bound": "hbm", "kernel": kind, "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "traffic": traffic_for(kind),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    # whole-solve HBM roofline on the algorithmic bytes of one Krylov-vector
    # evaluation, 36 + 80 K per cell (K SIMPLE passes: J.v reads v and U and
    # writes w in float32; each pass moves the float64 state and the float32
    # pressure right-hand side and correction), over the time per solve; beside
    # it the bytes this implementation moves by design (float64 x read by J.v,
    # D w, three transform launches and the fused correction per pass, join of
    # v and p to float64)
    solve_roof = None
    if mixed:
        bpc = 36 + 80 * passes
        impl = 48 + 16 + passes * (3 * 8 + 72) + 64
        bytes_solve = bpc * n ** 3
        ach = bytes_solve * value / ws / 1e9
        pk_hbm = pk.get("hbm_gbs", 6800.0)
        solve_roof = {"bound": "hbm", "bytes_per_solve": bytes_solve, "bytes_per_cell": bpc,
                      "achieved": ach, "peak": pk_hbm, "unit": "GB/s", "frac": ach / pk_hbm,
                      "implementation_bytes_per_cell": impl,
                      "implementation_frac": impl * n ** 3 * value / ws / 1e9 / pk_hbm,
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    step_ms = ms_max / args.steps
    # bytes moved per step
    h2d = g.n_vel * 8
    d2h = g.n_vel * 8
    res = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 state / f32 sweeps" if args.prec == "mixed" else "f64",
        "data": "synthetic (seeded Gaussian right-hand sides; analytic lid-driven-like base flow)",
        "config": {"workload": WORKLOAD, "grid": f"{n}^3", "map": "cosine", "re": RE, "alpha": ALPHA,
                   "tol": EPS, "prec": args.prec, "rhs_rotation": NRHS,
                   "l2": f"inputs rotate over {NRHS} vectors ({NRHS * g.n_vel * 8 / 1e6:.0f} MB) > L2",
                   "base_flow": "registered once per run (fv_grid_set_base), U=NULL per solve",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "simple_passes": passes,
        "sweeps_per_s": value * passes,
        "mcell_jv_per_s": None,
        "fp64_form_solves_per_s": fp64,
        "ff_form_solves_per_s": ff_rate,
        "arnoldi_iteration_ms": arnoldi_ms,
        "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pipeline": "pinned host buffers; copies of steps s+1 / s-1 overlap the solve of step s"},
        "gpu_launches": gpu_launches,
        "kernels_per_solve": kernels_per_solve,
        "roofline": roof,
        "solve_roofline": solve_roof,
        "kernel_breakdown": breakdown,
        "mg_pressure": mg,
        "clocks": clocks,
    }
    mom = prof.get("momentum")
    if mom:
        res["mcell_jv_per_s"] = n ** 3 / (mom[0] / 1e3) / 1e6
    if not args.no_eigenpair and rank == 0:
        res["time_to_leading_eigenpair"] = eigenpair_16(fv, torch, dev, synth)
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(n, budget_s=12.0)
    if ws > 1:
        dist.destroy_process_group()
    return res


def mg_levels(n):
    """Cell counts of the multigrid hierarchy of an n^3 grid (coarsening of
    every axis with more than 2 cells while one has more than 4)."""
    m, out = n, [n ** 3]
    while m > 4:
        m = (m + 1) // 2 if m > 2 else m
        out.append(m ** 3)
    return out


def mg_measure(fv, torch, g, U, v, n, stream, barrier, reps=5):
    """Multigrid pressure solve at rtol 1e-8: CG iterations, ms per solve and
    per V-cycle, and the line-smoothing sweeps' bandwidth on their
    algorithmic bytes (x in, b in, x out: 12 B per cell per sweep; six sweeps
    per level above the coarsest)."""
    w = torch.empty(g.n_vel, dtype=torch.float64, device=v.device)
    fv.ns_jacvec(g, U, v, w, prec="fp64")
    r = torch.empty(g.n_cell, dtype=torch.float64, device=v.device)
    fv.ns_divergence(g, w, r)
    phi = torch.empty_like(r)
    st = fv.fv_pressure_solve_mg(g, r, phi, rtol=1e-8)
    barrier()
    fv.fv_profile_enable(g, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fv.fv_pressure_solve_mg(g, r, phi, rtol=1e-8)
    e1.record(stream)
    barrier()
    prof = fv.fv_profile_read(g)
    fv.fv_profile_enable(g, False)
    ms = e0.elapsed_time(e1) / reps
    its = st["iterations"]
    sm_ms, sm_n = prof["mg_smooth"]
    lv = mg_levels(n)
    alg_bytes = 6 * 12 * sum(lv[:-1]) * its * reps
    peak = peaks().get("hbm_gbs", 6800.0)
    sm_gbs = alg_bytes / (sm_ms / 1e3) / 1e9 if sm_ms > 0 else None
    # the FP64 Krylov vector with multigrid pressure passes
    out = torch.empty_like(v)
    fv.simple_krylov_solve(g, None, v, out, eps=EPS, prec="fp64", pressure="mg")
    barrier()
    e0.record(stream)
    for _ in range(3):
        st2 = fv.simple_krylov_solve(g, None, v, out, eps=EPS, prec="fp64", pressure="mg")
    e1.record(stream)
    barrier()
    return {"rtol": 1e-8, "levels": st["levels"], "cg_iterations": its, "ms_per_solve": ms,
            "ms_per_vcycle_iteration": ms / max(its, 1),
            "smooth_ms_per_solve": sm_ms / reps, "smooth_launches_per_solve": sm_n / reps,
            "smooth_share": sm_ms / reps / ms,
            "smooth_roofline": {"bound": "hbm", "achieved": sm_gbs, "peak": peak, "unit": "GB/s",
                                "frac": sm_gbs / peak if sm_gbs else None,
                                "bytes_per_cell_per_sweep": 12},
            "fp64_krylov_vector_mg": {"solves_per_s": 3 / (e0.elapsed_time(e1) / 1e3),
                                      "passes": st2["passes"], "pressure_rtol_per_pass": 1e-3}}


def eigenpair_16(fv, torch, dev, synth, precs=("fp64", "mixed", "ff")):
    """Time to the leading eigenpair on the 16^3 configuration (Re 1000, lid
    parallel to the x sidewall, cosine grid): Newton from rest to ||F|| <
    1e-10 by continuation in Re (200, 400, ..., 1000), then the 5 leading
    eigenvalues by implicitly restarted Arnoldi (Krylov dimension 30, Philox
    Gaussian start vector of seed 1, Ritz tolerance 1e-10).  Wall time around
    the library calls, synchronised on both sides."""
    N = 16
    out = {"workload": "16^3 cosine grid, Re 1000, alpha 0: Newton from rest + Arnoldi(30, 5 eigenvalues)"}
    v0 = torch.tensor(synth.gaussian_velocity((N, N, N), 1), device=dev)
    for prec in precs:
        g = fv.Grid(N, N, N, "cosine", alpha=0.0, re=200.0)
        U = torch.zeros(g.n_vel, dtype=torch.float64, device=dev)
        P = torch.zeros(g.n_cell, dtype=torch.float64, device=dev)
        # the steady state by the FP64 form or by mixed precision (which turns
        # to FP64 Krylov vectors near the root); Arnoldi in the form named
        nprec = "fp64" if prec == "fp64" else "mixed"
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps = 0
            for re in (200.0, 400.0, 600.0, 800.0, 1000.0):
                g.set_re(re)
                steps += fv.newton_steady(g, U, P, tol=1e-10, prec=nprec)["iterations"]
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            lam, info = fv.arnoldi_leading(g, U, v0, m=30, nev=5, prec=prec)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            out[prec] = {"newton_prec": nprec, "newton_s": t1 - t0, "arnoldi_s": t2 - t1,
                         "total_s": t2 - t0, "newton_steps": steps,
                         "arnoldi_matvecs": info["matvecs"], "lambda_1": [lam[0].real, lam[0].imag]}
        except fv.FvError as e:
            out[prec] = {"error": str(e)[:160]}
    return out


def oracle_solver(n):
    import numpy as np
    import synth
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import layout
    from oracle import grid as og, poisson, simple
    shape = (n, n, n)
    G = og.Grid(n, n, n, "cosine")
    T = poisson.TPF(G)
    U = layout.to_oracle(synth.vortex_base_flow(shape, "cosine", ALPHA), shape)
    rhs = [layout.to_oracle(synth.gaussian_velocity(shape, 1 + s), shape) for s in range(2)]

    def solve(s):
        return simple.krylov_vector(G, T, U, rhs[s % 2], RE)
    return solve


def cores_used():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max(i.get("num_threads", 1) for i in info) if info else 1
    except Exception:
        return os.cpu_count()


def cpu_baseline(n, budget_s=12.0):
    solve = oracle_solver(n)
    solve(0)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < budget_s or k < 2:
        solve(k)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "solves/s", "cores": cores_used(), "kind": "oracle",
            "sample": f"{k} Krylov-vector solves of the {n}^3 workload (numpy FP64, exact projection)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    solve = oracle_solver(args.n)
    for s in range(args.warmup):
        solve(s)
    t0 = time.perf_counter()
    for s in range(args.steps):
        solve(s)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "grid": f"{args.n}^3"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores_used(), "kind": "oracle",
                             "sample": f"{args.steps} Krylov-vector solves of the {args.n}^3 workload"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
