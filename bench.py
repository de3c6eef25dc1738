"""Benchmark of the radiation-field hot path on the stellar-wind workload.

Workload: 50 000-point spherical wind (log-uniform r in [1, 100] R*, Delaunay
neighbours, beta-law velocity, T ~ r^-0.7), one line, 50 frequency bins,
HEALPix nside 4 (96 ray pairs per point).  One step = the whole hot path on
device-resident inputs: ray set -> trace (padded rows + overflow) -> velocity
and optical-depth sampling -> Feautrier solve of every (point, pair, bin) -> J.

Metric: ray-pair x frequency Feautrier solves per second of the single-precision
form (FP64 for the distance increments, the integer decisions of Section 2.1.1
and Eq. 2, and the J sum); the FP64 plain form is timed beside it.  Under torchrun every rank solves its own replica of the
workload (independent models, no collective: weak scaling); value is the total
over ranks divided by the slowest rank's time.

`--impl reference` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-pair x frequency Feautrier solves/s (FP32 form; FP64 distance increments, decisions, J sum) on the 50k-point wind"
UNIT = "solves/s"
WORKLOAD = dict(workload="stellar wind, 50000 points, Delaunay neighbours, 1 line x 50 bins, nside 4 "
                         "(96 ray pairs/point), dtau_max 0.5, dv_max 1/3 Doppler width",
                n_points=50000, n_pairs=96, n_bins=50)
FLOPS_PER_UPDATE = 14      # elimination + trapezoid + source function per (bin, sub-interval)
FLOPS_PER_SAMPLE_LINE = 9  # profile argument, Gaussian, chi/eta accumulation per (bin, sample, line)
L2_BYTES = 129 * 2 ** 20


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t: float, ws: int, device=None) -> float:
    """The slowest rank's value of t (t itself on one rank); device is "cuda"
    for NCCL process groups and None (host tensor) for gloo."""
    if ws <= 1:
        return t
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


# a rank that fails or never arrives ends the others' next collective with an
# error after this long, instead of leaving them waiting
PG_TIMEOUT_S = 600


def job_throughput(ws: int, units_per_rank_step: float, steps: int, t_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return ws * units_per_rank_step * steps / t_max


def make_workload(n=50000, seed=2):
    import synth

    return synth.wind_model(n, seed=seed, n_freq=50, level=2)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_physical_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            return int(vis.split(",")[local_rank])
        except (ValueError, IndexError):
            pass
    return local_rank


def cpu_baseline(m, rays, target_s=15.0, seed=0):
    """The FP64 oracle as it stands, on all host cores, on a bounded origin sample."""
    import oracle

    threads = os.cpu_count() or 1
    om = oracle.OracleModel(m, rays=rays)
    pr = oracle.params(dtau_max=0.5, dv_max=1.0 / 3.0)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(m["pos"]))
    probe = order[:2 * threads]
    t0 = time.perf_counter()
    Jp = om.solve_J(pr, origins=probe, threads=threads)
    tp = time.perf_counter() - t0
    k = int(max(len(probe), min(len(order), len(probe) * max(1.0, (target_s - tp) / max(tp, 1e-3)))))
    rest = order[len(probe):k]
    t1 = time.perf_counter()
    Jr = om.solve_J(pr, origins=rest, threads=threads) if len(rest) else np.zeros((0, Jp.shape[1]))
    tr = time.perf_counter() - t1
    origins = np.concatenate([probe, rest])
    J = np.concatenate([Jp, Jr])
    solves = len(origins) * rays.shape[1] * J.shape[1]
    t = tp + tr
    return dict(value=solves / t, unit=UNIT, cores=threads, kind="oracle",
                sample=f"{len(origins)} random origins of the 50k-point workload (all 96 pairs x 50 bins), "
                       f"{t:.1f} s on {threads} host threads"), origins, J


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    import synth

    oracle.build()
    m = make_workload()
    rays = oracle.rayset(m["pos"], 2, 2)
    threads = os.cpu_count() or 1
    om = oracle.OracleModel(m, rays=rays)
    pr = oracle.params(dtau_max=0.5, dv_max=1.0 / 3.0)
    rng = np.random.default_rng(1)
    per_step = max(threads, 4 * threads)  # origins per step: bounded sample
    for _ in range(args.warmup):  # untimed, one origin per thread each
        om.solve_J(pr, origins=rng.integers(0, len(m["pos"]), threads), threads=threads)
    times, solves = [], 0
    for _ in range(args.steps):
        o = rng.integers(0, len(m["pos"]), per_step)
        t0 = time.perf_counter()
        J = om.solve_J(pr, origins=o, threads=threads)
        times.append(time.perf_counter() - t0)
        solves += len(o) * rays.shape[1] * J.shape[1]
    T = sum(times)
    v = solves / T
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, parallelism="host threads"),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} random origins per step (all 96 pairs x 50 bins)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_mgx(args):
    import torch

    import paper_2011_14998_gb300 as mgx

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        import datetime

        dist.init_process_group("nccl", device_id=torch.device("cuda", local),
                                timeout=datetime.timedelta(seconds=PG_TIMEOUT_S))
    torch.cuda.set_device(local)
    mgx.build()
    m = make_workload()
    n, NB = len(m["pos"]), len(m["nu0"]) * int(m["n_freq"])
    stream = torch.cuda.Stream(local)
    ctx = mgx.Context(local, stream)
    mid = ctx.load(m)
    npairs = ctx.models[mid]["npairs"]
    solves_per_step = n * npairs * NB
    out32 = torch.empty((n, NB), dtype=torch.float64, device="cuda")
    out64 = torch.empty((n, NB), dtype=torch.float64, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    batched = mgx.MGX_BATCH_GRAPH | mgx.MGX_BATCH_RAYS

    def step32():
        # the FP32 batched form: ray sets, tracing, length-binned work list and the
        # persistent solve, replayed as one CUDA graph
        ctx.solve_J_batch([mid], precision=mgx.MGX_FP32, dtau_max=0.5, dv_max=1.0 / 3.0, outs=[out32],
                          flags=batched)

    out32h = torch.empty((n, NB), dtype=torch.float64, device="cuda")

    def step32h():
        # the same batched step with the Hermitian (fourth-order) scheme
        ctx.solve_J_batch([mid], precision=mgx.MGX_FP32, dtau_max=0.5, dv_max=1.0 / 3.0, outs=[out32h],
                          flags=batched, order=4)

    out32d = torch.empty((n, NB), dtype=torch.float64, device="cuda")

    def step32d():
        # the batched step with the optical-depth increments and the elimination pivots in FP64
        ctx.solve_J_batch([mid], precision=mgx.MGX_FP32_DT64, dtau_max=0.5, dv_max=1.0 / 3.0, outs=[out32d],
                          flags=batched)

    def step32_profiled():
        ctx.solve_J_batch([mid], precision=mgx.MGX_FP32, dtau_max=0.5, dv_max=1.0 / 3.0, outs=[out32],
                          flags=mgx.MGX_BATCH_RAYS)

    def step64():
        # the FP64 plain form: grid-mapped solve, one warp per origin and 32-bin tile
        ctx.set_rays(mid, 2, 2)
        ctx.solve_J(mid, precision=mgx.MGX_FP64, dtau_max=0.5, dv_max=1.0 / 3.0, out=out64)

    def timed(stepfn, k, warm, profile):
        for _ in range(warm):
            stepfn()
        torch.cuda.synchronize()
        ev = []
        if profile:
            ctx.profile(True)
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()  # evict the mesh from L2 between timed steps
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            stepfn()
            with torch.cuda.stream(stream):
                b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        prof = None
        if profile:
            prof = ctx.profile_read()
            ctx.profile(False)
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3, prof

    # measured throughput of the arithmetic pipes (the solve's roofline denominators), untimed
    alu = mgx.mgx_alu_peaks(ctx.ptr, 3)
    # launch parameters of the batched step from the autotuner (untimed; results do not depend on them)
    trials, _ = ctx.autotune([mid], precision=mgx.MGX_FP32, dtau_max=0.5, dv_max=1.0 / 3.0, outs=[out32],
                             flags=batched, reps=3)
    tuning = ctx.tuning()

    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_physical_index(local)) as clk:
        t32, _ = timed(step32, args.steps, args.warmup, False)
    t32 = max_over_ranks(t32, ws, "cuda")
    if ws > 1:
        torch.distributed.barrier()
    value = job_throughput(ws, solves_per_step, args.steps, t32)
    kh = max(1, min(args.steps, 5))
    t32h, _ = timed(step32h, kh, max(3, min(args.warmup, 3)), False)
    kd = max(1, min(args.steps, 3))
    t32d, _ = timed(step32d, kd, 1, False)
    # per-kernel CUDA-event breakdown of the same step, launched without the graph
    kb = max(1, min(args.steps, 3))
    tb, prof32 = timed(step32_profiled, kb, 1, True)

    # FP64 plain form on the same inputs (fewer steps: it is much slower on GB300)
    k64 = max(1, args.fp64_steps)
    t64, prof64 = timed(step64, k64, 1, True)
    value64 = solves_per_step * k64 / t64
    J32 = out32.cpu().numpy()
    J64 = out64.cpu().numpy()

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    host = {k: torch.from_numpy(np.ascontiguousarray(m[k])).pin_memory()
            for k in ("pos", "vel", "nbr_off", "nbr_idx", "nu0", "chi0", "eta0", "dvw", "chi_c", "eta_c")}
    host["nbr_idx"] = torch.from_numpy(np.ascontiguousarray(m["nbr_idx"], np.int32)).pin_memory()
    Jh = torch.empty((n, NB), dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = Jh.numel() * Jh.element_size()

    def e2e_step():
        # host inputs in, host J out (the batched call stages J on the device and copies it back)
        mm = mgx.mgx_load_mesh(ctx.ptr, host["pos"], host["vel"], host["nbr_off"], host["nbr_idx"])
        mgx.mgx_set_lines(ctx.ptr, mm, host["nu0"], host["chi0"], host["eta0"], host["dvw"], host["chi_c"],
                          host["eta_c"], m["n_freq"], m["x_span"])
        mgx.mgx_set_rays(ctx.ptr, mm, 2, 2, None)
        mgx.mgx_solve_J_batch(ctx.ptr, [mm], mgx.solve_params(0.5, 1.0 / 3.0, 0.0, mgx.MGX_FP32, True), [Jh], 0)
        mgx.mgx_free_model(ctx.ptr, mm)

    e2e_step()
    torch.cuda.synchronize()
    k_e2e = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    te = max_over_ranks(te, ws, "cuda")
    e2e_value = job_throughput(ws, solves_per_step, k_e2e, te)
    assert np.array_equal(Jh.numpy(), J32), "end-to-end J differs from the device-resident run"

    if rank != 0:
        ctx.close()
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    # accuracy of the FP32 form: against the GPU FP64 form everywhere, and against the oracle on a sample
    mx = np.abs(J64).max(axis=1, keepdims=True)
    mask = np.abs(J64) > 1e-6 * mx
    rel32_64 = np.abs(J32 - J64)[mask] / np.abs(J64[mask])
    J32d = out32d.cpu().numpy()
    rel32d_64 = np.abs(J32d - J64)[mask] / np.abs(J64[mask])
    cpu = None
    acc_oracle = None
    acc_herm = None
    if not args.no_cpu_baseline:
        cpu, origins, Jo = cpu_baseline(m, ctx.rays(mid), target_s=args.cpu_seconds)
        mo = np.abs(Jo) > 1e-6 * np.abs(Jo).max(axis=1, keepdims=True)
        acc_oracle = {
            "fp32_max_rel": float((np.abs(J32[origins] - Jo)[mo] / np.abs(Jo[mo])).max()),
            "fp64_max_rel": float((np.abs(J64[origins] - Jo)[mo] / np.abs(Jo[mo])).max()),
            "origins": int(len(origins)),
        }
        acc_herm = hermitian_accuracy(m, ctx.rays(mid), out32h.cpu().numpy())

    # roofline of the dominant kernel (the formal solution), per launch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_derived = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FMA counted as 2
    fp32_peak = alu["fp32_fma_tflops"]
    ms_solve = prof32["ms"]["solve"] / max(1, prof32["launches"]["solve"])
    flops = (FLOPS_PER_UPDATE * prof32["updates"] + FLOPS_PER_SAMPLE_LINE * len(m["nu0"]) * prof32["samples"])
    flops_per_launch = flops / max(1, prof32["launches"]["solve"])
    achieved = flops_per_launch / (ms_solve * 1e-3) / 1e12
    # special-function operations of the solve: one exp2 per (sample, bin, line), one reciprocal per update
    mufu_ops = (len(m["nu0"]) * prof32["samples"] + prof32["updates"]) / max(1, prof32["launches"]["solve"])
    # algorithmic bytes of the solve: a 4-byte point id per traced point and frequency tile (the tile is
    # 32 x bins-per-lane bins), the point data once (positions and velocities in double and single precision,
    # width, continuum and line data: 56 + 8 (L - 1) bytes) and 8 bytes of J per (point, bin)
    tiles = -(-NB // (32 * int(tuning.get("bins_per_lane") or 2)))
    solve_bytes = (prof32["trace_points"] // kb) * 4 * tiles + n * (56 + 8 * (len(m["nu0"]) - 1)) + n * NB * 8
    hbm_gbs = solve_bytes / (ms_solve * 1e-3) / 1e9
    step_ms = {k: v / kb for k, v in prof32["ms"].items()}
    # own kernels per step: ray sets, padded trace, tail trace, the work-list kernels (three for the
    # cost-binned schedule, one for plain order), the solve (scans and the sort are CUB's)
    lp = prof32["launches"]
    wl = 3 if tuning.get("schedule", 0) == 0 else 1
    launches = args.steps * (lp["rays"] + lp["trace_count"] + lp["trace_emit"] + wl * lp["other"] + lp["solve"]) // kb
    traffic = solve_traffic(prof32["trace_points"] // kb)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t32 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, parallelism=f"replicas x{ws}", l2="flushed between timed steps (256 MiB write)",
                       step="one CUDA-graph replay: ray sets, padded trace, tail offsets (scan), tail trace, "
                            "length-binned work list, persistent solve",
                       tuning=tuning, autotune_trials=trials),
        "fp64_plain": {"value": value64, "unit": UNIT, "ms_per_step": 1e3 * t64 / k64,
                       "speedup_fp32_over_fp64": value / ws / value64},
        "hermitian_fp32": {"value": solves_per_step * kh / t32h, "unit": UNIT, "ms_per_step": 1e3 * t32h / kh,
                           "cost_vs_second_order": (t32h / kh) / (t32 / args.steps),
                           "oracle_sample": acc_herm},
        "fp32_dt64": {"value": solves_per_step * kd / t32d, "unit": UNIT, "ms_per_step": 1e3 * t32d / kd,
                      "cost_vs_fp32": (t32d / kd) / (t32 / args.steps),
                      "vs_fp64_max_rel": float(rel32d_64.max()),
                      "vs_fp64_p99_rel": float(np.quantile(rel32d_64, 0.99))},
        "accuracy": {"fp32_vs_fp64_max_rel": float(rel32_64.max()),
                     "fp32_vs_fp64_p99_rel": float(np.quantile(rel32_64, 0.99)),
                     "oracle_sample": acc_oracle},
        "kernel_ms_per_step": step_ms,
        "eager_step_ms": 1e3 * tb / kb,  # same step without the graph, re-planned each call
        "work_per_step": {"solves": solves_per_step, "trace_points": prof32["trace_points"] // kb,
                          "updates": prof32["updates"] // kb, "samples": prof32["samples"] // kb,
                          "trace_steps": prof32["trace_steps"] // kb,
                          "trace_steps_redone_fp64": prof32["trace_exact_steps"] // kb,
                          "solve_decisions_redone_fp64": prof32["decisions_redone"] // kb},
        "roofline": {"kernel": "k_solve_queue<float>", "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                     "peak_source": "measured: FP32 FMA chains on every SM (mgx_alu_peaks), of measured",
                     "traffic_source": "ncu capture of the 20 000-point case (profiles/k_solve_queue_wind20k.md) "
                                       "scaled by traced points per launch; null once the solve source changed",
                     "derived_peak": fp32_derived, "frac_of_derived": achieved / fp32_derived,
                     "mufu": {"ops_per_launch": mufu_ops, "achieved_gops": mufu_ops / (ms_solve * 1e-3) / 1e9,
                              "peak_gops": alu["ex2_gops"],
                              "frac": mufu_ops / (ms_solve * 1e-3) / 1e9 / alu["ex2_gops"]},
                     "measured_alu_peaks": alu,
                     "hbm_algorithmic_gbs": hbm_gbs, "hbm_algorithmic_bytes_per_launch": solve_bytes},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


SOLVE_PROFILE = os.path.join(ROOT, "profiles", "k_solve_queue_wind20k.md")
SOLVE_SOURCES = ("k_solve_impl.cuh", "k_solve.cu")


def hermitian_accuracy(m, rays, J32h, n=200):
    """Largest relative error of the FP32 Hermitian step against the oracle's
    Hermitian solve on n random origins."""
    import oracle

    om = oracle.OracleModel(m, rays=rays)
    o = np.sort(np.random.default_rng(5).choice(len(m["pos"]), n, replace=False))
    Jo = om.solve_J(oracle.params(dtau_max=0.5, dv_max=1.0 / 3.0, order=4), origins=o)
    mask = np.abs(Jo) > 1e-6 * np.abs(Jo).max(axis=1, keepdims=True)
    rel = np.abs(J32h[o] - Jo)[mask] / np.abs(Jo[mask])
    return {"fp32_max_rel": float(rel.max()), "fp32_p99_rel": float(np.quantile(rel, 0.99)), "origins": n}


def solve_traffic(trace_points_per_launch):
    """DRAM bytes of one solve launch: the committed ncu summary's capture of the
    20 000-point case scaled by traced points per launch, or None when the
    kernel source has changed since the counters were taken (the summary
    records the SHA-256 of the solve's sources, concatenated in the order of
    SOLVE_SOURCES)."""
    import hashlib

    try:
        kv = dict(l.strip().split(":", 1) for l in open(SOLVE_PROFILE).read().splitlines()
                  if l.strip().startswith(("dram_", "k_solve_sha256", "trace_points_per_launch")))
        src = b"".join(open(os.path.join(ROOT, "paper_2011_14998_gb300", "csrc", f), "rb").read()
                       for f in SOLVE_SOURCES)
        if hashlib.sha256(src).hexdigest() != kv["k_solve_sha256"].strip():
            return None
        per_point = (int(kv["dram_bytes_read_20k"]) + int(kv["dram_bytes_write_20k"])) / int(
            kv["trace_points_per_launch_20k"])
        return int(per_point * trace_points_per_launch)
    except (OSError, KeyError, ValueError):
        return None


def run_profile_case(args):
    """Two solves of an N-point wind (same generator and settings as the
    benchmark) through the batched entry point without graph capture, so that
    each kernel of the timed step (ray sets, both trace passes, scan, work
    list, persistent solve) is a separate launch a profiler can select."""
    import torch

    import paper_2011_14998_gb300 as mgx

    mgx.build()
    n = args.profile_case
    m = make_workload(n)
    ctx = mgx.Context(0)
    mid = ctx.load(m)
    prec = mgx.MGX_FP64 if args.profile_fp64 else mgx.MGX_FP32
    ctx.profile(True)
    outs = None
    for _ in range(2):
        outs = ctx.solve_J_batch([mid], precision=prec, dtau_max=0.5, dv_max=1.0 / 3.0, outs=outs,
                                 flags=mgx.MGX_BATCH_RAYS)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": n, "counters": ctx.profile_read()}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mgx", choices=["mgx", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="only run two solves of an N-point wind (for profiler captures)")
    ap.add_argument("--profile-fp64", action="store_true")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_mgx(args)


if __name__ == "__main__":
    main()
