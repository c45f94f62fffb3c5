"""Benchmark of the monolithic block-preconditioned Stokes-Darcy solve on GB300.

One step = one implicit-Euler step of the coupled problem (right-hand side,
then block-preconditioned FGMRES to ||b - A x||_2 <= 1e-10 ||b||_2), the
whole hot path.  Default workload: 1024 x 1024 cells per subdomain
(4 196 352 unknowns), mu = 1e-3, alpha_BJ = 1, dt = 0.05, log-normal
permeability (ln K ~ N(-4, 1), exponential covariance, correlation length 16
cells, seed 0).  The headline runs the FP32 multigrid / FP64 outer form; the
FP64-throughout form of the same workload is measured beside it.

Prints one JSON line (rank 0).  Under torchrun every rank runs an
independent replica of the workload (the single-instance solve does not
shard) and the value is the sum of units over the max time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 1024]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "coupled DOF*steps/s at rel.res 1e-10 (FP32-MG vs FP64); p50/p99 solve latency"
UNIT = "DOF*steps/s"
HBM_FALLBACK_GBS = 6800.0
FP64_NOMINAL_TFLOPS = 1.25


def workload_desc(n: int, steps: int) -> str:
    return ("stokes-darcy monolithic, %dx%d cells per subdomain (%d DoF), lognormal K ln K~N(-4,1) "
            "corr 16 cells seed 0, mu=1e-3, alpha_BJ=1, dt=0.05, %d implicit-Euler steps, rtol 1e-10"
            % (n, n, 4 * n * n + 2 * n, steps))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(units: float, seconds: float, ws: int):
    """Whole-job (sum of units, max of seconds) over ranks; identity when ws == 1."""
    if ws == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    s = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def _barrier():
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            dist.barrier()
    except Exception:
        pass


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) < 9:
                        continue
                    try:
                        sm.append(float(p[1]))
                        smax.append(float(p[2]))
                    except ValueError:
                        continue
                    for nm, val in zip(names, p[5:9]):
                        if val.lower() in ("active", "1"):
                            reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


TUNED = ("tile_rows", "coarsest", "cheb_degree")


def tune_form(sd, n, K, precision, stream, enabled: bool):
    """Autotuned (tile_rows, coarsest, cheb_degree) for this grid and precision, outside any timed region."""
    base = sd.sd_options_default()
    base.precision = precision
    base.stream = stream.cuda_stream
    if not enabled:
        return {k: getattr(base, k) for k in TUNED}, None
    cache = os.environ.get("SD_TUNE_CACHE", os.path.join(tempfile.gettempdir(), "sd_tune.txt"))
    t0 = time.perf_counter()
    best, ms = sd.sd_autotune(n, 1e-3, K, 1.0, 0.05, base, 3, cache)
    tuned = {k: getattr(best, k) for k in TUNED}
    return tuned, {"choice": tuned, "tuned_ms_per_step": ms, "seconds": time.perf_counter() - t0,
                   "candidates": "tile_rows {by level,16,8} x coarsest {4,8,16} x cheb_degree {3,2,4}; 4+3 steps each; "
                                 "cache " + os.path.basename(cache)}


def run_form(sd, torch, n, K, precision, steps, warmup, stream, prof_kernel=None, tuned=None, keep_fields=None,
             name=None):
    """Warm up, then time `steps` implicit-Euler steps with CUDA events on `stream`."""
    opts = sd.sd_options_default()
    opts.precision = precision
    opts.stream = stream.cuda_stream
    for k, v in (tuned or {}).items():
        setattr(opts, k, v)
    h = sd.sd_create(n, 1e-3, K, 1.0, 0.05, opts)
    if warmup:
        sd.sd_step(h, warmup)
    if prof_kernel is not None:
        sd.sd_profile(h, prof_kernel, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier()
    torch.cuda.synchronize()
    l0 = sd.sd_launch_count()
    with torch.cuda.stream(stream):
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        infos = sd.sd_step(h, steps)
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    _barrier()
    launches = sd.sd_launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    prof = sd.sd_profile_read(h) if prof_kernel is not None else None
    if keep_fields is not None:
        keep_fields[name] = sd.sd_get_fields(h)
    sd.sd_destroy(h)
    return ms, infos, launches, prof


KERNELS = {0: ("k_apply_full", "sd_ops.cu", True), 1: ("k_smooth_tile_V<float> fine level", "sd_ops.cu", False),
           2: ("k_mupdate", "sd_krylov.cu", True), 3: ("k_mdot", "sd_krylov.cu", True)}


def source_hash(fname: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_2108_13229_gb300", "csrc", fname), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(name: str, fname: str):
    """DRAM bytes per algorithmic byte from the committed ncu summary, if the kernel is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            tab = json.load(f)
        e = tab[name]
        if e.get("source_hash") != source_hash(fname):
            return None
        return e["dram_bytes_per_launch"] / e["algorithmic_bytes_per_launch"]
    except Exception:
        return None


def roofline_entry(kid: int, prof, step_ms: float):
    kms, klaunch, kbytes, kflops = prof
    name, fname, fp64 = KERNELS[kid]
    hbm_peak, hbm_src = read_peaks()
    gbs = (kbytes / 1e9) / (kms / 1e3) if kms > 0 else 0.0
    ratio = ncu_traffic(name, fname)
    traffic = ratio * kbytes / max(klaunch, 1) if ratio is not None else None
    e = {"kernel": name, "launches": klaunch, "avg_launch_us": 1e3 * kms / max(klaunch, 1),
         "share_of_step_time": kms / step_ms if step_ms > 0 else None,
         "bytes_per_launch": kbytes / max(klaunch, 1), "flops_per_launch": kflops / max(klaunch, 1),
         "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak, "traffic": traffic}
    if fp64:
        tf = (kflops / 1e12) / (kms / 1e3) if kms > 0 else 0.0
        e.update({"bound": "alu", "achieved": tf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                  "frac": tf / FP64_NOMINAL_TFLOPS,
                  "peak_source": "nominal FP64 rate of the part (1.25 TFLOP/s at 2070 MHz); FP64 is not in the "
                                 "measured peaks file"})
    else:
        e.update({"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                  "peak_source": hbm_src})
    return e


def level_sizes(n: int, coarsest: int = 16):
    """Cells per side of every multigrid level (the library's halving rule), the last one the dense solve."""
    out = [n]
    while n % 2 == 0 and n // 2 >= 2 and n > coarsest:
        n //= 2
        out.append(n)
    return out


def step_model_bytes(n: int, info: dict, mixed: bool, coarsest: int = 16) -> float:
    """Compulsory HBM bytes of one implicit-Euler step of this algorithm (every array each kernel of the step must
    read or write, once), from the step's FGMRES iterations, restart cycles and second Gram-Schmidt passes.

    FP64 vectors of the Krylov method are 8 B per unknown; the V-cycles move es = 4 (mixed) or 8 B per value:
    per level the velocity block 9.5 passes over its 2n(n+1) faces (pre-smoothing b in x out, residual, restriction,
    post-smoothing with the coarse correction), the Darcy and pressure-Laplacian blocks 13.5 over their n^2 cells
    (the same with the two transmissibility arrays read by each smoothing and residual), the coarsest grid's dense
    FP64 inverses once per V-cycle, and the preconditioner's FP64/FP32 glue."""
    dof = 4.0 * n * n + 2.0 * n
    v8 = 8.0 * dof
    es = 4.0 if mixed else 8.0
    apply_b = 8.0 * (2 * dof + 2.0 * n * (n + 1) + 2 * n)
    resid_b = 8.0 * (3 * dof + 2.0 * n * (n + 1) + 2 * n)
    levels = level_sizes(n, coarsest)
    pre = 0.0
    for m in levels[:-1]:
        pre += 9.5 * es * 2.0 * m * (m + 1) + 2 * 13.5 * es * m * m
    mc = levels[-1]
    mV, mD = 2 * mc * (mc + 1), mc * mc
    pre += 8.0 * (mV * mV + 2 * mD * mD)
    NV, ND = 2.0 * n * (n + 1), float(n * n)
    g = 8.0 + es  # an FP64 value read and its multigrid copy written (or the reverse)
    pre += g * ND + (g * NV + (8 + 4 + 8) * ND if mixed else 16 * NV + 24 * ND) + (g * NV + g * ND) + g * ND
    total = 4 * v8 + 4 * v8 + v8 + resid_b + v8  # rhs, extrapolation, ||b||, first residual and its norm
    iters, restarts, reo = int(info["iters"]), max(1, int(info["restarts"])), int(info.get("reorths", 0))
    m = 30
    for it in range(iters):
        k = it % m + 1
        # the first pass's dots: inside the operator's launch up to 4 basis vectors (k reads), else a multi-dot
        # that reads w as well; the update reads k + 1 vectors and writes one; the new basis vector is scaled
        total += pre + apply_b + (2 * k + (2 if k <= 4 else 3)) * v8 + 2 * v8
    total += reo * 5 * v8  # a second pass, about (2k+3) vectors at the typical k = 1
    for _ in range(restarts):
        total += (min(iters, m) + 2) * v8 + resid_b + v8  # x update, true residual and its norm
    return total + v8  # per-block residual norms


def bench_batch(sd, count: int, steps: int, threads: int, seed: int = 0, lockstep: bool = True, graph: bool = False):
    """Independent instances with uneven grids advanced together by sd_solve_batch: instances of one grid size
    run in lockstep (one launch serves the whole group), groups concurrently on their own streams; graph: every
    step's solves of all groups as one graph launch, decided on the device (SD_BATCH_GRAPH)."""
    from paper_2108_13229_gb300 import inputs as I
    wls = I.batch_instances(count, seed=seed, steps=steps)
    hs = []
    for wl in wls:
        o = sd.sd_options_default()
        hs.append(sd.sd_create(wl.n, wl.mu, wl.K(), wl.alpha, wl.dt, o))
    flags = (sd.SD_BATCH_LOCKSTEP if lockstep else 0) | (sd.SD_BATCH_GRAPH if graph else 0)
    sd.sd_solve_batch_ex(hs, [3] * count, max_threads=threads, flags=flags)  # warm-up (graph captures)
    l0 = sd.sd_launch_count()
    t0 = time.perf_counter()
    infos = sd.sd_solve_batch_ex(hs, [steps] * count, max_threads=threads, flags=flags)
    el = time.perf_counter() - t0
    launches = sd.sd_launch_count() - l0
    dof = sum(wl.dof for wl in wls)
    its = [i["iters"] for inf in infos for i in inf]
    for h in hs:
        sd.sd_destroy(h)
    return {"value": dof * steps / el, "unit": UNIT, "instances": count, "steps_each": steps, "threads": threads,
            "mode": ("all groups' solves of a step in one graph launch, decided on the device" if graph else
                     "lockstep groups by grid size" if lockstep else "one stream and host thread per instance"),
            "seconds": el, "total_dof": dof, "grids": sorted(set(wl.n for wl in wls)), "gpu_launches": launches,
            "iters_per_step_mean": float(np.mean(its)), "max_relres": max(i["relres"] for inf in infos for i in inf)}


_SERVE_K = {}


def bench_serve(sd, rate: float, count: int, max_running: int, budget_gb: float = 120.0, seed: int = 0,
                lockstep: bool = False):
    """Poisson arrivals of time-dependent runs submitted to the continuous-batching server."""
    from paper_2108_13229_gb300 import inputs as I
    reqs = I.serving_requests(count, rate, seed=seed)
    # the rates share their draws of grid, length and K seed: draw each field once
    for _, wl in reqs:
        if (wl.n, wl.K_seed) not in _SERVE_K:
            _SERVE_K[(wl.n, wl.K_seed)] = wl.K()
    Ks = [_SERVE_K[(wl.n, wl.K_seed)] for _, wl in reqs]
    srv = sd.sd_server_create(int(budget_gb * (1 << 30)), max_running, lockstep=lockstep)
    t0 = time.perf_counter()
    tickets = []
    for (ta, wl), K in zip(reqs, Ks):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append((sd.sd_submit(srv, wl.n, wl.mu, K, wl.alpha, wl.dt, wl.steps), wl))
    sd.sd_server_drain(srv)
    el = time.perf_counter() - t0
    lat, work, its = [], 0, 0
    for tk, wl in tickets:
        rc, res, _ = sd.sd_poll(srv, tk)
        if rc != 0:
            raise RuntimeError("request failed: %d" % rc)
        lat.append(res["latency_ms"])
        work += res["dof"] * res["steps_done"]
        its += res["total_iters"]
    sd.sd_server_destroy(srv)
    return {"rate_per_s": rate, "requests": count, "max_running": max_running, "hbm_budget_gb": budget_gb,
            "mode": "lockstep size classes below 1M DoF" if lockstep else "one worker and stream per run",
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(np.mean(lat))},
            "value": work / el, "unit": UNIT, "makespan_s": el,
            "grids": [int(x) for x in np.percentile([wl.n for _, wl in reqs], [0, 50, 100])]}


def cpu_oracle_sample(n_sample: int, steps: int):
    """Time the oracle on a bounded sample: same physics on an n_sample grid."""
    import oracle as O
    from paper_2108_13229_gb300 import inputs as I
    K = I.lognormal_K(n_sample, -4.0, 1.0, 16.0, seed=0)
    t0 = time.perf_counter()
    o = O.Oracle(n_sample, 1e-3, 1.0, 0.05, K)
    o.factor()
    t1 = time.perf_counter()
    o.run(O.exact(n_sample, 0.0, 1e-3), 0.0, steps)
    t2 = time.perf_counter()
    dof = 4 * n_sample * n_sample + 2 * n_sample
    return {"value": dof * steps / (t2 - t0), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "same physics on %dx%d cells (%d DoF), %d steps; banded-LU factorisation %.2fs + steps %.2fs "
                      "on one host core; the %s grid is beyond the banded LU's memory" %
                      (n_sample, n_sample, dof, steps, t1 - t0, t2 - t1, "workload")}


def bench_reference(args, ws, rank):
    if rank != 0:
        return 0
    n_sample = 128
    import oracle as O
    from paper_2108_13229_gb300 import inputs as I
    K = I.lognormal_K(n_sample, -4.0, 1.0, 16.0, seed=0)
    o = O.Oracle(n_sample, 1e-3, 1.0, 0.05, K)
    tf0 = time.perf_counter()
    o.factor()
    tf = time.perf_counter() - tf0
    x = O.exact(n_sample, 0.0, 1e-3)
    x = o.run(x, 0.0, args.warmup)
    t0 = time.perf_counter()
    x = o.run(x, args.warmup * 0.05, args.steps)
    el = time.perf_counter() - t0
    dof = 4 * n_sample * n_sample + 2 * n_sample
    val = dof * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(args.n, args.steps),
                                            "sample_grid": n_sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: right-hand side + banded-LU triangular solves of the same "
                                       "physics on %dx%d cells (%d DoF), one host core; factorisation %.2fs "
                                       "outside the timed steps" % (n_sample, n_sample, dof, tf)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_ours(args, ws, rank, local):
    import torch
    from paper_2108_13229_gb300 import inputs as I
    from paper_2108_13229_gb300 import sd

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    n, steps, warmup = args.n, args.steps, args.warmup
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=rank)
    dof = 4 * n * n + 2 * n
    stream = torch.cuda.Stream()

    # headline: FP32 multigrid inside FP64 FGMRES, launch shape and hierarchy autotuned
    tuned, tune_info = tune_form(sd, n, K, sd.SD_MIXED, stream, not args.no_autotune)
    sampler = ClockSampler(local)
    sampler.start()
    ms, infos, launches, _ = run_form(sd, torch, n, K, sd.SD_MIXED, steps, warmup, stream, tuned=tuned)
    clocks = sampler.stop()
    units, secs = aggregate(dof * steps, ms / 1e3, ws)
    value = units / secs
    lat = [i["ms"] for i in infos]
    iters = [i["iters"] for i in infos]
    relres = max(i["relres"] for i in infos)

    fp64 = None
    if not args.quick:
        # FP64 throughout, same workload
        tuned64, tune64 = tune_form(sd, n, K, sd.SD_FP64, stream, not args.no_autotune)
        ms64, infos64, _, _ = run_form(sd, torch, n, K, sd.SD_FP64, steps, warmup, stream, tuned=tuned64)
        u64, s64 = aggregate(dof * steps, ms64 / 1e3, ws)
        lat64 = [i["ms"] for i in infos64]
        fp64 = {"value": u64 / s64, "ms_per_step": s64 * 1e3 / steps,
                "latency_ms": {"p50": float(np.percentile(lat64, 50)), "p99": float(np.percentile(lat64, 99))},
                "iters_per_step": [i["iters"] for i in infos64], "autotune": tune64}

    # the FP64 form's rate and the ratio come right after the headline value
    line = {"metric": METRIC, "value": value, "unit": UNIT,
            "fp64_value": fp64["value"] if fp64 else None,
            "mixed_over_fp64": value / fp64["value"] if fp64 else None,
            "n_gpus": ws, "steps": steps, "warmup": warmup,
            "ms_per_step": secs * 1e3 / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 outer / f32 multigrid", "data": "synthetic",
            "config": {"workload": workload_desc(n, steps), "n": n, "dof": dof, "precision": "mixed",
                       "parallelism": "replicas only" if ws > 1 else "single instance",
                       "l2": "working set %.1f GB per instance (sd_memory_estimate), larger than the 129 MB L2 "
                             "(no flush needed)" % (sd.sd_memory_estimate(n, sd.sd_options_default()) / 1e9)},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "iters_per_step": iters, "max_relres": relres, "gpu_launches": launches,
            "launches_per_step": launches / steps, "clocks": clocks}
    # the whole step against its compulsory HBM traffic
    hbm_peak, hbm_src = read_peaks()
    mbytes = sum(step_model_bytes(n, i, True, tuned.get("coarsest", 16)) for i in infos)
    gbs = mbytes / (ms / 1e3) / 1e9
    line["roofline_step"] = {"bound": "hbm", "bytes_per_step": mbytes / steps, "achieved": gbs, "peak": hbm_peak,
                             "unit": "GB/s", "frac": gbs / hbm_peak, "peak_source": hbm_src,
                             "model": "compulsory bytes of every kernel of the step (bench.py step_model_bytes) "
                                      "from each step's iterations, restarts and second Gram-Schmidt passes"}
    line["autotune"] = tune_info

    if not args.quick:
        line["fp64"] = fp64

        # roofline: each candidate kernel class is timed live (CUDA events around
        # every launch) during its own timed run; the largest share of the step
        # time is the dominant kernel
        cands = []
        for kid in (sd.SD_PROF_MUPDATE, sd.SD_PROF_APPLY, sd.SD_PROF_MDOT, sd.SD_PROF_CHEB_V):
            msk, _, _, prof = run_form(sd, torch, n, K, sd.SD_MIXED, steps, warmup, stream, prof_kernel=kid,
                                       tuned=tuned)
            if prof[1] > 0:  # the multi-dot runs only beyond four basis vectors
                cands.append(roofline_entry(kid, prof, msk))
        cands.sort(key=lambda e: -(e["share_of_step_time"] or 0.0))
        line["roofline"] = cands[0]
        line["roofline_kernels"] = cands[1:]

        # end to end through the public API with host buffers: create from host K,
        # then every step read the fields back into pinned host memory
        pinned = torch.empty(dof, dtype=torch.float64, pin_memory=True)
        Kh = torch.from_numpy(np.ascontiguousarray(K)).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        opts = sd.sd_options_default()
        for k, v in tuned.items():
            setattr(opts, k, v)
        h = sd.sd_create(n, 1e-3, Kh, 1.0, 0.05, opts)
        for _ in range(steps):
            sd.sd_step(h, 1)
            sd.sd_get_state(h, pinned)
        sd.sd_destroy(h)
        el = time.perf_counter() - t0
        ue, se = aggregate(dof * steps, el, ws)
        line["e2e"] = {"value": ue / se, "unit": UNIT, "h2d_bytes_per_step": n * n * 8 / steps,
                       "d2h_bytes_per_step": dof * 8,
                       "note": "setup (sd_create from host K, hierarchy, coarse inverses) inside the timed region"}

        # the other workloads: the mixed-precision 2048^2 case, the paper's
        # pressure-driven problem, the 256 batched instances and the serving
        # loop at three arrival rates
        line["c3_2048"] = bench_c3(sd, torch, stream, rank)
        line["paper_problem"] = bench_paper_problem(sd, torch, stream, rank)
        line["paper_problem_channel"] = bench_paper_problem(sd, torch, stream, rank, geometry=sd.SD_GEO_CHANNEL)
        line["paper_parameters"] = {"square_1024": bench_paper_parameters(sd, torch, stream, 1024, 0),
                                    "channel_256": bench_paper_parameters(sd, torch, stream, 256, 1)}
        line["batch"] = bench_batch(sd, 256, 10, 32, seed=rank)
        line["batch"]["per_instance_streams"] = bench_batch(sd, 256, 10, 32, seed=rank, lockstep=False)
        line["batch"]["one_graph_per_step"] = bench_batch(sd, 256, 10, 32, seed=rank, graph=True)
        line["serving"] = [bench_serve(sd, rate, 60, 16) for rate in (20.0, 100.0, 500.0)]

        if rank == 0 and ws >= 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_oracle_sample(args.cpu_n, 20)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def bench_c3(sd, torch, stream, rank: int, steps: int = 20):
    """The mixed-precision workload: 2048^2 cells per subdomain, 20 implicit-Euler steps from the initial state in
    each precision (setup outside the timed region), and the per-field difference of the two final states."""
    from paper_2108_13229_gb300 import inputs as I
    n = 2048
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=rank)
    dof = 4 * n * n + 2 * n
    out, xs = {}, {}
    for name, prec in (("mixed", sd.SD_MIXED), ("fp64", sd.SD_FP64)):
        ms, infos, launches, _ = run_form(sd, torch, n, K, prec, steps, 0, stream, keep_fields=xs, name=name)
        out[name] = {"value": dof * steps / (ms / 1e3), "ms_per_step": ms / steps,
                     "iters_per_step": [i["iters"] for i in infos], "max_relres": max(i["relres"] for i in infos),
                     "launches_per_step": launches / steps}
    err = {k: float(np.linalg.norm(xs["mixed"][k] - xs["fp64"][k]) / np.linalg.norm(xs["fp64"][k]))
           for k in xs["fp64"]}
    return {"workload": "lognormal 2048x2048 (%d DoF), mu=1e-3, alpha_BJ=1, dt=0.05, %d steps from the initial "
                        "state, rtol 1e-10, library defaults" % (dof, steps),
            "unit": UNIT, "mixed": out["mixed"], "fp64": out["fp64"],
            "mixed_over_fp64": out["mixed"]["value"] / out["fp64"]["value"], "rel_l2_mixed_vs_fp64": err}


def bench_paper_problem(sd, torch, stream, rank: int, n: int = 1024, steps: int = 25, geometry: int = 0):
    """The paper's pressure-driven problem (Sec. 5: half-cosine inflow pressure over t_end = 25 steps, traction
    sides, no slip on top, p = 0 at the porous-medium bottom) at 1024^2 on the log-normal workload's parameters;
    geometry 1: on the model problem's channel (free flow 3n x n, the interface the middle third of its floor)."""
    from paper_2108_13229_gb300 import inputs as I
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=rank)
    dof = sd.sd_dof_count_geometry(n, geometry)
    ms, infos, launches, _ = run_form(sd, torch, n, K, sd.SD_MIXED, steps, 0, stream,
                                      tuned={"bc": sd.SD_BC_PAPER, "geometry": geometry})
    lat = [i["ms"] for i in infos]
    where = ("%dx%d cells" % (n, n) if geometry == 0 else
             "channel: free flow %dx%d cells over %dx%d pm cells, interface the floor's middle third" % (3 * n, n, n, n))
    return {"workload": "pressure-driven problem (bc 2), %s (%d DoF), lognormal K, mu=1e-3, alpha_BJ=1, "
                        "dt=0.05, %d steps from rest (the whole inflow ramp), rtol 1e-10" % (where, dof, steps),
            "value": dof * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "iters_per_step": [i["iters"] for i in infos], "max_relres": max(i["relres"] for i in infos),
            "launches_per_step": launches / steps}


def bench_paper_parameters(sd, torch, stream, n: int, geometry: int, steps: int = 25):
    """The pressure-driven problem at the paper's own parameters (Sec. 5: K = 1e-6 constant, mu = 1e-3,
    alpha_BJ = 1, dt = 2e5, t_end = 50e5, amplitude 1e-9), 25 steps from rest, library defaults."""
    K = np.full((n, n), 1e-6)
    dof = sd.sd_dof_count_geometry(n, geometry)
    opts = sd.sd_options_default()
    opts.stream = stream.cuda_stream
    opts.bc, opts.bc_dp, opts.bc_tend, opts.geometry = sd.SD_BC_PAPER, 1e-9, 50e5, geometry
    h = sd.sd_create(n, 1e-3, K, 1.0, 2e5, opts)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0.record(stream)
        infos = sd.sd_step(h, steps, raise_on_error=False)
        ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    sd.sd_destroy(h)
    return {"workload": "%s, %d DoF, K = 1e-6, mu = 1e-3, alpha_BJ = 1, dt = 2e5, %d steps from rest" %
                        ("square %dx%d" % (n, n) if geometry == 0 else "channel %dx%d over %dx%d" % (3 * n, n, n, n),
                         dof, steps),
            "value": dof * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "iters_per_step": [i["iters"] for i in infos], "status": sorted({i["status"] for i in infos}),
            "max_relres": max(i["relres"] for i in infos)}


def bench_configs(sd, torch, steps_small: int = 10, steps_big: int = 5):
    """One JSON line per workload that is not the headline: the manufactured case (32^2, FP64, mu = K = alpha = 1,
    dt = 0.1, 10 steps) and the 2048^2 log-normal case in both precisions with the per-field difference of the
    mixed-precision solution from the FP64 one."""
    from paper_2108_13229_gb300 import inputs as I
    out = []
    # manufactured solution, FP64 throughout
    n = 32
    o = sd.sd_options_default()
    o.precision = sd.SD_FP64
    h = sd.sd_create(n, 1.0, np.ones(n * n), 1.0, 0.1, o)
    sd.sd_step(h, 3)
    infos = sd.sd_step(h, steps_small)
    lat = [i["ms"] for i in infos]
    dof = 4 * n * n + 2 * n
    out.append({"workload": "manufactured solution 32x32 (4160 DoF), FP64, mu=K=alpha=1, dt=0.1",
                "value": dof * len(lat) / (sum(lat) / 1e3), "unit": UNIT, "ms_per_step": float(np.mean(lat)),
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "iters_per_step": [i["iters"] for i in infos], "max_relres": max(i["relres"] for i in infos),
                "note": "L2-resident and launch-latency bound; parity with the oracle is in tests/"})
    sd.sd_destroy(h)
    # 2048^2: mixed vs FP64 from the same initial state
    n = 2048
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    dof = 4 * n * n + 2 * n
    res, xs = {}, {}
    for name, prec in (("mixed", sd.SD_MIXED), ("fp64", sd.SD_FP64)):
        o = sd.sd_options_default()
        o.precision = prec
        h = sd.sd_create(n, 1e-3, K, 1.0, 0.05, o)
        infos = sd.sd_step(h, steps_big)
        lat = [i["ms"] for i in infos[1:]]
        res[name] = {"value": dof * len(lat) / (sum(lat) / 1e3), "ms_per_step": float(np.mean(lat)),
                     "iters_per_step": [i["iters"] for i in infos], "max_relres": max(i["relres"] for i in infos)}
        xs[name] = sd.sd_get_fields(h)
        sd.sd_destroy(h)
    err = {k: float(np.linalg.norm(xs["mixed"][k] - xs["fp64"][k]) / np.linalg.norm(xs["fp64"][k]))
           for k in xs["fp64"]}
    out.append({"workload": "lognormal 2048x2048 (%d DoF), mu=1e-3, dt=0.05, %d steps from the initial state, "
                            "rtol 1e-10" % (dof, steps_big),
                "unit": UNIT, "mixed": res["mixed"], "fp64": res["fp64"],
                "mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"],
                "rel_l2_mixed_vs_fp64": err,
                "note": "first step excluded from the rates (unextrapolated start); both solves reach rtol 1e-10, "
                        "so the per-field difference is bounded by the conditioning times 1e-10"})
    # the partitioned coupling of Sec. 3 against the monolithic solve, same workload
    n = 1024
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    dof = 4 * n * n + 2 * n
    res, xs = {}, {}
    for name, coupling in (("monolithic", sd.SD_MONOLITHIC), ("partitioned", sd.SD_PARTITIONED)):
        o = sd.sd_options_default()
        o.coupling = coupling
        h = sd.sd_create(n, 1e-3, K, 1.0, 0.05, o)
        infos = sd.sd_step(h, 1 + steps_big)
        lat = [i["ms"] for i in infos[1:]]
        res[name] = {"value": dof * len(lat) / (sum(lat) / 1e3), "ms_per_step": float(np.mean(lat)),
                     "fgmres_iters_per_step": [i["iters"] for i in infos],
                     "coupling_iters_per_step": [i["coupling_iters"] for i in infos],
                     "max_relres": max(i["relres"] for i in infos)}
        xs[name] = sd.sd_get_fields(h)
        sd.sd_destroy(h)
    err = {k: float(np.linalg.norm(xs["partitioned"][k] - xs["monolithic"][k]) / np.linalg.norm(xs["monolithic"][k]))
           for k in xs["monolithic"]}
    out.append({"workload": "lognormal 1024x1024 (%d DoF), mu=1e-3, dt=0.05, mixed precision, %d steps after one "
                            "untimed" % (dof, steps_big),
                "unit": UNIT, "monolithic": res["monolithic"], "partitioned": res["partitioned"],
                "rel_l2_partitioned_vs_monolithic": err,
                "note": "partitioned: Darcy and free-flow subdomain FGMRES solves (coupling_rtol: 1e-12, three decades below coupling_eps) with IQN-ILS on the "
                        "interface velocity, coupling_eps 1e-9"})
    # the paper's pressure-driven problem (Sec. 5) on the square geometry: from rest, inflow pressure rising
    # as a half cosine over 25 steps
    n, steps = 1024, 25
    K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
    dof = 4 * n * n + 2 * n
    res = {}
    for name, coupling in (("monolithic", sd.SD_MONOLITHIC), ("partitioned", sd.SD_PARTITIONED)):
        o = sd.sd_options_default()
        o.bc = sd.SD_BC_PAPER
        o.coupling = coupling
        h = sd.sd_create(n, 1e-3, K, 1.0, 0.05, o)
        infos = sd.sd_step(h, steps)
        lat = [i["ms"] for i in infos[1:]]
        f = sd.sd_get_fields(h)
        res[name] = {"value": dof * len(lat) / (sum(lat) / 1e3), "ms_per_step": float(np.mean(lat)),
                     "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                     "fgmres_iters_per_step": [i["iters"] for i in infos],
                     "coupling_iters_per_step": [i["coupling_iters"] for i in infos],
                     "max_relres": max(i["relres"] for i in infos),
                     "inflow_flux": float(f["u"][:, 0].sum() / n), "outflow_flux": float(f["u"][:, n].sum() / n),
                     "flux_into_pm": float(-f["v"][0].sum() / n)}
        sd.sd_destroy(h)
    out.append({"workload": "pressure-driven problem of Sec. 5 on 1024x1024 cells per subdomain (%d DoF): inflow "
                            "pressure half-cosine 0 -> 1 over 25 steps, lognormal K, mu=1e-3, dt=0.05, mixed "
                            "precision, from rest" % dof,
                "unit": UNIT, "monolithic": res["monolithic"], "partitioned": res["partitioned"],
                "note": "first step excluded from the rates"})
    return out


def oracle_scan(sizes=(32, 64, 128, 256), steps: int = 5, resid_sizes=(1024, 2048)):
    """The oracle on one host core: banded-LU factorisation and per-step solves at small grids, and the CSR
    residual evaluator (assembly + one residual) at workload sizes the LU cannot hold."""
    import oracle as O
    from paper_2108_13229_gb300 import inputs as I
    rows = []
    for n in sizes:
        K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
        t0 = time.perf_counter()
        o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
        o.factor()
        t1 = time.perf_counter()
        o.run(O.exact(n, 0.0, 1e-3), 0.0, steps)
        t2 = time.perf_counter()
        dof = 4 * n * n + 2 * n
        rows.append({"n": n, "dof": dof, "factor_s": t1 - t0, "step_s": (t2 - t1) / steps,
                     "dof_steps_per_s_steps_only": dof * steps / (t2 - t1),
                     "dof_steps_per_s_with_factor": dof * steps / (t2 - t0)})
    for n in resid_sizes:
        K = I.lognormal_K(n, -4.0, 1.0, 16.0, seed=0)
        t0 = time.perf_counter()
        o = O.Oracle(n, 1e-3, 1.0, 0.05, K)
        x = O.exact(n, 0.0, 1e-3)
        b = o.rhs(x, 0.05)
        t1 = time.perf_counter()
        o.residual(x, b)
        t2 = time.perf_counter()
        rows.append({"n": n, "dof": 4 * n * n + 2 * n, "assemble_and_rhs_s": t1 - t0, "residual_s": t2 - t1,
                     "note": "banded LU infeasible (memory); residual evaluator only"})
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"metric": "oracle timing on one host core", "cpu": model, "arch": platform.machine(),
            "cores_used": 1, "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--cpu-n", type=int, default=128)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline form only")
    ap.add_argument("--no-autotune", action="store_true", help="library defaults instead of autotuned options")
    ap.add_argument("--mode", default="single", choices=["single", "batch", "serve", "configs", "oracle"])
    ap.add_argument("--count", type=int, default=256, help="batch instances / serving requests")
    ap.add_argument("--threads", type=int, default=32, help="host threads (batch) / running slots (serve)")
    ap.add_argument("--rates", type=float, nargs="*", default=[10.0, 20.0, 50.0, 100.0, 200.0, 500.0])
    args = ap.parse_args()
    if args.mode == "oracle":
        print(json.dumps(oracle_scan()), flush=True)
        return 0
    if args.mode == "configs":
        import torch
        from paper_2108_13229_gb300 import sd
        torch.cuda.set_device(dist_env()[2])
        for r in bench_configs(sd, torch):
            r["bench_mode"] = "configs"
            print(json.dumps(r), flush=True)
        return 0
    if args.mode in ("batch", "serve"):
        import torch
        from paper_2108_13229_gb300 import sd
        torch.cuda.set_device(dist_env()[2])
        if args.mode == "batch":
            for lockstep in (True, False):
                r = bench_batch(sd, args.count, args.steps if args.steps != 20 else 10, args.threads,
                                lockstep=lockstep)
                r.update({"metric": "batched coupled DOF*steps/s, independent instances of uneven grids",
                          "bench_mode": "batch"})
                print(json.dumps(r), flush=True)
        else:
            for rate in args.rates:
                for lockstep in (False, True):
                    r = bench_serve(sd, rate, args.count, args.threads, lockstep=lockstep)
                    r.update({"metric": "serving: p50/p99 request latency and DOF*steps/s under Poisson arrivals",
                              "bench_mode": "serve"})
                    print(json.dumps(r), flush=True)
        return 0
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        dist.barrier()
    try:
        if args.impl == "reference":
            return bench_reference(args, ws, rank)
        return bench_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
