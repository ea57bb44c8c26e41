#!/usr/bin/env python
"""Benchmark of the micropolar elastoplastic FFT solver on one GB300.

Workload: the 256^3 periodic Voronoi cell with 200 seeded grains (per-grain
moduli and yield stresses +-20 % around the matrix values), uniaxial E11 to
1 % in 20 load increments, tolerance 1e-6 (local error measure), FP32 fields
and FFTs with the radial return's scalar solve, the error norms and the
homogenized averages in FP64.  One bench "step" is one load increment of that
path: predictor, fixed-point iterations to convergence, commit (every step of
the hot path).  The metric is voxel-iterations per second:
sum over timed increments of (voxels x fixed-point iterations) / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica on its own GPU ("replicas
only": one cell does not shard), the timed region is bracketed by a barrier and
cudaDeviceSynchronize, and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-iters/s at 256^3 and batched RVE solves/s vs plain FP64; serving p50/p99"
UNIT = "voxel-iters/s"
FALLBACK_HBM_GBS = 6800.0
KERNEL_CLASSES = ("fft_y_fwd", "green_z", "fft_y_inv", "pass_a", "reduce", "start", "commit", "spectral")


# ---------------------------------------------------------------- algorithmic bytes

def algorithmic_bytes(n, precision=1):
    """Bytes one launch of each iteration kernel must move (inputs + outputs),
    for an N1 x N2 x N3 cell: the half spectrum holds 18 complex values per
    (N1 / 2) N2 N3 points; pass A also reads the history record (h_t, h_m,
    phase id: 20 reals) and p, q (2 doubles), and reads + writes the previous
    iterate (e, gamma, f_t, f_m: 20 reals)."""
    r = 8 if precision == 0 else 4
    nvox = n[0] * n[1] * n[2]
    nspec = max(n[0] // 2, 1) * n[1] * n[2]
    spec = nspec * 18 * 2 * r
    return {
        "fft_y_fwd": 2 * spec,
        "green_z": 2 * spec,
        "fft_y_inv": 2 * spec,
        "spectral": 2 * spec,
        "pass_a": 2 * spec + nvox * (2 * 20 * r + 20 * r + 16),
    }


# Host-only sources (entry points, the batched engine's host loop, the static
# entry point, host helpers): a change there leaves the kernels' DRAM traffic
# as it was, so they do not enter the hash that dates a traffic capture.
HOST_ONLY_SOURCES = ("mp_api.cu", "mp_batch.cu", "mp_static.cu", "mp_host.cuh")


def _source_hash():
    """Hash of the device-code sources (kernels and the headers they use)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2409_10774_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in HOST_ONLY_SOURCES:
            continue
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload="voronoi200-256^3"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources for this workload."""
    path = os.path.join(ROOT, "profiles", "traffic_voronoi256.txt")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    if data.get("source_hash") != _source_hash() or data.get("workload") != workload:
        return None
    return data.get("bytes_per_launch", {}).get(kernel)


def _peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for _, _, flags in rows:
            for nm, f in zip(names, flags):
                if f.lower().startswith("active"):
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(r[0] for r in rows), sm_max_mhz=max(r[1] for r in rows),
                   reasons=sorted(reasons), samples=len(rows))
        return out


# ---------------------------------------------------------------- oracle legs (CPU)

ORACLE_N = 64  # the 64^3 regeneration of the 256^3 Voronoi cell (same seeds / 4)


def oracle_sample(budget_s=15.0, max_iters=None, warmup_iters=1):
    """Times the FP64 oracle's fixed-point iterations of the first load
    increment of the 64^3 regeneration of the Voronoi workload; returns
    (voxel-iters/s, iterations timed, seconds)."""
    import numpy as np  # noqa: F401
    import workloads as W
    from oracle import solver

    prob = W.workload_voronoi(n=ORACLE_N)
    nvox = ORACLE_N ** 3
    stamps = []

    class _Stop(Exception):
        pass

    def t_start():
        return stamps[warmup_iters - 1] if warmup_iters >= 1 else start

    def cb(step, it, err):
        stamps.append(time.perf_counter())
        timed = len(stamps) - warmup_iters
        if timed <= 0:
            return
        if max_iters is not None and timed >= max_iters:
            raise _Stop()
        if max_iters is None and stamps[-1] - t_start() > budget_s:
            raise _Stop()

    start = time.perf_counter()
    try:
        solver.solve(prob, callback=cb)
    except _Stop:
        pass
    iters = len(stamps) - warmup_iters
    if iters <= 0:
        raise RuntimeError("oracle sample ended before the timed iterations")
    secs = stamps[-1] - t_start()
    return nvox * iters / secs, iters, secs


def _oracle_subprocess(args):
    """Run an oracle leg in a fresh single-threaded process (spawned before any
    CUDA use in this process)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "r = bench.oracle_sample(**%r); print(json.dumps(r))" % (ROOT, args))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=900)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_block():
    value, iters, secs = _oracle_subprocess({"budget_s": 15.0})
    return {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 numpy oracle, {iters} fixed-point iterations ({secs:.1f} s) of the first "
                      f"load increment of the {ORACLE_N}^3 regeneration of the Voronoi cell "
                      f"(same seeds scaled by 1/4), after 1 untimed iteration"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    value, iters, secs = _oracle_subprocess({"max_iters": args.steps, "warmup_iters": args.warmup})
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(iters, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"each step = one FP64 oracle fixed-point iteration of the first "
                                       f"load increment of the {ORACLE_N}^3 regeneration of the Voronoi "
                                       f"cell; {args.warmup} untimed, {iters} timed"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU leg

def combine_ranks(ms, voxel_iters, world):
    """Whole-job figures of the replicas: the slowest rank's time and the
    voxel-iterations of all ranks (every rank calls this; process group
    already initialised when world > 1)."""
    if world <= 1:
        return float(ms), float(voxel_iters)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = torch.tensor([float(voxel_iters)], dtype=torch.float64)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(t[0]), float(tot[0])


def _shape(args):
    return tuple(int(v) for v in args.shape.split(",")) if args.shape else None


def _config(args):
    shape = _shape(args)
    name = f"voronoi{args.cells}-" + ("x".join(map(str, shape)) if shape else f"{args.n}^3")
    return {"workload": name, "n": list(shape) if shape else args.n, "cells": args.cells,
            "increments": 20, "load": "E11 to 1%", "tol": 1e-6, "err": "local",
            "ref_medium": "mean", "fields": "fp32", "scalars": "fp64 scalar return, p, q, error sums; averages in compensated fp32 pairs folded in fp64",
            "l2": "no flush: the cell's device state (~5.3 GB) exceeds L2",
            "parallelism": f"replicas x{args.gpus}"}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    cpu_block = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_block = cpu_baseline_block()  # before the first CUDA call of this process

    import paper_2409_10774_gb300 as M
    import workloads as W

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    prob = W.workload_voronoi(n=args.n, n_cells=args.cells, shape=_shape(args))
    n = prob["n"]
    nvox = n[0] * n[1] * n[2]
    n_steps = len(prob["time"]) - 1
    ctx = M.Context(local_rank)

    # ---------------- device-resident timed run (value)
    def timed_run(precision, profile, steps, warmup):
        """K load increments of the path (wrapping around its 20 increments)
        after W untimed ones, timed with CUDA events on the run's stream.
        profile: per-kernel CUDA events (the host then decides each
        fixed-point loop); otherwise the loop is decided on the device (one
        graph launch per increment).  Returns (iterations, ms, per-kernel
        profile, clocks)."""
        rve = M.Rve(ctx, prob, precision=precision, stream=stream)

        def advance(k):
            # iterations counted per increment: a reset zeroes the cell's total
            done, its = 0, 0
            while done < k:
                if rve.steps_done >= n_steps:
                    rve.reset(stream=stream)  # wrap around the 20-increment path
                before = rve.iterations
                st = rve.run(1, stream=stream)
                if st != 0:
                    raise RuntimeError(f"increment failed: {M.binding.last_error(ctx.ptr)}")
                its += rve.iterations - before
                done += 1
            return its

        advance(warmup)
        torch.cuda.synchronize(dev)
        rve.profile(profile)
        rve.profile_read(reset=True)
        sampler = ClockSampler(local_rank)
        sampler.start()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        its = advance(steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        clk = sampler.stop()
        prof_ = rve.profile_read(reset=True)
        if its <= 0 or prof_["pass_a"][1] != its:
            raise RuntimeError(f"timed iteration count {its} disagrees with the pass-A launches "
                               f"{prof_['pass_a'][1]}")
        rve.profile(False)
        rve.close()
        return its, ev0.elapsed_time(ev1), prof_, clk

    iters, ms, prof, clocks = timed_run(1, True, args.steps, args.warmup)
    # the same increments with the loop decided on the device, and with the
    # level return in FP32 (precision 2), for comparison
    extra = {}
    if not args.no_variants:
        for key, prec, prf in (("device_loop", 1, False), ("fp32_return", 2, True)):
            it_v, ms_v, _, clk_v = timed_run(prec, prf, args.steps, args.warmup)
            extra[key] = {"value": it_v * nvox / (ms_v / 1e3), "unit": UNIT, "ms_per_step": ms_v / args.steps,
                          "iterations_timed": it_v, "precision": prec,
                          "loop": "host, per-kernel events" if prf else "device (graph WHILE node)",
                          "clocks": clk_v}

    ms_max, vox_it = combine_ranks(ms, float(iters) * nvox, world)
    value = vox_it / (ms_max / 1e3)

    # ---------------- roofline of the dominant kernel (events on the run's stream)
    abytes = algorithmic_bytes(n, precision=1)
    timed = {k: prof[k] for k in abytes if prof[k][1] > 0}
    dom = max(timed, key=lambda k: timed[k][0])
    dom_ms = timed[dom][0] / timed[dom][1]
    achieved = abytes[dom] / (dom_ms / 1e3) / 1e9
    peak, peak_src = _peaks()
    kernels = {k: {"ms_per_launch": prof[k][0] / prof[k][1] if prof[k][1] else None,
                   "launches": prof[k][1],
                   "gbs": (abytes[k] / (prof[k][0] / prof[k][1] / 1e3) / 1e9)
                   if (k in abytes and prof[k][1] and prof[k][0] > 0) else None}
               for k in KERNEL_CLASSES}
    launches = int(sum(v[1] for v in prof.values()))

    # ---------------- plain FP64 GPU solver on the same workload (speed-up base)
    fp64 = None
    if not args.no_fp64:
        r64 = M.Rve(ctx, prob, precision=0, stream=stream)
        r64.run(args.warmup, stream=stream)
        torch.cuda.synchronize(dev)
        i0 = r64.iterations
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k64 = max(1, min(args.steps, args.fp64_steps))
        e0.record(stream)
        r64.run(k64, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        v64 = (r64.iterations - i0) * nvox / (e0.elapsed_time(e1) / 1e3)
        res64 = r64.results(fields=False, stream=stream)
        r64.close()
        fp64 = {"value": v64, "unit": UNIT, "increments": k64,
                "note": f"plain FP64 GPU solver, increments {args.warmup + 1}..{args.warmup + k64}"}

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(nvox, dtype=torch.int16, pin_memory=True)
        pin_np = pinned.numpy().view(np.uint16)
        pin_np[:] = prob["phase"].reshape(-1)
        prob_pinned = dict(prob, phase=pin_np)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = M.Rve(ctx, prob_pinned, precision=1, stream=stream)     # H2D: phase map, tables, path
        k_e2e = min(args.steps, n_steps)
        r.run(k_e2e, stream=stream)
        res = r.results(fields=False, stream=stream)                  # D2H: homogenized results
        res32 = res
        iters_e2e = r.iterations
        r.close()
        torch.cuda.synchronize(dev)
        secs = time.perf_counter() - t0
        h2d = nvox * 2 + len(prob["phases"]) * 104 + (n_steps + 1) * 19 * 8
        d2h = k_e2e * (40 * 8) + iters_e2e * 5 * 8
        e2e = {"value": iters_e2e * nvox / secs, "unit": UNIT, "h2d_bytes_per_step": h2d // k_e2e,
               "d2h_bytes_per_step": d2h // k_e2e,
               "note": f"Rve create (uploads) + {k_e2e} increments from the zero state + results + destroy; "
                       f"T11 after increment {k_e2e}: {res['T'][-1][0, 0]:.6e}"}

    # ---------------- FP32-mixed error against the plain FP64 GPU solver, per result
    fp32_err = None
    if fp64 is not None and e2e is not None:
        k = min(res64["steps_done"], res32["steps_done"])

        def rel(key, partner=None):
            a, b = np.asarray(res32[key][:k]), np.asarray(res64[key][:k])
            d = np.abs(a - b).reshape(k, -1).max(axis=1)
            sc = np.abs(b).reshape(k, -1).max(axis=1)
            return [float(x) for x in d / np.maximum(sc, 1e-300)]

        fp32_err = {"increments": list(range(1, k + 1)),
                    "note": "relative difference of the FP32-mixed results (same cell, same load path, "
                            "from the zero state) to the plain FP64 GPU solver's, per increment; "
                            "the FP32 fields against the FP64 oracle are checked by the -m gpu tests",
                    **{f"{key}_rel": rel(key) for key in ("T", "Eavg", "P", "Teq")}}
        fp32_err["max_T_rel"] = max(fp32_err["T_rel"])

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(args),
        "iterations_timed": iters,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": _traffic(dom, _config(args)["workload"]), "algorithmic_bytes_per_launch": abytes[dom]},
        "kernels": kernels,
        "fp64_gpu": fp64,
        "speedup_vs_fp64_gpu": (value / world / fp64["value"]) if fp64 else None,
        "fp32_vs_fp64_gpu": fp32_err,
        "variants": extra,
        "clocks": clocks,
        "cpu_baseline": cpu_block,
    }
    if not args.no_cufft:
        line["cufft"] = cufft_comparison(n)
        if kernels["spectral"]["launches"]:
            # the fused pass does both y transforms and the z pass in one launch
            line["cufft"]["ours_spectral_ms"] = kernels["spectral"]["ms_per_launch"]
            line["cufft"]["library_same_work_ms"] = (2 * line["cufft"]["y_one_direction_ms"]
                                                     + line["cufft"]["z_forward_inverse_ms"])
        else:
            line["cufft"]["ours_y_ms"] = kernels["fft_y_fwd"]["ms_per_launch"]
            line["cufft"]["ours_green_z_ms"] = kernels["green_z"]["ms_per_launch"]
    if world == 1 and not args.no_batch:
        line["batch"] = batch_measure(args)
    if world == 1 and not args.no_serve:
        line["serve"] = serve_measure(args)
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- library FFT comparison

def cufft_comparison(n, reps=10):
    """Timed comparison only (never on the product path): cuFFT (through
    torch.fft) on a spectrum of the solver's shape, complex64
    [N3][N2][N1/2][18], transformed along y (one direction) and along z
    (forward then inverse, the z pass's two transforms without the Green
    operator).  Each transform reads and writes the whole spectrum once."""
    import torch
    kx = max(n[0] // 2, 1)
    x = torch.randn((n[2], n[1], kx, 18), dtype=torch.complex64, device="cuda")
    nbytes = 2 * x.numel() * x.element_size()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    y_ms = timed(lambda: torch.fft.fft(x, dim=1))
    z_ms = timed(lambda: torch.fft.ifft(torch.fft.fft(x, dim=0), dim=0))
    out = {"library": "cuFFT via torch.fft " + torch.__version__, "layout": "complex64 [N3][N2][N1/2][18]",
           "y_one_direction_ms": y_ms, "y_gbs": nbytes / (y_ms / 1e3) / 1e9,
           "z_forward_inverse_ms": z_ms, "z_gbs": 2 * nbytes / (z_ms / 1e3) / 1e9,
           "note": "out-of-place library transforms with their own allocations; timed on the bench stream "
                   "after one untimed call"}
    del x
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- batched and served solves

def _percentile(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def batch_measure(args):
    """Batched dataset generation: `--batch-count` RVEs (default 512) of
    uneven size solved in one mp_batch_solve call (FP32 fields, tolerance
    1e-6), timed end to end (problem upload, all rounds, results download),
    beside the plain single-instance FP64 GPU solver at the same tolerance on
    the first `--fp64-sample` of the same RVEs, one after another."""
    import numpy as np
    import torch

    import paper_2409_10774_gb300 as M
    import workloads as W

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t_gen = time.perf_counter()
    probs = W.workload_batch(count=args.batch_count)
    t_gen = time.perf_counter() - t_gen
    ctx = M.Context(0)
    nvox = [int(np.prod(p["n"])) for p in probs]
    # warm-up: module load, allocator pools, the multi-cell kernels
    M.mp_batch_solve(ctx, probs[:16], precision=1, lockstep_iters=[[2] * 10] * 16, stream=stream)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()
    bstats = {}
    res = M.mp_batch_solve(ctx, probs, precision=1, stream=stream, stats=bstats)
    torch.cuda.synchronize(dev)
    secs = time.perf_counter() - t0
    clocks = sampler.stop()
    statuses = {}
    for r in res:
        statuses[r["status"]] = statuses.get(r["status"], 0) + 1
    vox_it = float(sum(nv * int(np.sum(r["iters"])) for nv, r in zip(nvox, res)))
    iters = np.array([int(np.sum(r["iters"])) for r in res])
    # plain single-instance FP64 solver on a sample of the same RVEs
    k = min(args.fp64_sample, len(probs))
    fp64 = None
    if k > 0:
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        vi64 = 0.0
        st64 = {}
        for p, nv in zip(probs[:k], nvox[:k]):
            r = M.mp_solve(ctx, p, precision=0, stream=stream)
            vi64 += nv * float(np.sum(r["iters"]))
            st64[r["status"]] = st64.get(r["status"], 0) + 1
        torch.cuda.synchronize(dev)
        s64 = time.perf_counter() - t1
        # the batch's own time for the same RVEs is not separable; compare rates
        fp64 = {"solves_per_s": k / s64, "voxel_iters_per_s": vi64 / s64, "sample": k,
                "seconds": s64, "statuses": st64}
    return {
        "leg": "batch", "metric": "batched RVE solves/s", "value": len(probs) / secs, "unit": "solves/s",
        "higher_is_better": True, "seconds": secs, "voxel_iters_per_s": vox_it / secs,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch{len(probs)}-N{{16,24,32,48}}", "rves": len(probs),
                   "voxels_total": int(sum(nvox)), "increments": 10, "tol": 1e-6, "err": "local",
                   "ref_medium": "midrange", "generation_s": t_gen},
        "statuses": statuses,
        "engine": bstats,
        "iterations_per_rve": {"p50": _percentile(iters, 50), "p90": _percentile(iters, 90),
                               "max": int(iters.max())},
        "fp64_single": fp64,
        "speedup_vs_fp64_single": (len(probs) / secs) / fp64["solves_per_s"] if fp64 else None,
        "clocks": clocks,
    }


def run_batch_leg(args):
    print(json.dumps(batch_measure(args)), flush=True)
    return 0


def serve_measure(args):
    """Serving: requests (RSA spheres, N in {32,64,96,128}, 5-20 increments,
    FP32, tolerance 1e-6) arrive as a Poisson process at each rate of
    `--rates`; each is submitted to one mp_server at its arrival time and
    waited for by its own thread; latency = result on the host - arrival.
    Baseline: the same requests one by one with the plain single-instance
    FP64 solver, queued FIFO at the same arrival times (their service times
    measured, the queue computed)."""
    import threading

    import numpy as np
    import torch

    import paper_2409_10774_gb300 as M
    import workloads as W

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = M.Context(0)
    n_req = args.requests
    t_gen = time.perf_counter()
    reqs = [W.workload_serving_request(i) for i in range(n_req)]
    t_gen = time.perf_counter() - t_gen
    # warm-up
    M.mp_batch_solve(ctx, reqs[:2], precision=1, lockstep_iters=[[1] * (len(r["time"]) - 1) for r in reqs[:2]])
    torch.cuda.synchronize(dev)
    rates = [float(x) for x in args.rates.split(",")]
    out = []
    for rate in rates:
        rng = np.random.Generator(np.random.PCG64(2409_10774 + int(rate * 1000)))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        done = [None] * n_req
        status = [None] * n_req
        srv = M.Server(ctx, budget_bytes=args.budget_gb << 30)
        t0 = time.perf_counter()
        threads = []

        def waiter(i, ticket):
            r = srv.wait(ticket)
            done[i] = time.perf_counter() - t0
            status[i] = r["status"]

        sampler = ClockSampler(0)
        sampler.start()
        for i in range(n_req):
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tk = srv.submit(reqs[i], precision=1)
            th = threading.Thread(target=waiter, args=(i, tk))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        clocks = sampler.stop()
        st = srv.stats()
        srv.close()
        lat = np.array(done) - arrivals
        span = max(done) - arrivals[0]
        out.append({"rate_per_s": rate, "p50_s": _percentile(lat, 50), "p99_s": _percentile(lat, 99),
                    "solves_per_s": n_req / span, "voxel_iters_per_s": st["voxel_iters"] / span,
                    "peak_resident": st["peak_resident"], "rounds": st["rounds"],
                    "statuses": {s_: status.count(s_) for s_ in set(status)}, "clocks": clocks})
    # baseline: plain FP64 single-instance solves, one by one
    service = []
    n_base = n_req if args.serve_fp64_sample < 0 else min(n_req, args.serve_fp64_sample)
    for r in reqs[:n_base]:
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        M.mp_solve(ctx, r, precision=0)
        torch.cuda.synchronize(dev)
        service.append(time.perf_counter() - t1)
    base = []
    if service:
        m = len(service)
        for rate in rates:
            rng = np.random.Generator(np.random.PCG64(2409_10774 + int(rate * 1000)))
            arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))[:m]
            free_at, lat = 0.0, []
            for a, sv in zip(arrivals, service):
                start = max(a, free_at)
                free_at = start + sv
                lat.append(free_at - a)
            base.append({"rate_per_s": rate, "p50_s": _percentile(lat, 50), "p99_s": _percentile(lat, 99),
                         "solves_per_s": m / (free_at - arrivals[0]), "requests": m})
    return {
        "leg": "serve", "metric": "serving p50/p99 latency and solves/s", "unit": "s",
        "higher_is_better": False, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "requests RSA spheres r=6 vf0.3, N in {32,64,96,128}, 5-20 increments",
                   "requests_per_rate": n_req, "tol": 1e-6, "budget_gb": args.budget_gb,
                   "generation_s": t_gen},
        "rates": out,
        "fp64_one_by_one": {"service_s": service, "queue": base},
    }


def run_serve_leg(args):
    print(json.dumps(serve_measure(args)), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--cells", type=int, default=200)
    ap.add_argument("--shape", default=None,
                    help="N1,N2,N3: the Voronoi cell on a box-shaped grid instead of n^3 (profiling cases)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--leg", choices=("single", "batch", "serve"), default="single",
                    help="single: the 256^3 cell (the bench line); batch / serve: the batched and "
                         "serving measurements")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--fp64-sample", type=int, default=16)
    ap.add_argument("--rates", default="0.25")
    ap.add_argument("--requests", type=int, default=6)
    ap.add_argument("--serve-fp64-sample", type=int, default=-1,
                    help="requests of the plain-FP64 one-by-one baseline (-1: all of them)")
    ap.add_argument("--no-cufft", action="store_true", help="leave the cuFFT timing out of the line")
    ap.add_argument("--no-variants", action="store_true",
                    help="leave out the device-loop and FP32-return repeats of the timed increments")
    ap.add_argument("--no-batch", action="store_true", help="leave the batch sub-object out of the line")
    ap.add_argument("--no-serve", action="store_true", help="leave the serving sub-object out of the line")
    ap.add_argument("--budget-gb", type=int, default=64)
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.leg == "batch":
        return run_batch_leg(args)
    if args.leg == "serve":
        return run_serve_leg(args)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("gloo")
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
