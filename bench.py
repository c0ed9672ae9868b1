"""Benchmark: batched FP16 FFT GFLOP/s (5 N log2 N per transform) on GB300.

Default workload (the 1D sweep): N = 2^8, 2^10, ..., 2^24 with batch =
2^28 / N, so every exec moves 2^28 complex FP16 points (1 GiB in, 1 GiB
out).  One "step" runs the whole sweep: one tcfft_exec per size, inputs
already resident in HBM.  Inputs are larger than L2 (1 GiB per exec), so no
L2 flush is needed between execs.

Printed on rank 0 as ONE JSON line:
  value      -- whole-job GFLOP/s over all ranks (sum of 5 N log2N * batch
                over the step, divided by the step time, max over ranks)
  e2e        -- the same metric through tcfft_exec_host with pinned host
                buffers (host->device copy, exec, device->host copy timed)
  roofline   -- algorithmic HBM bytes (8 B per point per exec) / exec time
                of the pass kernel launches, against the measured copy peak
  cpu_baseline -- the FP64 CPU oracle on a bounded sample of the workload
  gpu_launches -- libtcfft kernel launches inside the timed region

--impl reference runs the FP64 CPU oracle (the reference for this method)
on the host cores instead, each step a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched FP16 FFT GFLOP/s (5NlogN) & %HBM peak at stated rel-err; serve p99 latency"
UNIT = "GFLOP/s"
POINTS = 1 << 28
SWEEP = [8, 10, 12, 14, 16, 18, 20, 22, 24]


def flops_1d(n: int, batch: int) -> float:
    return 5.0 * n * math.log2(n) * batch


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class _NvmlPoller:
    """Read-only NVML queries (SM clock, its maximum, power, clock-event
    reasons) every `period` seconds from a thread, as nvidia-smi CSV lines.
    NVML's poll rate keeps >= 10 samples inside a sub-second timed region,
    where nvidia-smi's 200 ms loop records one or two."""

    REASONS = ((0x8, "hw_slowdown"), (0x40, "hw_thermal_slowdown"), (0x20, "sw_thermal_slowdown"),
               (0x4, "sw_power_cap"))

    def __init__(self, gpu_index: int, period: float = 0.01):
        import ctypes
        import threading
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.gpu, self.period, self.lines = gpu_index, period, []
        self.stop_ev = threading.Event()
        self.th = threading.Thread(target=self._run, daemon=True)

    def _line(self):
        ct = self.ct
        sm, smax, mw, mask = ct.c_uint(), ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(sm)) != 0:  # NVML_CLOCK_SM
            return None
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(smax))
        self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(mw))
        self.reasons_fn(self.h, ct.byref(mask))
        flags = ["Active" if mask.value & bit else "Not Active" for bit, _ in self.REASONS]
        return ", ".join([str(self.gpu), str(sm.value), str(smax.value), f"{mw.value / 1000:.1f}",
                          hex(mask.value)] + flags)

    def _run(self):
        while not self.stop_ev.is_set():
            ln = self._line()
            if ln:
                self.lines.append(ln)
            self.stop_ev.wait(self.period)

    def start(self):
        self.th.start()

    def stop(self):
        self.stop_ev.set()
        self.th.join(timeout=2)
        return list(self.lines)


class ClockSampler:
    """Samples clocks and throttle reasons during the timed region: nvidia-smi
    (200 ms loop) plus NVML polling every 10 ms where libnvidia-ml loads."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        import tempfile
        self.gpu = gpu_index
        self.proc = None
        # raw samples: $TCFFT_CLOCKS_DIR/clocks_gpu<i>.csv when set, else a temporary file
        d = os.environ.get("TCFFT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_gpu{gpu_index}.csv")

    def start(self):
        self.nvml = None
        try:
            self.nvml = _NvmlPoller(self.gpu)
            self.nvml.start()
        except Exception:
            self.nvml = None
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        extra = self.nvml.stop() if getattr(self, "nvml", None) is not None else []
        if self.proc is None and not extra:
            return None
        lines = list(extra)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
            with open(self.path) as f:
                lines += f.readlines()
            if extra:  # keep the NVML samples beside nvidia-smi's
                with open(self.path, "a") as f:
                    f.write("\n".join(extra) + "\n")
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle
_ORACLE_INPUTS = {}


def oracle_sample(sizes, budget_points: int):
    """FP64 oracle on a bounded sample: per size, max(1, budget_points // n)
    transforms of the size's seeded input.  Returns (flops, seconds, threads, desc)."""
    import oracle
    import seeded_inputs as si
    oracle.build()
    threads = oracle.default_threads()
    total_flops, total_s = 0.0, 0.0
    parts = []
    for lg in sizes:
        n = 1 << lg
        b = max(1, budget_points // n)
        key = (lg, b)
        if key not in _ORACLE_INPUTS:
            _ORACLE_INPUTS[key] = si.as_complex128(si.half_input((b, n), seed=si.sweep_seed(lg)))
        x = _ORACLE_INPUTS[key]
        t0 = time.perf_counter()
        oracle.fft_batch(x, nthreads=threads)
        total_s += time.perf_counter() - t0
        total_flops += flops_1d(n, b)
        parts.append(f"2^{lg}x{b}")
    return total_flops, total_s, min(threads, os.cpu_count() or 1), " ".join(parts)


def oracle_sample_2d(sides):
    """FP64 oracle, one 2D transform per side; returns (flops, seconds, threads, desc)."""
    import oracle
    import seeded_inputs as si
    oracle.build()
    threads = oracle.default_threads()
    flops, secs, parts = 0.0, 0.0, []
    for side in sides:
        key = ("2d", side)
        if key not in _ORACLE_INPUTS:
            _ORACLE_INPUTS[key] = si.as_complex128(si.half_input((side, side), seed=si.seed_2d(side.bit_length() - 1)))
        x = _ORACLE_INPUTS[key]
        t0 = time.perf_counter()
        oracle.fft_2d(x, nthreads=threads)
        secs += time.perf_counter() - t0
        flops += 5.0 * side * side * math.log2(side * side)
        parts.append(f"{side}x{side}x1")
    return flops, secs, min(threads, os.cpu_count() or 1), " ".join(parts)


def oracle_sample_shapes(shapes):
    """FP64 oracle on a list of 1D (n,) / 2D (nx, ny) shapes; (flops, seconds, threads, desc)."""
    import numpy as np
    import oracle
    import seeded_inputs as si
    oracle.build()
    threads = oracle.default_threads()
    flops, secs = 0.0, 0.0
    for i, sh in enumerate(shapes):
        x = si.as_complex128(si.half_input(tuple(sh), seed=4000 + i))
        t0 = time.perf_counter()
        if len(sh) == 1:
            oracle.fft_batch(x[None, :], nthreads=threads)
        else:
            oracle.fft_2d(x, nthreads=threads)
        secs += time.perf_counter() - t0
        flops += 5.0 * np.prod(sh) * math.log2(np.prod(sh))
    return flops, secs, min(threads, os.cpu_count() or 1), f"first {len(shapes)} transforms of the ragged list"


# ------------------------------------------------------------------ dist
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ arms
def run_reference(args, world, rank):
    """The FP64 CPU oracle as it stands, on the host cores; one bounded sample per step."""
    if rank != 0:
        return
    budget = args.cpu_sample_points
    if args.workload == "2d":
        sides = [int(x) for x in args.sizes.split(",")] if args.sizes else [256, 512, 1024, 4096, 8192]
        sample = lambda: oracle_sample_2d(sides)
        wl = f"2d: sides {sides}, batch=2^{args.log2_points}/side^2, FP16 uniform[-1,1] inputs"
        sdesc = "FP64 CPU oracle, one transform per side"
    else:
        sizes = [int(x) for x in args.sizes.split(",")] if args.sizes else SWEEP
        sample = lambda: oracle_sample(sizes, budget)
        wl = f"1d_sweep: N=2^8..2^24 step 2^2, batch=2^{args.log2_points}/N, FP16 uniform[-1,1] inputs"
        sdesc = f"FP64 CPU oracle, per size max(1, {budget}//N) transforms"
    flops, secs, cores, desc = 0.0, 0.0, 1, ""
    if args.warmup:
        sample()  # untimed: builds the oracle, draws the inputs
    for _ in range(args.steps):
        f, s, cores, desc = sample()
        flops += f
        secs += s
    value = flops / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl, "sample": sdesc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class Entry:
    """One exec per step: a plan with its device buffers and accounting."""

    def __init__(self, label, plan, x, y, flops, alg_bytes, check):
        self.label, self.plan, self.x, self.y = label, plan, x, y
        self.flops, self.alg_bytes, self.check = flops, alg_bytes, check


def _half_draw(n_values: int, seed: int):
    """n_values FP16 numbers uniform in [-1, 1] (re/im interleaved when used as complex)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n_values).astype(np.float16)


def _split_draw(n_values: int, seed: int):
    """(hi, lo) FP16 planes of an FP64 uniform[-1, 1] draw: lo = fp16((v - hi) * 2^11)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, size=n_values)
    hi = v.astype(np.float16)
    lo = ((v - hi.astype(np.float64)) * 2048.0).astype(np.float16)
    return hi, lo


DTYPES = {"fp16": "f16", "split": "f16 split (hi+lo, 3 products)", "fp32": "f32 io, f16 split (3 products)"}


def _fast_uniform(n_values: int, seed: int, dtype):
    """n_values numbers uniform in [-1, 1) from a seeded FP32 draw, cast to dtype."""
    import numpy as np
    rng = np.random.default_rng(seed)
    v = rng.random(n_values, dtype=np.float32)
    v *= 2.0
    v -= 1.0
    return v.astype(dtype)


def build_sweep(args, dev, rank):
    """The 1D sweep: one exec per N = 2^8..2^24 over 2^28-point buffers, each
    size with its own seeded input (seed 1000 + log2 N, plus 100 per rank),
    in plain FP16 (the benchmark), split FP16 or FP32 in and out."""
    import numpy as np
    import torch
    import paper_2104_11471_gb300 as tc
    import seeded_inputs as si
    sizes = [int(s) for s in args.sizes.split(",")] if args.sizes else SWEEP
    prec = args.precision
    if prec == "fp32":
        code, bpp, label = tc.TCFFT_FP32, 16.0, "FP32 complex in and out (split FP16 tensor-core stages)"
    elif prec == "split":
        code, bpp, label = tc.TCFFT_FP16_SPLIT, 16.0, "split FP16 (hi + 2^-11 lo planes)"
    else:
        code, bpp, label = tc.TCFFT_FP16, 8.0, "plain FP16"
    y = None
    entries = []
    host = (None, None)
    for lg in sizes:
        n = 1 << lg
        b = POINTS // n
        seed = si.sweep_seed(lg) + 100 * rank
        lo = None
        if prec == "fp32":
            h = _fast_uniform(2 * POINTS, seed, np.float32)
            x = torch.from_numpy(h).to(dev)
        elif prec == "split":
            v = _fast_uniform(2 * POINTS, seed, np.float64)
            h = v.astype(np.float16)
            lo = ((v - h.astype(np.float64)) * 2048.0).astype(np.float16)
            del v
            x = torch.from_numpy(np.concatenate([h, lo]).view(np.uint16)).to(dev)
        else:
            h = _fast_uniform(2 * POINTS, seed, np.float16)
            x = torch.from_numpy(h.view(np.uint16)).to(dev)
        if y is None:
            y = torch.empty_like(x)
        host = (h, lo)
        plan = tc.Plan.plan_1d(n, b, code, 0 if args.no_autotune else tc.TCFFT_PLAN_AUTOTUNE)
        row = b // 2  # one transform from the middle of the batch
        sl = slice(row * 2 * n, (row + 1) * 2 * n)
        xin = h[sl].astype(np.float64)
        if prec == "split":
            xin = xin + lo[sl].astype(np.float64) / 2048.0

        def check(orc, y=y, n=n, sl=sl, xin=xin):
            if prec == "fp32":
                out = y[sl].cpu().numpy().astype(np.float64)
            else:
                out = y[sl].cpu().numpy().view(np.float16).astype(np.float64)
            if prec == "split":
                out = out + y[2 * POINTS:][sl].cpu().numpy().view(np.float16).astype(np.float64) / 2048.0
            ref = orc.fft_batch((xin[0::2] + 1j * xin[1::2])[None, :])[0]
            return orc.rel_l2(out[0::2] + 1j * out[1::2], ref)

        entries.append(Entry(f"1d n={n} batch={b}", plan, x, y, flops_1d(n, b), bpp * n * b, check))
    cfg = {"workload": f"1d_sweep: N=2^8..2^24 step 2^2, batch=2^{args.log2_points}/N, "
                       "one exec per size per step, uniform[-1,1] inputs seeded per size (1000 + log2 N)",
           "sizes": [1 << s for s in sizes], "points_per_exec": POINTS, "precision": label,
           "geometry": "fixed planner" if args.no_autotune else "plan-time autotuner (not timed)",
           "l2": "inputs larger than L2 (1 GiB per exec), no flush"}
    cpu_sizes = [(1 << s,) for s in sizes]
    return entries, cfg, cpu_sizes, host


def build_2d(args, dev, rank):
    """Batched 2D: sides 256, 512, 1024, 4096, 8192, batch = 2^28 / side^2, plain and split."""
    import numpy as np
    import torch
    import paper_2104_11471_gb300 as tc
    sides = [int(s) for s in args.sizes.split(",")] if args.sizes else [256, 512, 1024, 4096, 8192]
    hi, lo = _split_draw(2 * POINTS, 2000 + rank)
    planes = np.concatenate([hi, lo])
    x = torch.from_numpy(planes.view(np.uint16)).to(dev)
    y = torch.empty_like(x)
    entries = []
    for split in (False, True):
        for side in sides:
            b = POINTS // (side * side)
            prec = tc.TCFFT_FP16_SPLIT if split else tc.TCFFT_FP16
            plan = tc.Plan.plan_2d(side, side, b, prec, 0 if args.no_autotune else tc.TCFFT_PLAN_AUTOTUNE)
            xs = x if split else x[:2 * POINTS]
            ys = y if split else y[:2 * POINTS]

            def check(orc, y=y, side=side, b=b, split=split):
                m = side * side
                row = b // 2
                sl = slice(row * 2 * m, (row + 1) * 2 * m)
                xin = hi[sl].astype(np.float64)
                o_hi = y[sl].cpu().numpy().view(np.float16).astype(np.float64)
                if split:
                    xin = xin + lo[sl].astype(np.float64) / 2048.0
                    o_lo = y[2 * POINTS:][sl].cpu().numpy().view(np.float16).astype(np.float64)
                    o_hi = o_hi + o_lo / 2048.0
                z = (xin[0::2] + 1j * xin[1::2]).reshape(side, side)
                ref = orc.fft_2d(z)
                got = (o_hi[0::2] + 1j * o_hi[1::2]).reshape(side, side)
                return orc.rel_l2(got, ref)
            entries.append(Entry(f"2d {side}x{side} batch={b} {'split' if split else 'plain'}", plan, xs, ys,
                                 5.0 * side * side * math.log2(side * side) * b,
                                 (16.0 if split else 8.0) * side * side * b, check))
    cfg = {"workload": f"2d: sides {sides}, batch=2^{args.log2_points}/side^2, plain FP16 and split FP16 "
                       "(hi + 2^-11 lo), one exec per (side, precision) per step, uniform[-1,1] seeded inputs",
           "points_per_exec": POINTS, "precision": "plain and split FP16",
           "geometry": "fixed planner" if args.no_autotune else "plan-time autotuner (not timed)",
           "l2": "inputs larger than L2 (1-2 GiB per exec), no flush"}
    cpu_sizes = [(s, s) for s in sides]
    return entries, cfg, cpu_sizes, (hi, lo)


def ragged_shapes(seed: int = 4):
    """The ragged workload: 4096 1D transforms, N = 2^k with k uniform in 8..16
    (log-uniform N), plus 256 2D transforms with side uniform in
    {128, 256, 512, 1024}; shuffled into one packed buffer."""
    import numpy as np
    rng = np.random.default_rng(seed)
    shapes = [(1 << int(k),) for k in rng.integers(8, 17, size=4096)]
    shapes += [(int(s), int(s)) for s in rng.choice([128, 256, 512, 1024], size=256)]
    return [shapes[i] for i in rng.permutation(len(shapes))]


def build_ragged(args, dev, rank):
    """One tcfft_plan_many plan over the ragged workload, replayed as one graph
    launch per step (autotuned geometry); the same plan run with one launch per
    pass is timed beside it."""
    import numpy as np
    import torch
    import paper_2104_11471_gb300 as tc
    shapes = ragged_shapes(4 + rank)
    pts = sum(int(np.prod(sh)) for sh in shapes)
    h = _half_draw(2 * pts, 4 + rank)
    x = torch.from_numpy(h.view(np.uint16)).to(dev)
    y = torch.empty_like(x)
    tune = 0 if args.no_autotune else tc.TCFFT_PLAN_AUTOTUNE
    persistent = args.ragged_mode == "persistent"
    flags = tc.TCFFT_PLAN_PERSISTENT if persistent else (tc.TCFFT_PLAN_GRAPH | tune)
    plan = tc.Plan.plan_many(shapes, tc.TCFFT_FP16, flags)
    flops = sum(5.0 * np.prod(sh) * math.log2(np.prod(sh)) for sh in shapes)
    offs = np.concatenate([[0], np.cumsum([int(np.prod(sh)) for sh in shapes])])

    def check(orc, y=y):
        worst = 0.0
        picks = [i for i, sh in enumerate(shapes) if len(sh) == 2][:2] + \
                [i for i, sh in enumerate(shapes) if len(sh) == 1][:6]
        for i in picks:
            a, b = offs[i], offs[i + 1]
            xin = h[2 * a:2 * b].astype(np.float64)
            out = y[2 * a:2 * b].cpu().numpy().view(np.float16).astype(np.float64)
            z = (xin[0::2] + 1j * xin[1::2]).reshape(shapes[i])
            g = (out[0::2] + 1j * out[1::2]).reshape(shapes[i])
            ref = orc.fft_batch(z) if len(shapes[i]) == 1 else orc.fft_2d(z)
            worst = max(worst, orc.rel_l2(g, ref))
        return worst
    how = "one persistent work-queue launch" if persistent else "one graph launch"
    entries = [Entry(f"ragged {len(shapes)} transforms, {how}", plan, x, y, flops, 8.0 * pts, check)]
    cfg = {"workload": "ragged: 4096 1D transforms N=2^k, k~U{8..16}, + 256 2D transforms side~U{128,256,512,1024}, "
                       "shuffled into one packed buffer, one tcfft_plan_many plan per step: "
                       + ("one persistent launch claiming (pass, chunk) items from a device work queue"
                          if persistent else "replayed as one CUDA graph launch, geometry from the plan-time "
                          "autotuner") + "; uniform[-1,1] seeded inputs",
           "transforms": len(shapes), "points_per_exec": pts, "precision": "plain FP16",
           "l2": f"inputs {pts * 4 / 2**20:.0f} MiB per exec (> L2), no flush"}

    def per_size_launches(steps, stream):
        """The same shapes with one launch per pass (no graph), and with the
        other of the graph / persistent-queue modes."""
        out = {}
        modes = [("per_pass", tune), ("graph" if persistent else "persistent",
                                       (tc.TCFFT_PLAN_GRAPH | tune) if persistent else tc.TCFFT_PLAN_PERSISTENT)]
        for name, fl in modes:
            p2 = tc.Plan.plan_many(shapes, tc.TCFFT_FP16, fl)
            for _ in range(2):
                p2.exec(x, y, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                p2.exec(x, y, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            out[name] = {"ms_per_step": round(ms, 4), "gflops": round(flops / (ms / 1e3) / 1e9, 1),
                         "launches_per_step": p2.num_launches}
            p2.destroy()
        return out
    cpu_sizes = [sh for sh in shapes[:64]]
    return entries, cfg, cpu_sizes, (h, None), per_size_launches


def run_serve(args, world, rank, local):
    """The serving stream: Poisson arrivals at 2000/s for 10 s, batches of 1-64
    transforms, 1D N = 2^8..2^20 or 2D side 2^6..2^11, plain/split 50/50,
    under a 16 GB HBM budget; continuous batching over 4 streams."""
    import torch
    import paper_2104_11471_gb300 as tc
    from paper_2104_11471_gb300.serve import FFTServer, poisson_trace
    tc.build()
    torch.cuda.set_device(local)
    srv = FFTServer(hbm_budget=16 << 30, slots=4)
    # warm-up trace (untimed): same mix, shorter
    warm = poisson_trace(rate=2000.0, seconds=0.5 * max(1, args.warmup) / 3, seed=105 + rank)
    reqs = poisson_trace(rate=2000.0, seconds=args.serve_seconds, seed=5 + rank)
    srv.assign_inputs(warm, seed=106)
    srv.assign_inputs(reqs, seed=6 + rank)
    srv.prewarm(warm + reqs)
    srv.run(warm)
    clk = ClockSampler(local)
    barrier(world)
    clk.start()
    st = srv.run(reqs)
    clocks = clk.stop()
    srv.close()
    span = max_over_ranks(st["span_s"], world)
    flops = sum(r.flops for r in reqs)
    value = world * flops / span / 1e9
    peak, peak_kind = peaks()
    alg = sum(8.0 * r.points * (2 if r.split else 1) for r in reqs)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(reqs),
        "warmup": len(warm), "ms_per_step": span / len(reqs) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": f"serve: Poisson 2000 req/s for {args.serve_seconds:g} s, batch U{{1..64}}, "
                               "50% 1D N=2^k k~U{8..20}, 50% 2D side 2^k k~U{6..11}, plain/split 50/50, "
                               "16 GB HBM budget, continuous batching on 4 streams; step = one request",
                   "parallelism": f"replicas x{world}"},
        "serve": {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                  "requests": st["requests"], "batches": st["batches"], "peak_hbm_bytes": st["peak_hbm_bytes"],
                  "device_peak_bytes": st.get("device_peak_bytes"), "resident_bytes": st.get("resident_bytes"),
                  "budget_bytes": st.get("budget_bytes"), "plan_evictions": st.get("plan_evictions"),
                  "plain": st.get("plain"), "split": st.get("split"),
                  "by_size": {k: st[k] for k in ("small_points", "medium_points", "large_points") if k in st}},
        "roofline": {"bound": "hbm", "achieved": round(alg / span / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(alg / span / 1e9 / peak, 4), "traffic": None,
                     "kernel": "pass_kernel (offered load, not saturating)", "peak_kind": peak_kind},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_latency(args, world, rank, local):
    """Small-batch latency: one large transform (or a few) at a time, inputs
    resident; per configuration the median over repeated execs of the device
    time (CUDA events around tcfft_exec) and of the host time (tcfft_exec plus
    a stream synchronize), with per-pass launches and with one graph launch."""
    import numpy as np
    import torch
    import paper_2104_11471_gb300 as tc
    tc.build()
    torch.cuda.set_device(local)
    reps = max(50, args.steps)
    configs = [(16, 1), (16, 4), (20, 1), (20, 4), (24, 1), (24, 4)]
    if args.sizes:
        keep = {int(v) for v in args.sizes.split(",")}
        configs = [c for c in configs if c[0] in keep]
    s = torch.cuda.current_stream()
    out, tot_flops, tot_s = [], 0.0, 0.0
    clk = ClockSampler(local)
    barrier(world)
    clk.start()
    launches = 0
    for lg, batch in configs:
        n = 1 << lg
        x = torch.from_numpy(_half_draw(2 * n * batch, 3000 + lg).view(np.uint16)).to(f"cuda:{local}")
        y = torch.empty_like(x)
        row = {"n": n, "batch": batch}
        for name, flags in (("launches", 0), ("graph", tc.TCFFT_PLAN_GRAPH)):
            plan = tc.Plan.plan_1d(n, batch, tc.TCFFT_FP16, flags)
            for _ in range(5):
                plan.exec(x, y, s)
            torch.cuda.synchronize()
            dev, host = [], []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                e0.record(s)
                plan.exec(x, y, s)
                e1.record(s)
                s.synchronize()
                host.append(time.perf_counter() - t0)
                dev.append(e0.elapsed_time(e1) * 1e-3)
            launches += reps * plan.num_launches
            row[name] = {"device_us": round(float(np.median(dev)) * 1e6, 2),
                         "host_us": round(float(np.median(host)) * 1e6, 2),
                         "passes": plan.num_launches}
            if name == "graph":
                tot_flops += flops_1d(n, batch)
                tot_s += float(np.median(dev))
            plan.destroy()
        out.append(row)
    clocks = clk.stop()
    value = world * tot_flops / tot_s / 1e9
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": reps,
        "warmup": 5, "ms_per_step": tot_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16", "data": "synthetic",
        "config": {"workload": "latency: 1D N = 2^16, 2^20, 2^24 at batch 1 and 4, one exec at a time, "
                               "inputs resident; value = flops over the sum of median graph-launch device times",
                   "parallelism": f"replicas x{world}"},
        "latency": out,
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2104_11471_gb300 as tc

    # one rank compiles (if the library is out of date), the others then load it
    if local == 0:
        tc.build()
    barrier(world)
    tc.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build = {"sweep1d": build_sweep, "2d": build_2d, "ragged": build_ragged}[args.workload]
    built = build(args, dev, rank)
    entries, cfg, cpu_sizes, host = built[:4]
    aux = built[4] if len(built) > 4 else None
    stream = torch.cuda.current_stream()
    launches_per_step = sum(e.plan.num_launches for e in entries)

    def step(events=None):
        for i, e in enumerate(entries):
            if events is not None:
                events[i][0].record(stream)
            e.plan.exec(e.x, e.y, stream)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for e in entries:
        st = e.plan.last_error()
        if st != 0:
            raise RuntimeError(f"device status {st} in warm-up ({e.label})")

    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in entries] for _ in range(args.steps)]
    t_start, t_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    t_start.record(stream)
    for k in range(args.steps):
        step(ev[k])
    t_stop.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    barrier(world)
    elapsed_ms = t_start.elapsed_time(t_stop)
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    flops_step = sum(e.flops for e in entries)
    value = world * flops_step * args.steps / (elapsed_ms / 1e3) / 1e9
    for e in entries:
        st = e.plan.last_error()
        if st != 0:
            raise RuntimeError(f"device status {st} in timed region ({e.label})")

    peak, peak_kind = peaks()
    per = []
    tot_bytes, tot_ms = 0.0, 0.0
    for i, e in enumerate(entries):
        ms = [ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps)]
        avg = sum(ms) / len(ms)
        tot_bytes += e.alg_bytes
        tot_ms += avg
        gbs = e.alg_bytes / (avg / 1e3) / 1e9
        per.append({"exec": e.label, "launches": e.plan.num_launches, "ms": round(avg, 4),
                    "gflops": round(e.flops / (avg / 1e3) / 1e9, 1), "alg_gbs": round(gbs, 1),
                    "frac": round(gbs / peak, 4),
                    "passes": [{k: d[k] for k in ("log2n", "mode", "per_cta", "grid", "async_load", "ctas_per_sm", "threads")}
                               for d in e.plan.describe()]})
    achieved = tot_bytes / (tot_ms / 1e3) / 1e9

    compare = aux(args.steps, stream) if aux else None

    # end to end: pinned host buffers through tcfft_exec_host
    e2e = None
    if not args.no_e2e:
        hin = torch.from_numpy(np.concatenate([p for p in host if p is not None]).view(np.uint16)).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        for e in entries:
            e.plan.exec_host(hin, hout, stream)  # warm-up (allocates the plan's device buffers)
        barrier(world)
        t0 = time.perf_counter()
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            for e in entries:
                e.plan.exec_host(hin, hout, stream)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        io = sum(e.plan.io_bytes for e in entries)
        e2e = {"value": world * flops_step * e2e_steps / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": io, "d2h_bytes_per_step": io}

    # CPU oracle leg (the FP64 oracle on the host cores): the accuracy of the
    # timed outputs (one sampled transform per exec, recomputed on the host)
    # and the CPU baseline
    if not args.no_check:
        import oracle
        for i, e in enumerate(entries):
            e.plan.exec(e.x, e.y, stream)
            torch.cuda.synchronize()
            per[i]["rel_l2"] = float(f"{e.check(oracle):.3e}")
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        if args.workload == "sweep1d":
            f, s_, cores, desc = oracle_sample([int(math.log2(c[0])) for c in cpu_sizes], args.cpu_sample_points)
        elif args.workload == "2d":
            f, s_, cores, desc = oracle_sample_2d([c[0] for c in cpu_sizes])
        else:
            f, s_, cores, desc = oracle_sample_shapes(cpu_sizes)
        cpu = {"value": f / s_ / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    traffic = None
    suffix = "" if args.precision == "fp16" else f"_{args.precision}"
    tpath = os.path.join(ROOT, "profiles", f"traffic_{args.workload}{suffix}.json")
    if os.path.exists(tpath):
        try:
            with open(tpath) as f:
                td = json.load(f)
            if td.get("kernel_hash") == kernel_hash():
                traffic = td.get("traffic_bytes_per_step")
        except Exception:
            traffic = None
    for e in entries:
        e.plan.destroy()
    if rank != 0:
        return
    cfg["parallelism"] = f"replicas x{world}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision] if args.workload == "sweep1d" else "f16", "data": "synthetic",
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": "pass_kernel (all launches of the step; unit = one exec, 8 B/point plain, "
                               "16 B/point split)",
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "per_exec": per,
    }
    if compare is not None:
        line["per_size_launches"] = compare
    print(json.dumps(line), flush=True)


def write_traffic(args):
    """Per-step DRAM traffic from an ncu CSV log (one warm-up and one timed
    step, pass_kernel launches only), scaled from the captured points per exec
    to the benchmark's; stored with the kernel-source hash it belongs to."""
    import csv
    by_id = {}
    with open(args.write_traffic) as f:
        rows = [r for r in csv.reader(line for line in f if line.startswith('"'))]
    hdr = rows[0]
    ki, mi, vi, ii = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "ID"))
    for r in rows[1:]:
        if "pass_kernel" not in r[ki] or r[mi] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        by_id[int(r[ii])] = by_id.get(int(r[ii]), 0.0) + float(r[vi].replace(",", ""))
    ids = sorted(by_id)
    if not ids or len(ids) % 2:
        raise SystemExit(f"expected the launches of two steps, found {len(ids)}")
    step = ids[len(ids) // 2:]
    measured = sum(by_id[i] for i in step)
    scale = 2 ** (28 - args.log2_points)
    out = {"kernel_hash": kernel_hash(), "traffic_bytes_per_step": int(measured * scale),
           "measured_bytes_per_step_at_2^%d_points" % args.log2_points: int(measured), "scale": scale,
           "launches_per_step": len(step),
           "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum over the pass_kernel launches of the "
                   "timed step, scaled to 2^28 points per exec (every launch reads and writes its data "
                   "once, so traffic grows in proportion)"}
    suffix = "" if args.precision == "fp16" else f"_{args.precision}"
    path = os.path.join(ROOT, "profiles", f"traffic_{args.workload}{suffix}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


def kernel_hash() -> str:
    """Hash of the kernel sources, so stored ncu traffic is dropped once they change."""
    import hashlib
    hsh = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2104_11471_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, name), "rb") as f:
                hsh.update(f.read())
    return hsh.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tcfft", choices=["tcfft", "reference"])
    ap.add_argument("--sizes", default="", help="comma-separated log2 sizes (default: the sweep)")
    ap.add_argument("--cpu-sample-points", type=int, default=1 << 21)
    ap.add_argument("--log2-points", type=int, default=28,
                    help="points per exec (smaller values for profiling captures only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the sampled oracle check of the outputs")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--workload", default="sweep1d", choices=["sweep1d", "2d", "ragged", "serve", "latency"],
                    help="sweep1d: the 1D sweep (default); 2d: batched 2D plain and split; "
                         "ragged: mixed sizes in one graph launch; serve: the request stream; "
                         "latency: single large transforms")
    ap.add_argument("--precision", default="fp16", choices=["fp16", "split", "fp32"],
                    help="sweep1d: plain FP16 (the benchmark), split FP16, or FP32 in and out")
    ap.add_argument("--ragged-mode", default="graph", choices=["graph", "persistent"],
                    help="ragged workload: one CUDA graph launch (default; the persistent work-queue launch is "
                         "timed beside it) or one persistent work-queue launch")
    ap.add_argument("--no-autotune", action="store_true",
                    help="plan with the fixed geometry heuristics instead of the plan-time autotuner")
    ap.add_argument("--write-traffic", default="", metavar="CSV",
                    help="write profiles/traffic_<workload>.json from an ncu --csv log of "
                         "dram__bytes_read.sum and dram__bytes_write.sum over pass_kernel launches of "
                         "this command run with --steps 1 --warmup 1 (the second step is kept)")
    args = ap.parse_args()
    if args.write_traffic:
        write_traffic(args)
        return
    global POINTS
    POINTS = 1 << args.log2_points
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    elif args.workload == "latency":
        run_latency(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
