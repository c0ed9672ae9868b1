"""Continuous-batching FFT server on one GPU.

Requests (a batch of 1D or 2D transforms of one shape and precision) arrive
over time.  The server keeps one resident plan per (shape, precision), sized
for the largest merged batch, with its twiddle tables and workspace on the
device.  A scheduling loop on the host:

* admits arrived requests into a FIFO queue;
* whenever one of its CUDA streams (slots) has room, takes the oldest queued
  request plus every other queued request of the same shape and precision
  (up to the plan's capacity), reserves their input and output memory
  against the HBM budget, gathers their inputs into one contiguous batch
  (device-to-device copies) and runs the plan on that batch with
  tcfft_exec_batch -- so requests that arrive while others run on the GPU
  join the next batch and their work overlaps on the device;
* keeps small jobs (at most `small_points` points) off the queues of large
  ones: they run on their own high-priority streams, and every plan leaves
  half of each SM's CTA slots free (TCFFT_PLAN_SHARE_SM), so a small job
  does not wait for a large job's persistent grid to drain;
* retires finished batches (CUDA events), releasing their memory.

Admission counts everything the server holds on the device against the HBM
budget: the input pool, every resident plan's own memory (workspace, twiddle
tables, DFT-matrix images: tcfft_workspace_bytes) and the input and output
buffers of the batches in flight.  A request whose plan is not resident
brings the plan's estimated bytes with it.  When the total would pass the
budget the request waits until running batches free memory; only when the
resident set alone leaves no room are idle plans (no batch in flight)
destroyed, least recently used first (re-creating a plan synchronises the
device), and a new plan that still does not fit is made for fewer
transforms (its capacity halved down to the batch at hand).

Latency is arrival to completion as seen by the host.  All transform work
runs in libtcfft's kernels; this module only schedules, allocates and copies.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import TCFFT_FP16, TCFFT_FP16_SPLIT, TCFFT_PLAN_SHARE_SM, Plan


@dataclass
class Request:
    rid: int
    t_arrival: float          # seconds from the start of the trace
    shape: tuple              # (n,) or (nx, ny)
    batch: int
    split: bool
    pool_off: int = 0         # element offset of the input in the device pool
    t_done: float = -1.0
    out: object = None        # device tensor view of the result (kept on request)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape)) * self.batch

    @property
    def flops(self) -> float:
        m = int(np.prod(self.shape))
        return 5.0 * m * math.log2(m) * self.batch


@dataclass
class _Job:
    reqs: list
    key: tuple
    stream_idx: int
    event: object
    nbytes: int
    buffers: tuple = field(default=())


def poisson_trace(rate: float = 2000.0, seconds: float = 10.0, seed: int = 5, max_batch: int = 64,
                  k1d=(8, 20), k2d=(6, 11)):
    """The serving workload: Poisson arrivals; each request a batch of 1..64
    transforms, 50% 1D with N = 2^k (k uniform in k1d), 50% 2D with side 2^k
    (k uniform in k2d); precision plain / split 50/50."""
    rng = np.random.default_rng(seed)
    t, out, rid = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        b = int(rng.integers(1, max_batch + 1))
        if rng.random() < 0.5:
            shape = (1 << int(rng.integers(k1d[0], k1d[1] + 1)),)
        else:
            s = 1 << int(rng.integers(k2d[0], k2d[1] + 1))
            shape = (s, s)
        out.append(Request(rid, t, shape, b, bool(rng.random() < 0.5)))
        rid += 1
    return out


class FFTServer:
    def __init__(self, hbm_budget: int = 16 << 30, slots: int = 4, depth: int = 2,
                 job_points: int = 1 << 26, pool_points: int = 1 << 28, seed: int = 5,
                 small_slots: int = 3, small_points: int = 1 << 22, share_sm: bool = True):
        import torch
        self.torch = torch
        self.budget = hbm_budget
        # streams 0..slots-1 take large jobs; the high-priority rest small ones
        self.slots = [torch.cuda.Stream() for _ in range(slots)]
        self.n_large = slots
        hi_prio = torch.cuda.Stream.priority_range()[1] if hasattr(torch.cuda.Stream, "priority_range") else -1
        self.slots += [torch.cuda.Stream(priority=hi_prio) for _ in range(small_slots)]
        self.small_points = small_points
        self.share_sm = share_sm
        self.depth = depth                # batches in flight per stream
        self.job_points = job_points      # merge requests up to this many points
        self.plans = {}
        self.plan_bytes = {}   # key -> device bytes the plan holds (tcfft_workspace_bytes)
        self.plan_cap = {}     # key -> transforms per batch the plan was made for
        self.plan_used = {}    # key -> last launch (monotonic counter), for LRU eviction
        self.plan_jobs = {}    # key -> batches in flight
        self.evictions = 0
        self.in_use = 0
        self.peak_in_use = 0
        self.peak_plan_bytes = 0
        # seeded input pool on the device (hi plane, lo plane): requests read slices
        rng = np.random.default_rng(seed)
        v = rng.uniform(-1.0, 1.0, size=2 * pool_points)
        hi = v.astype(np.float16)
        lo = ((v - hi.astype(np.float64)) * 2048.0).astype(np.float16)
        self.pool_points = pool_points
        self.pool_hi = torch.from_numpy(hi.view(np.uint16)).cuda()
        self.pool_lo = torch.from_numpy(lo.view(np.uint16)).cuda()
        self.pool_host = (hi, lo)
        self.pool_bytes = 2 * self.pool_hi.numel() * self.pool_hi.element_size()

    # ---------------------------------------------------------------- plans
    def capacity(self, shape, split: bool = False) -> int:
        """Transforms per batch: the resident plan's, else the default
        (max(64, job_points / transform size))."""
        key = (tuple(shape), split)
        if key in self.plan_cap:
            return self.plan_cap[key]
        m = int(np.prod(shape))
        return max(64, self.job_points // m)

    def resident_bytes(self) -> int:
        """Device memory held between batches: input pool + resident plans."""
        return getattr(self, "pool_bytes", 0) + sum(self.plan_bytes.values())

    def plan_estimate(self, shape, split: bool, cap: int) -> int:
        """Device bytes a plan for `cap` transforms will hold: the multi-pass
        workspace (1D beyond 16384 points, 8192 in split precision; 2D
        columns beyond 2048 rows) plus a margin for its tables and images
        (well under 1 MiB up to 2^20 points)."""
        m = int(np.prod(shape))
        planes = 2 if split else 1
        multi = m > (8192 if split else 16384) if len(shape) == 1 else shape[0] > 2048
        return (cap * m * 4 * planes if multi else 0) + (1 << 20)

    def _create_plan(self, shape, split: bool, cap: int):
        prec = TCFFT_FP16_SPLIT if split else TCFFT_FP16
        flags = TCFFT_PLAN_SHARE_SM if self.share_sm else 0
        p = (Plan.plan_1d(shape[0], cap, prec, flags) if len(shape) == 1
             else Plan.plan_2d(shape[0], shape[1], cap, prec, flags))
        return p, p.workspace_bytes

    def _destroy_plan(self, key):
        p = self.plans.pop(key, None)
        if p is not None:
            p.destroy()
        self.plan_bytes.pop(key, None)
        self.plan_cap.pop(key, None)
        self.plan_used.pop(key, None)

    def _evict_idle(self, need: int, keep) -> None:
        """Destroys idle plans (no batch in flight), least recently used
        first, until `need` more bytes fit the budget beside what is in use."""
        idle = sorted((k for k in self.plan_bytes if k != keep and not self.plan_jobs.get(k)),
                      key=lambda k: self.plan_used.get(k, -1))
        for k in idle:
            if self.resident_bytes() + self.in_use + need <= self.budget:
                break
            self._destroy_plan(k)
            self.evictions += 1

    def ensure_plan(self, shape, split: bool, cap: int = 0):
        """The resident plan of (shape, precision), made for `cap` transforms
        (default capacity) if missing."""
        key = (tuple(shape), split)
        if key not in self.plan_bytes:
            cap = cap or self.capacity(shape, split)
            p, nbytes = self._create_plan(tuple(shape), split, cap)
            self.plans[key] = p
            self.plan_bytes[key] = nbytes
            self.plan_cap[key] = cap
            self.plan_used.setdefault(key, -1)
            self.peak_plan_bytes = max(self.peak_plan_bytes, sum(self.plan_bytes.values()))
        return self.plans.get(key)

    def plan(self, shape, split: bool) -> Plan:
        return self.ensure_plan(shape, split)

    def prewarm(self, requests):
        """Makes the plans of the trace's shapes while they fit in half the
        budget (the others are made when first needed)."""
        for key in sorted({(r.shape, r.split) for r in requests}):
            cap = self.capacity(*key)
            est = self.plan_estimate(key[0], key[1], cap)
            if self.resident_bytes() + est <= self.budget // 2:
                self.ensure_plan(key[0], key[1], cap)
        self.torch.cuda.synchronize()

    def _admit(self, key, head, queue, inflight):
        """Chooses the group for `key` (oldest request first) and the bytes it
        needs, evicting idle plans or shrinking a new plan so that pool +
        plans + batches in flight stay within the budget.  Returns (group,
        job bytes) or None when the group has to wait."""
        shape, split = key
        m = int(np.prod(shape))
        planes = 2 if split else 1
        resident = key in self.plan_bytes
        cap = self.capacity(shape, split)
        plan_need = 0
        if not resident:
            # a new plan: halve its capacity while it cannot fit beside the
            # head request (down to the head's own batch)
            head_bytes = 2 * planes * head.points * 4
            while True:
                plan_need = self.plan_estimate(shape, split, cap)
                room = self.budget - self.resident_bytes() - self.in_use
                if plan_need + head_bytes <= room or cap <= head.batch:
                    break
                cap = max(head.batch, cap // 2)
        group, total = [], 0
        for r in queue:
            if (r.shape, r.split) == key and total + r.batch <= cap:
                group.append(r)
                total += r.batch
        nbytes = 2 * planes * total * m * 4
        need = nbytes + plan_need
        if self.resident_bytes() + self.in_use + need > self.budget:
            # running batches free their memory soon: wait for them, unless
            # the resident set alone leaves no room (then evict idle plans;
            # re-creating an evicted plan synchronises the device)
            if self.resident_bytes() + need > self.budget:
                self._evict_idle(need - self.in_use, keep=key)
            if self.resident_bytes() + self.in_use + need > self.budget:
                if not inflight:
                    raise RuntimeError("request larger than the HBM budget")
                return None
        if not resident:
            self.ensure_plan(shape, split, cap)
        return group, nbytes

    def assign_inputs(self, requests, seed: int = 6):
        rng = np.random.default_rng(seed)
        for r in requests:
            if r.points > self.pool_points:
                raise ValueError("request larger than the input pool")
            r.pool_off = int(rng.integers(0, self.pool_points - r.points + 1)) & ~3  # 16-byte aligned

    # ---------------------------------------------------------------- loop
    def _launch(self, group, key, sidx):
        torch = self.torch
        shape, split = key
        m = int(np.prod(shape))
        total = sum(r.batch for r in group)
        pts = total * m
        planes = 2 if split else 1
        s = self.slots[sidx]
        with torch.cuda.stream(s):
            xin = torch.empty(planes * 2 * pts, dtype=torch.uint16, device="cuda")
            yout = torch.empty_like(xin)
            off = 0
            for r in group:  # gather the inputs into one contiguous batch
                n = 2 * r.points
                xin[2 * off:2 * off + n].copy_(self.pool_hi[2 * r.pool_off:2 * r.pool_off + n], non_blocking=True)
                if split:
                    xin[2 * pts + 2 * off:2 * pts + 2 * off + n].copy_(
                        self.pool_lo[2 * r.pool_off:2 * r.pool_off + n], non_blocking=True)
                off += r.points
            self.plan(shape, split).exec_batch(xin, yout, total, s)
            ev = torch.cuda.Event()
            ev.record(s)
        return _Job(group, key, sidx, ev, 2 * xin.numel() * 2, (xin, yout))

    def run(self, requests, keep_outputs: bool = False, time_limit: float = 600.0):
        """Serve the trace in real time; returns statistics."""
        torch = self.torch
        cuda = torch.cuda
        # measured footprint: torch's allocations (pool, batch buffers; minus
        # what the caller held before) plus the library's plan bytes, sampled
        # after every launch (the only place either grows)
        measure = hasattr(cuda, "memory_allocated")
        base = (cuda.memory_allocated() - getattr(self, "pool_bytes", 0)) if measure else 0
        device_peak = 0
        self.peak_plan_bytes = sum(self.plan_bytes.values())
        self.peak_in_use = self.resident_bytes()
        pending = deque(sorted(requests, key=lambda r: r.t_arrival))
        queue = deque()
        inflight = []
        per_slot = [0] * len(self.slots)
        batches = 0
        t0 = time.perf_counter()
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            if now > time_limit:
                raise RuntimeError("serving loop exceeded its time limit")
            while pending and pending[0].t_arrival <= now:
                queue.append(pending.popleft())
            for job in list(inflight):
                if job.event.query():
                    t = time.perf_counter() - t0
                    m = int(np.prod(job.key[0]))
                    off = 0
                    total = sum(r.batch for r in job.reqs)
                    for r in job.reqs:
                        r.t_done = t
                        if keep_outputs:
                            y = job.buffers[1]
                            planes = 2 if job.key[1] else 1
                            yv = y.view(planes, 2 * total * m)
                            r.out = yv[:, 2 * off:2 * (off + r.points)].clone()
                        off += r.points
                    self.in_use -= job.nbytes
                    per_slot[job.stream_idx] -= 1
                    self.plan_jobs[job.key] -= 1
                    job.buffers = ()  # release the batch buffers now, as counted
                    inflight.remove(job)
            job = None
            launched = False
            # start every job that has room: scan the queue in arrival order,
            # one group per (shape, precision); small and large jobs use their
            # own streams, and a pool that cannot start its oldest job stays
            # closed for this scan (arrival order within each pool)
            blocked = set()
            progressed = True
            while queue and progressed:
                progressed = False
                seen = set()
                for head in list(queue):
                    key = (head.shape, head.split)
                    if key in seen:
                        continue
                    seen.add(key)
                    cap = self.capacity(head.shape, head.split)
                    total = 0
                    for r in queue:
                        if (r.shape, r.split) == key and total + r.batch <= cap:
                            total += r.batch
                    pts = total * int(np.prod(head.shape))
                    pool = "small" if pts <= self.small_points else "large"
                    if pool in blocked:
                        continue
                    if pool == "small":
                        free = [i for i in range(self.n_large, len(self.slots)) if per_slot[i] < self.depth]
                        free = free or [i for i in range(self.n_large) if per_slot[i] == 0]
                    else:
                        free = [i for i in range(self.n_large) if per_slot[i] < self.depth]
                    if not free:
                        blocked.add(pool)
                        continue
                    admitted = self._admit(key, head, queue, inflight)
                    if admitted is None:
                        blocked.add(pool)  # admission: wait until running batches free memory
                        continue
                    group, nbytes = admitted
                    for r in group:
                        queue.remove(r)
                    sidx = min(free, key=lambda i: per_slot[i])
                    job = self._launch(group, key, sidx)
                    job.nbytes = nbytes
                    inflight.append(job)
                    per_slot[sidx] += 1
                    self.plan_jobs[key] = self.plan_jobs.get(key, 0) + 1
                    self.plan_used[key] = batches
                    self.in_use += nbytes
                    self.peak_in_use = max(self.peak_in_use, self.in_use + self.resident_bytes())
                    if measure:
                        device_peak = max(device_peak, cuda.memory_allocated() - base + sum(self.plan_bytes.values()))
                    batches += 1
                    launched = True
                    progressed = True
                    break  # the queue changed: scan again from its head
            if not launched and not (pending and pending[0].t_arrival <= time.perf_counter() - t0):
                time.sleep(20e-6)
        torch.cuda.synchronize()
        out = self.stats(requests, batches)
        if measure:
            out["device_peak_bytes"] = int(device_peak)
        return out

    def stats(self, requests, batches):
        lat = np.array([r.t_done - r.t_arrival for r in requests])
        span = max(r.t_done for r in requests) - min(r.t_arrival for r in requests)
        flops = sum(r.flops for r in requests)
        out = {"requests": len(requests), "batches": batches,
               "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
               "mean_ms": float(lat.mean() * 1e3), "gflops": flops / span / 1e9, "span_s": span,
               "peak_hbm_bytes": self.peak_in_use, "budget_bytes": self.budget,
               "resident_bytes": self.resident_bytes(), "plan_evictions": self.evictions}
        # by request size: small requests stuck behind large ones show here
        for name, lo, hi in (("small", 0, 1 << 20), ("medium", 1 << 20, 1 << 24), ("large", 1 << 24, 1 << 62)):
            sel = [r for r in requests if lo <= r.points < hi]
            if sel:
                la = np.array([r.t_done - r.t_arrival for r in sel])
                out[f"{name}_points"] = {"requests": len(sel), "p50_ms": float(np.percentile(la, 50) * 1e3),
                                         "p99_ms": float(np.percentile(la, 99) * 1e3)}
        for split in (False, True):
            sel = [r for r in requests if r.split == split]
            if sel:
                la = np.array([r.t_done - r.t_arrival for r in sel])
                out["split" if split else "plain"] = {
                    "requests": len(sel), "p50_ms": float(np.percentile(la, 50) * 1e3),
                    "p99_ms": float(np.percentile(la, 99) * 1e3),
                    "gflops": sum(r.flops for r in sel) / span / 1e9}
        return out

    def close(self):
        for k in list(self.plan_bytes):
            self._destroy_plan(k)
        self.plans.clear()
