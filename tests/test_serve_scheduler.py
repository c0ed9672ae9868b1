"""The serving scheduler's host logic on CPU: FFTServer.run with a simulated
executor (a job "completes" after a time proportional to its points).
Checks continuous batching, the small/large stream pools, FIFO order within
a pool, HBM-budget admission and the statistics, without a GPU."""
import time
from types import SimpleNamespace

import pytest

from paper_2104_11471_gb300.serve import FFTServer, Request, _Job, poisson_trace


class _SimEvent:
    """Completes at time `t`; counts the job off its stream when first seen done."""

    def __init__(self, t, on_done):
        self.t, self.on_done, self.seen = t, on_done, False

    def query(self):
        done = time.perf_counter() >= self.t
        if done and not self.seen:
            self.seen = True
            self.on_done()
        return done


class SimServer(FFTServer):
    """FFTServer whose launches are simulated: no device, no plans."""

    def __init__(self, hbm_budget, slots=2, small_slots=2, depth=2, job_points=1 << 22,
                 small_points=1 << 18, ns_per_point=0.05):
        self.torch = SimpleNamespace(cuda=SimpleNamespace(synchronize=lambda: None))
        self.budget = hbm_budget
        self.slots = [None] * (slots + small_slots)
        self.n_large = slots
        self.small_points = small_points
        self.share_sm = True
        self.depth = depth
        self.job_points = job_points
        self.plans = {}
        self.plan_bytes, self.plan_cap, self.plan_used, self.plan_jobs = {}, {}, {}, {}
        self.evictions = 0
        self.pool_bytes = 0
        self.in_use = 0
        self.peak_in_use = 0
        self.peak_plan_bytes = 0
        self.footprints = []  # pool + plans + batches in flight, at every launch
        self.ns = ns_per_point
        self.log = []  # (launch time, stream, key, request ids, points)
        self.busy = [0] * len(self.slots)
        self.max_busy = [0] * len(self.slots)

    def _create_plan(self, shape, split, cap):
        return None, self.plan_estimate(shape, split, cap)  # no device: the estimate stands in

    def _launch(self, group, key, sidx):
        m = 1
        for d in key[0]:
            m *= d
        pts = sum(r.batch for r in group) * m
        planes = 2 if key[1] else 1
        self.footprints.append(self.resident_bytes() + self.in_use + 8 * planes * pts)
        self.log.append((time.perf_counter(), sidx, key, [r.rid for r in group], pts))
        self.busy[sidx] += 1
        self.max_busy[sidx] = max(self.max_busy[sidx], self.busy[sidx])

        def done():
            self.busy[sidx] -= 1
        ev = _SimEvent(time.perf_counter() + pts * self.ns * 1e-9 + 2e-4, done)
        return _Job(group, key, sidx, ev, 8 * planes * pts)


def _trace(seconds=0.3, rate=400.0, seed=3):
    return poisson_trace(rate=rate, seconds=seconds, seed=seed, max_batch=64, k1d=(8, 14), k2d=(6, 9))


def test_every_request_completes_after_it_arrives():
    srv = SimServer(hbm_budget=1 << 34)
    reqs = _trace()
    st = srv.run(reqs, time_limit=30.0)
    assert st["requests"] == len(reqs) and st["batches"] <= len(reqs)
    assert all(r.t_done >= r.t_arrival for r in reqs)
    assert st["p50_ms"] <= st["p99_ms"]
    # every request ran exactly once
    ran = sorted(rid for _, _, _, ids, _ in srv.log for rid in ids)
    assert ran == sorted(r.rid for r in reqs)


def test_pools_depth_and_merging():
    srv = SimServer(hbm_budget=1 << 34)
    reqs = _trace(seed=4)
    srv.run(reqs, time_limit=30.0)
    by_id = {r.rid: r for r in reqs}
    for _, sidx, key, ids, pts in srv.log:
        # a job is one (shape, precision) and at most the plan's capacity
        assert all((by_id[i].shape, by_id[i].split) == key for i in ids)
        assert sum(by_id[i].batch for i in ids) <= srv.capacity(key[0], key[1])
        # large jobs never take the small jobs' streams
        if pts > srv.small_points:
            assert sidx < srv.n_large
    assert max(srv.max_busy) <= srv.depth


def test_fifo_within_a_pool():
    # requests of one shape and pool start in arrival order
    srv = SimServer(hbm_budget=1 << 34)
    reqs = _trace(seed=5)
    srv.run(reqs, time_limit=30.0)
    first_start = {}
    for t, _, _, ids, _ in srv.log:
        for i in ids:
            first_start[i] = t
    for key in {(r.shape, r.split) for r in reqs}:
        same = sorted((r for r in reqs if (r.shape, r.split) == key), key=lambda r: r.t_arrival)
        starts = [first_start[r.rid] for r in same]
        assert starts == sorted(starts)


def test_admission_respects_the_budget():
    budget = 1 << 27  # 128 MiB: large jobs must wait for memory
    srv = SimServer(hbm_budget=budget, job_points=1 << 22)
    reqs = [Request(i, 0.001 * i, (4096,), 64, bool(i % 2)) for i in range(24)]
    srv.run(reqs, time_limit=30.0)
    assert 0 < srv.peak_in_use <= budget
    assert srv.in_use == 0


def test_request_larger_than_the_budget_is_refused():
    srv = SimServer(hbm_budget=1 << 20)
    with pytest.raises(RuntimeError, match="HBM budget"):
        srv.run([Request(0, 0.0, (1 << 14,), 64, True)], time_limit=10.0)


def test_admission_counts_plans_and_pool_and_evicts_idle_plans():
    # multi-pass 1D shapes whose plans hold a workspace: with the pool and the
    # batches in flight they do not all fit, so idle plans are evicted (LRU)
    # and the footprint at every launch stays within the budget
    budget = 96 << 20
    srv = SimServer(hbm_budget=budget, job_points=1 << 20)
    srv.pool_bytes = 16 << 20
    reqs = [Request(i, 0.0005 * i, (1 << (15 + i % 4),), 4, bool((i // 4) % 2)) for i in range(48)]
    st = srv.run(reqs, time_limit=30.0)
    assert st["requests"] == len(reqs) and all(r.t_done > 0 for r in reqs)
    assert srv.evictions > 0 and st["plan_evictions"] == srv.evictions
    assert max(srv.footprints) <= budget
    assert 0 < srv.peak_in_use <= budget and srv.in_use == 0
    assert st["resident_bytes"] == srv.resident_bytes() >= srv.pool_bytes


def test_new_plan_shrinks_to_fit_the_budget():
    # a plan whose default capacity cannot fit is made for fewer transforms
    budget = 16 << 20  # the default 64-transform plan needs 16 MiB of workspace + tables
    srv = SimServer(hbm_budget=budget, job_points=1 << 22)
    reqs = [Request(i, 0.001 * i, (1 << 16,), 2, False) for i in range(6)]
    st = srv.run(reqs, time_limit=30.0)
    assert st["requests"] == 6
    assert srv.plan_cap[((1 << 16,), False)] < max(64, (1 << 22) >> 16)
    assert max(srv.footprints) <= budget
