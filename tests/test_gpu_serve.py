"""Serving loop: continuous batching over a Poisson request trace.

Requests of equal shape and precision that wait together are merged into one
batch; the test checks every result against the same request run alone
(bit-identical), spot-checks results against the FP64 oracle, and runs a
trace under a tight HBM budget to exercise admission."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from gpu_helpers import PLAIN_TOL, SPLIT_TOL, check_rows

pytestmark = pytest.mark.gpu


def _alone(server, r):
    import torch
    import paper_2104_11471_gb300 as tc
    prec = tc.TCFFT_FP16_SPLIT if r.split else tc.TCFFT_FP16
    plan = (tc.Plan.plan_1d(r.shape[0], r.batch, prec) if len(r.shape) == 1
            else tc.Plan.plan_2d(r.shape[0], r.shape[1], r.batch, prec))
    n = 2 * r.points
    x = server.pool_hi[2 * r.pool_off:2 * r.pool_off + n].clone()
    if r.split:
        x = torch.cat([x, server.pool_lo[2 * r.pool_off:2 * r.pool_off + n]])
    y = torch.empty_like(x)
    plan.exec(x, y)
    torch.cuda.synchronize()
    plan.destroy()
    return y.view(2 if r.split else 1, n)


def _trace():
    from paper_2104_11471_gb300.serve import poisson_trace
    return poisson_trace(rate=2000.0, seconds=0.2, seed=9, max_batch=8, k1d=(8, 15), k2d=(6, 8))


def test_each_result_same_alone_and_in_the_mix():
    from paper_2104_11471_gb300.serve import FFTServer
    reqs = _trace()
    srv = FFTServer(hbm_budget=4 << 30, slots=3, pool_points=1 << 22)
    srv.assign_inputs(reqs)
    srv.prewarm(reqs)
    st = srv.run(reqs, keep_outputs=True)
    assert st["requests"] == len(reqs) and all(r.t_done > 0 for r in reqs)
    assert st["batches"] < len(reqs), "no request was merged into a shared batch"
    for r in reqs:
        assert np.array_equal(r.out.cpu().numpy(), _alone(srv, r).cpu().numpy()), r
    # spot-check against the oracle
    hi, lo = srv.pool_host
    for r in reqs[:12]:
        m = int(np.prod(r.shape))
        a = 2 * r.pool_off
        xin = hi[a:a + 2 * r.points].astype(np.float64)
        got = r.out.cpu().numpy().view(np.float16).astype(np.float64)
        g = got[0]
        if r.split:
            xin = xin + lo[a:a + 2 * r.points].astype(np.float64) / 2048.0
            g = g + got[1] / 2048.0
        z = (xin[0::2] + 1j * xin[1::2]).reshape((r.batch,) + r.shape)
        gz = (g[0::2] + 1j * g[1::2]).reshape((r.batch,) + r.shape)
        ref = oracle.fft_batch(z) if len(r.shape) == 1 else oracle.fft_2d(z)
        tol = SPLIT_TOL if r.split else PLAIN_TOL
        check_rows(gz.reshape(r.batch, -1), ref.reshape(r.batch, -1), tol, f"served {r.shape} x{r.batch}")
    srv.close()


def test_admission_under_a_tight_budget():
    from paper_2104_11471_gb300.serve import FFTServer
    reqs = _trace()
    srv = FFTServer(hbm_budget=64 << 20, slots=2, pool_points=1 << 22)
    srv.assign_inputs(reqs)
    srv.prewarm(reqs)
    st = srv.run(reqs)
    assert st["requests"] == len(reqs)
    # pool + resident plans + batches in flight, as counted and as measured
    # (torch's peak allocation plus the library's plan bytes)
    assert st["peak_hbm_bytes"] <= 64 << 20
    assert st["device_peak_bytes"] <= 64 << 20
    assert st["resident_bytes"] >= srv.pool_bytes
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
