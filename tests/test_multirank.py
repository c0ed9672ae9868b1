"""The N > 1 path on CPU: world-size-2 gloo process groups.

The benchmark runs one independent replica per rank (no data-path
collective); ranks meet only at the timing barrier and the MAX all-reduce of
the elapsed time, and rank 0 alone prints the result line.  Both are
exercised here without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    m = bench.max_over_ranks(1.5 + r, w)
    with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
        f.write(f"{w} {m}")
    import torch.distributed as dist
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        w, m = open(tmp_path / f"rank{r}.txt").read().split()
        assert int(w) == 2
        assert float(m) == 2.5  # every rank sees the slowest rank's time


@pytest.mark.timeout(300)
def test_reference_arm_under_torchrun_prints_once():
    # the launch the benchmark driver uses for N = 2 (gloo without a GPU):
    # exit 0 on every rank, one JSON line from rank 0
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--sizes", "8,10",
           "--cpu-sample-points", "4096"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=280, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_write_traffic_keeps_the_timed_step(tmp_path, monkeypatch):
    # ncu CSV of two steps (warm-up, timed) of two pass_kernel launches plus a
    # table kernel: the timed step's DRAM bytes, scaled to 2^28 points per exec
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    rows = ['"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
            '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"']
    vals = {0: (100, 50), 1: (200, 70), 2: (1000, 500), 3: (2000, 700)}
    for i, (rd, wr) in vals.items():
        for name, v in (("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr), ("gpu__time_duration.sum", 9)):
            rows.append(f'"{i}","1","p","h","void pass_kernel<8, 0, 0>(PassParams)","1","7","(128, 1, 1)",'
                        f'"(912, 1, 1)","0","10.3","s","{name}","byte","{v:,}"')
    rows.append('"9","1","p","h","twiddle_table_kernel(float *, int)","1","7","(256, 1, 1)","(1, 1, 1)","0",'
                '"10.3","s","dram__bytes_read.sum","byte","123456"')
    csv_path = tmp_path / "t.csv"
    csv_path.write_text("==PROF== Connected\n" + "\n".join(rows) + "\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h")
    args = argparse.Namespace(write_traffic=str(csv_path), log2_points=26, workload="sweep1d", precision="fp16")
    bench.write_traffic(args)
    d = json.load(open(tmp_path / "profiles" / "traffic_sweep1d.json"))
    assert d["measured_bytes_per_step_at_2^26_points"] == 1000 + 500 + 2000 + 700
    assert d["traffic_bytes_per_step"] == 4 * 4200 and d["launches_per_step"] == 2 and d["kernel_hash"] == "h"


def test_clock_sampler_summary(tmp_path, monkeypatch):
    # nvidia-smi samples (index, sm MHz, max MHz, power, active mask, hw slowdown,
    # hw thermal, sw thermal, sw power cap) -> median SM clock and the reasons seen
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("TCFFT_CLOCKS_DIR", str(tmp_path))
    cs = bench.ClockSampler(0)
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage line"]
    with open(cs.path, "w") as f:
        f.write("\n".join(lines) + "\n")

    class _Proc:  # a sampler that already exited
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    cs.proc = _Proc()
    cs.f = open(os.devnull, "w")
    out = cs.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
