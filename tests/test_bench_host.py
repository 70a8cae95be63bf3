"""Host logic of bench.py on the CPU: the reference arm's JSON line (the CPU
oracle on a bounded sample), its behaviour under torchrun with two ranks
(rank 0 alone prints, the others exit 0), and the max-over-ranks reduction
and whole-job aggregation of the N-replica path, run with the gloo backend
on two processes."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check_reference_line(d, n_gpus, workload):
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is False and d["n_gpus"] == n_gpus
    assert d["config"]["workload"] == workload
    # value: seconds per iteration estimated from the timed elements; a step
    # is one element, so an iteration takes far longer than a step
    assert d["value"] > 0 and 0 < d["ms_per_step"] < d["value"] * 1e3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


# the reference arm's logic on the smallest named workload (its elements take
# milliseconds; the benchmark's own workload takes seconds per element)
def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "10", "--warmup", "2",
                        "--config", "c1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 1, "c1")


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "10", "--warmup", "2", "--config", "c1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1  # rank 0 only
    _check_reference_line(lines[0], 2, "c1")


def _reduce_worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t = bench.reduce_max(dist, 0.25 + rank, "cpu")  # per-rank step times 0.25 s and 1.25 s
        q.put((rank, t, bench.whole_job_value(t, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_reduce_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; two replicas do two iterations in it
    assert got == [(0, 1.25, 0.625), (1, 1.25, 0.625)]


def test_single_process_path_is_the_identity():
    import bench
    assert bench.reduce_max(None, 0.4, "cpu") == 0.4
    assert bench.whole_job_value(0.4, 1) == 0.4
