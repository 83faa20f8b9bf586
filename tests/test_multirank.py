"""The benchmark's multi-rank path on CPU: two gloo ranks, no GPU.

With N > 1 every rank evaluates its own replica (independent systems, no
data-path collective); the only collectives are the barriers around the timed
region and the max over ranks of the measured time.  These tests run that
host logic as two processes: the max over ranks reaches every rank, the
whole-job rate counts every rank's units over the slowest rank's time, and
the reference arm does its work on rank 0 only.
"""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.5 + 2.0 * rank                                 # rank 1 is the slow one
        t_max = bench.max_over_ranks(t)
        dist.barrier()
        rate = bench.whole_job_rate(1000.0, world, t_max)
        # the reference arm: rank 0 alone runs it; the others return without work or output
        out = io.StringIO()
        ran = None
        if rank != 0:
            with contextlib.redirect_stdout(out):
                ran = bench.run_reference(None)
        q.put((rank, t_max, rate, ran, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [3.5, 3.5]                # every rank sees the slowest time
    assert res[0][2] == pytest.approx(2000.0 / 3.5)          # all ranks' units over the max time
    assert res[1][3] is None and res[1][4] == ""             # rank 1 ran no reference work


def test_single_process_is_identity():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.25) == 2.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_json_line():
    # `bench.py --impl reference` at N = 1: the FP64 oracle on the host cores prints one JSON line with the
    # benchmark's metric, unit and direction, its cpu_baseline description and an e2e entry without copies
    import json
    import subprocess
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 0 and d["ms_per_step"] > 0 and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("membrane_slab")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
