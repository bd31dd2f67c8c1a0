"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2).

The bench's N > 1 path runs one independent hologram job per rank (no data-path
collective); ranks meet only in a barrier and in the max over ranks of the timed
region.  These tests run that logic as two gloo processes on 127.0.0.1.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, lr = bench.dist_setup(None)
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(local_ms[r], dist)
        value = bench.job_value(w, 3, 100, slowest)
        dist.barrier()
        out.put((r, w, lr, slowest, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_two_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    local_ms = [120.0, 150.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, local_ms, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(out.get(timeout=5) for _ in range(2))
    for r, (rank, world, local, slowest, value) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == 150.0                       # every rank sees the slowest rank
        assert value == pytest.approx(2 * 3 * 100 / 0.150)


def test_single_rank_has_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, None) == 42.0
    assert bench.job_value(1, 2, 100, 10.0) == pytest.approx(20000.0)


def _ref_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    # ranks other than 0 leave the reference arm at once, without work or output
    out.put((rank, bench.run_reference(None, world, rank) if rank != 0 else "rank0"))


def test_reference_arm_other_ranks_exit_without_work():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    p = ctx.Process(target=_ref_worker, args=(1, 2, _free_port(), out))
    p.start()
    p.join(60)
    assert p.exitcode == 0
    assert out.get(timeout=5) == (1, 0)


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints one JSON
    line with the same metric as the CUDA arm and describes itself as the oracle."""
    import json
    import subprocess
    sys.path.insert(0, ROOT)
    import bench
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"], cwd=ROOT, env=env, check=True,
                         capture_output=True, text=True, timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 1 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
