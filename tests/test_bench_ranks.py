"""The multi-rank host logic of bench.py on CPU: two gloo ranks (the GPU runs
use one process per GPU over NCCL with the same helpers).  Each rank renders
its own replica, so the job time is the slowest rank's and the value counts
every rank's pixels; the reference arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, local = bench._dist()
    assert (w, r, local) == (ws, rank, rank)
    bench._init_ranks(w, local)
    assert dist.get_backend() == "gloo"
    ms = bench._max_over_ranks(1.0 + rank, w, "cpu")
    out.put((rank, ms, bench._whole_job_value(1.616, w, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]                # max over ranks
    assert res[0][2] == pytest.approx(2 * 1.616 / 2e-3)     # both ranks' pixels


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench._whole_job_value(1.616, 1, 2.0) == pytest.approx(808.0)


def test_reference_arm_prints_on_rank_zero_only():
    """Rank 1 of a reference run exits 0 without work or output."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
