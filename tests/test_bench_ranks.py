"""The N>1 bench path on CPU: two gloo ranks.

Each rank solves its own independent batch (no data-path exchange); the job's
time is the slowest rank's, taken by an all-reduce MAX, and the whole-job
value counts every rank's solves.  Runs as two spawned processes on 127.0.0.1.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from synth.inputs import batched_case  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench.dist_init(None)
        seconds = 1.0 + 0.5 * rank                      # rank 1 is the slower one
        t = bench.max_over_ranks(seconds, got_ws)
        v = bench.whole_job_value(64 * 3, t, got_ws)
        dist.barrier()
        out[rank] = (got_ws, got_rank, got_local, t, v, bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_value():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for r in range(ws):
        got_ws, got_rank, got_local, t, v, seed = out[r]
        assert (got_ws, got_rank, got_local) == (ws, r, r)
        assert t == 1.5                                  # the slowest rank's time on every rank
        assert v == pytest.approx(ws * 64 * 3 / 1.5)
    assert out[0][5] != out[1][5]


def test_single_rank_is_identity():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_value(64, 2.0, 1) == 32.0


def test_rank_batches_are_independent():
    assert bench.rank_seed(0) == 4                       # rank 0 solves the pinned seed-4 batch
    a = batched_case(6, 4, seed=bench.rank_seed(0))
    b = batched_case(6, 4, seed=bench.rank_seed(1))
    assert all((x.m0 != y.m0).any() for x, y in zip(a, b))
    assert len({bench.rank_seed(r) for r in range(8)}) == 8
