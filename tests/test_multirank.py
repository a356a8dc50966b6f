"""The bench's multi-rank logic on CPU (world size 2, gloo): replicas only --
no collective on the data path, only the max-over-ranks timing and the
whole-job figure; each rank renders its own views."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = 100.0 + 25.0 * rank  # the slower rank sets the job time
    m = bench.max_over_ranks(elapsed, world, "cpu")
    views = [(rank * bench.N_VIEWS + j * 10) % 160 for j in range(bench.N_VIEWS)]
    out.put((rank, m, bench.job_ms_per_view(m, 30, world), views))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_job_figure():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, v0, views0), (r1, m1, v1, views1) = res
    assert m0 == m1 == 125.0
    assert v0 == v1 == pytest.approx(125.0 / 60)
    assert set(views0).isdisjoint(views1)  # replicas render different views


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_ms_per_view(90.0, 30, 1) == 3.0
