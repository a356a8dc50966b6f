"""The bench's multi-rank logic on CPU (world size 2, gloo): replicas only --
no collective on the data path, only the max-over-ranks timing and the
whole-job figure; each rank renders its own views.  The reference arm (the
FP64 oracle on the host cores) runs on rank 0 alone."""
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


def _bench_reference(rank, world, extra=()):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", str(world),
                        "--n-gauss", "3000", "--steps", "1", "--warmup", "0", *extra],
                       cwd=root, env=env, capture_output=True, text=True, timeout=300)
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    return r.returncode, lines, r.stderr


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle; the others exit 0 and print nothing."""
    rc, lines, err = _bench_reference(1, 2)
    assert rc == 0, err
    assert lines == []


def test_reference_arm_rank0_prints_one_line():
    rc, lines, err = _bench_reference(0, 2)
    assert rc == 0, err
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"] > 0
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
