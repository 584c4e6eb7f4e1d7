"""The multi-GPU path is replicas only (every rank renders its own batch,
no exchange on the data path): its host logic on two CPU ranks over gloo.
The timed region is the slowest rank's, the whole-job value counts every
rank's frames, the ranks' workloads differ but share their shape, and the
reference arm runs on rank 0 only."""
import os
import socket
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        timed = [12.5, 40.0][rank]  # rank 1 is the slow one
        worst = bench.max_over_ranks(timed, world, torch.device("cpu"))
        bench.SCENES = 4
        counts, soas, optics = bench.workload(seed_offset=1000 * rank)
        ref = bench.run_reference(SimpleNamespace(warmup=0, steps=1), rank, world)
        out.put((rank, worst, [int(c) for c in counts], float(soas[0][0, 0]),
                 [s.shape[0] for s in soas], ref is None))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = out.get(timeout=600)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time
    assert res[0][1] == res[1][1] == 40.0
    # replicas: each rank its own batch of the same shape
    assert res[0][2] != res[1][2] or res[0][3] != res[1][3]
    assert len(res[0][2]) == len(res[1][2]) == 4
    assert res[0][4] == res[1][4] == [9] * 4
    # the reference arm: rank 0 runs it, rank 1 exits without work
    assert res[0][5] is False and res[1][5] is True


def test_job_throughput_counts_every_rank():
    # 32 frames per step on each of 4 ranks, 10 steps, slowest rank 20 ms
    assert bench.job_throughput(32, 10, 4, 20.0) == pytest.approx(32 * 10 * 4 / 0.02)
    assert bench.job_throughput(32, 10, 1, 20.0) == pytest.approx(16000.0)
