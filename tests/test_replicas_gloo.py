"""The multi-replica measurement logic (barrier, slowest-rank time, whole-job
throughput) with two gloo ranks on CPU.  The force path itself has no
exchange step: ranks only agree on the timing."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_0902_0827_gb300 import replicas
    w, r, local = replicas.setup("gloo")
    assert (w, r, local) == (world, rank, rank)
    replicas.barrier(w)
    ms = 2.0 + rank          # per-rank step times: 2 ms and 3 ms
    units = 1000.0 * (rank + 1)  # per-rank units per step: 1000 and 2000
    slow = replicas.max_over_ranks(ms, w, "cpu")
    thr = replicas.job_throughput(units, ms, w, "cpu")
    out.put((rank, slow, thr))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, slow, thr in res:
        assert slow == 3.0
        assert thr == pytest.approx(3000.0 / 3e-3)


def test_single_process_needs_no_process_group():
    from paper_0902_0827_gb300 import replicas
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert replicas.setup("gloo") == (1, 0, 0)
    assert replicas.max_over_ranks(4.5, 1, "cpu") == 4.5
    assert replicas.job_throughput(100.0, 2.0, 1, "cpu") == pytest.approx(100.0 / 2e-3)
