"""The multi-rank bench path on CPU: two gloo ranks, each with its own job
(replicas; the method has no cross-GPU exchange), the whole-job time taken
as the max over ranks, and the value counting every rank's iterations."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1507_08751_gb300 import synth
    t = bench.job_time_over_ranks(1.0 + 0.5 * rank, world, torch.device("cpu"))
    Y, _, _ = synth.video(seed=bench.replica_seed(rank), M=256, N=256)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, float(np.abs(Y).sum())))


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_jobs():
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
    assert [r[1] for r in res] == [1.5, 1.5]          # max over ranks, on every rank
    assert res[0][2] != res[1][2]                     # each rank has its own input
    import bench
    assert bench.whole_job_value(2, 300, 5, 1.5) == 2000.0   # 2 ranks x 300 x 5 / 1.5 s


def test_one_rank_keeps_its_own_time():
    import bench
    assert bench.job_time_over_ranks(0.25, 1, None) == 0.25
