"""Multi-rank path of bench.py on CPU: gloo, world size 2 (no GPU needed)."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2204_00326_gb300 import replicas

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank  # rank 1 is the slow one
    mx = replicas.max_over_ranks(ms_local)
    out[rank] = (mx, replicas.job_throughput(16384, world, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import random

    port = 29500 + random.randint(0, 2000)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == pytest.approx(16384 * 2 / 15e-3 / 1e6)


def test_single_process_is_identity():
    from paper_2204_00326_gb300 import replicas

    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(1e6, 1, 1000.0) == pytest.approx(1.0)
