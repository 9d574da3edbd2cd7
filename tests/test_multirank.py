"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own batch of cells (weak
scaling, no data-path collective), the job time is the slowest rank's and the rate counts the
units of every rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import bench
    from paper_2510_07843_gb300 import synth as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = S.spec_small_51prb(n_prb=2)
        slot = S.make_slot(spec, bench.rank_seed(rank), keep_h=False)
        local_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
        job_ms = bench.max_over_ranks(local_ms)
        n_re = bench.n_data_res(spec)
        rate = bench.whole_job_rate(world, n_re, 5, job_ms)
        out[rank] = (job_ms, rate, float(np.abs(slot.Y).sum()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    (t0, r0, y0), (t1, r1, y1) = out[0], out[1]
    assert t0 == t1 == 20.0  # every rank reports the slowest rank's time
    assert r0 == r1
    from paper_2510_07843_gb300 import synth as S
    import bench
    n_re = bench.n_data_res(S.spec_small_51prb(n_prb=2))
    assert r0 == pytest.approx(2 * n_re * 5 / 0.020)
    assert y0 != y1  # each rank draws its own cells


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 100, 10, 1000.0) == pytest.approx(1000.0)
