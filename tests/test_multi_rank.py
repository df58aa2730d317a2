"""The N > 1 path of bench.py on CPU: two gloo ranks.

Queries are independent (Sec. 3.2, multi-many-core querying), so the ranks
share no data-path collective: each answers its own query stream, and only
the timing is reduced (maximum over ranks) for the whole-job rate.  These
tests run that bookkeeping with world size 2 on the gloo backend.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import workloads  # noqa: E402

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        w = workloads.scaled(workloads.MIXTURE_64M, 4096, 300, 4)
        Q = bench.rank_queries(w, rank)
        np.save(os.path.join(out_dir, f"q{rank}.npy"), Q)
        # rank r "took" 10 (r + 1) ms: the job's time is the slowest rank's
        ms = 10.0 * (rank + 1)
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        rate = bench.whole_job_rate(WORLD, Q.shape[0], 3, ms_max)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([ms_max, rate]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=WORLD,
             join=True)
    q0, q1 = (np.load(tmp_path / f"q{r}.npy") for r in range(WORLD))
    r0, r1 = (np.load(tmp_path / f"r{r}.npy") for r in range(WORLD))
    # independent query streams of the same shape: no query answered twice
    assert q0.shape == q1.shape == (300, 10)
    assert not (q0[:, None, :] == q1[None, :, :]).all(-1).any()
    # every rank sees the slowest rank's time and the same whole-job rate
    assert r0[0] == r1[0] == 20.0
    assert r0[1] == r1[1] == pytest.approx(WORLD * 300 * 3 / 0.020)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(1, 1000, 2, 500.0) == pytest.approx(4000.0)
