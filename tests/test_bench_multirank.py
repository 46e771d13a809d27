"""Host logic of bench.py's N > 1 form (replicas, max-over-ranks timing) on CPU ranks
with the gloo backend: world size 2, rendezvous on 127.0.0.1."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # rank r measured (r + 1) ms per step and 2 (r + 1) ms end to end
        ms, e2e = bench.max_over_ranks([rank + 1.0, 2.0 * (rank + 1)], world, "cpu")
        dist.barrier()
        out[rank] = (ms, e2e, bench.job_sweeps_per_s(world, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for r in range(world):
        ms, e2e, value = out[r]
        assert ms == 2.0 and e2e == 4.0          # every rank sees the slowest rank's time
        assert value == pytest.approx(world * bench.SWEEPS * 1e3 / 2.0)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 5.0], 1, "cpu") == [3.0, 5.0]
    assert bench.job_sweeps_per_s(1, 5.0) == pytest.approx(bench.SWEEPS * 200.0)
