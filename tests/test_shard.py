"""The input sketch sharded over ranks (Alg. 4's right-hand side is linear in the
entries): two gloo CPU ranks each sketch their share and all_reduce the partials; the
result must equal the one-rank sketch.  The per-share sketch is the oracle's here (a CPU
stand-in for the library's kernels); the GPU test runs the library on every share."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(kind):
    from oracle import rng
    from paper_2104_01101_gb300 import synth
    if kind == "coo":
        dims, m = (300, 250, 200, 150), 512
        idx, vals, _, _ = synth.coo_zipf_tucker(dims, 20000, (3, 3, 3, 3), seed=7,
                                                val_dtype=np.float64)
        X = (idx, vals)
    else:
        dims, m = (37, 30, 26), 200   # 37 slabs: uneven shares
        X = np.random.default_rng(4).standard_normal(dims)
    tables = {}
    for n in range(len(dims)):
        tables[n] = [rng.hash_table(3, 1, 0, n, k, dims[k], m) if k != n else None
                     for k in range(len(dims))]
    return dims, m, X, tables


def _oracle_stand_in(kind, dims_full):
    """sketch_fn for shard.partial_input_sketch computing a share's sketch with the
    oracle (float64 numpy), the packed tables unpacked."""
    from oracle import rng, sketch
    from paper_2104_01101_gb300.tsketch import Coo

    def fn(Xs, mode, tabs, m):
        host = [rng.unpack_table(t.numpy()) for k, t in enumerate(tabs) if k != mode]
        if isinstance(Xs, Coo):
            Y = sketch.input_sketch_coo(Xs.indices.numpy().astype(np.int64), Xs.values.numpy(),
                                        Xs.dims, mode, host, m)
        else:
            Y = sketch.input_sketch_dense(Xs.numpy(), mode, host, m)
        return torch.from_numpy(Y)
    return fn


def _torch_problem(kind, dims, X, tables, n):
    from oracle import rng
    from paper_2104_01101_gb300.tsketch import Coo
    tabs = [torch.from_numpy(rng.pack_table(*tables[n][k])) if k != n else None
            for k in range(len(dims))]
    if kind == "coo":
        idx, vals = X
        Xt = Coo(torch.from_numpy(idx.astype(np.int32)), torch.from_numpy(vals), dims)
    else:
        Xt = torch.from_numpy(X)
    return Xt, tabs


def _rank_main(rank, world, port, kind, out):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2104_01101_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        dims, m, X, tables = _problem(kind)
        res = {}
        for n in range(len(dims)):
            Xt, tabs = _torch_problem(kind, dims, X, tables, n)
            Y = shard.sharded_input_sketch(Xt, n, tabs, m, sketch_fn=_oracle_stand_in(kind, dims))
            res[n] = Y.numpy()
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["coo", "dense"])
def test_sharded_input_sketch_two_gloo_ranks_equals_one_rank(kind):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import sketch
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, kind, out), nprocs=world, join=True)
    dims, m, X, tables = _problem(kind)
    for n in range(len(dims)):
        host = [tables[n][k] for k in range(len(dims)) if k != n]
        if kind == "coo":
            idx, vals = X
            want = sketch.input_sketch_coo(idx.astype(np.int64), vals, dims, n, host, m)
            absY = sketch.input_sketch_coo(idx.astype(np.int64), np.abs(vals), dims, n,
                                           [(b, np.ones_like(s)) for b, s in host], m)
        else:
            want = sketch.input_sketch_dense(X, n, host, m)
            absY = sketch.input_sketch_dense(np.abs(X), n,
                                             [(b, np.ones_like(s)) for b, s in host], m)
        for r in range(world):
            Y = out[r][n]
            assert np.array_equal(Y != 0, want != 0)       # the same bins are filled
            assert np.all(np.abs(Y - want) <= 8 * 2.0 ** -53 * absY + 1e-300)
        assert np.array_equal(out[0][n], out[1][n])        # every rank holds the same sum


def test_share_ranges_partition_every_size():
    from paper_2104_01101_gb300 import shard
    for total in (0, 1, 5, 37, 100):
        for world in (1, 2, 3, 8):
            spans = [shard.share_range(total, q, world) for q in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(spans[q][1] == spans[q + 1][0] for q in range(world - 1))
            assert max(e - b for b, e in spans) - min(e - b for b, e in spans) <= 1
    with pytest.raises(ValueError):
        shard.share_range(10, 2, 2)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["coo", "dense"])
@pytest.mark.parametrize("world", [2, 3])
def test_library_shares_sum_to_the_whole_sketch(kind, world):
    # The library's kernels on every share of a partition (the ranks of a sharded run,
    # here one after the other on one GPU) sum to the library's sketch of the whole
    # tensor: the same bins, values within FP32 rounding of the summation.
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from bounds import U32, summation_bound
    from oracle import sketch
    from paper_2104_01101_gb300 import build, shard, tsketch
    build.build_library()
    dims, m, X, tables = _problem(kind)
    for n in range(len(dims)):
        Xt, tabs = _torch_problem(kind, dims, X, tables, n)
        if kind == "coo":
            Xg = tsketch.Coo(Xt.indices.cuda(), Xt.values.float().cuda(), dims)
        else:
            Xg = Xt.float().cuda()
        tg = [t.cuda() if t is not None else None for t in tabs]
        whole = tsketch.tensorsketch_input(Xg, n, tg, m).double().cpu().numpy()
        parts = sum(shard.partial_input_sketch(Xg, n, tg, m, q, world).double().cpu().numpy()
                    for q in range(world))
        host = [tables[n][k] for k in range(len(dims)) if k != n]
        if kind == "coo":
            idx, vals = X
            v32 = vals.astype(np.float32).astype(np.float64)
            absY = sketch.input_sketch_coo(idx.astype(np.int64), np.abs(v32), dims, n,
                                           [(b, np.ones_like(s)) for b, s in host], m)
            cnt = sketch.input_sketch_coo(idx.astype(np.int64), np.ones_like(v32), dims, n,
                                          [(b, np.ones_like(s)) for b, s in host], m)
        else:
            x32 = X.astype(np.float32).astype(np.float64)
            absY = sketch.input_sketch_dense(np.abs(x32), n,
                                             [(b, np.ones_like(s)) for b, s in host], m)
            cnt = sketch.input_sketch_dense(np.ones_like(x32), n,
                                            [(b, np.ones_like(s)) for b, s in host], m)
        assert np.array_equal(parts != 0, whole != 0)
        assert np.all(np.abs(parts - whole) <= summation_bound(absY, cnt + world, U32) + 1e-30)
