"""The one-pass input sketch (Alg. 4's right-hand side Y_n = S^(n) T_(n)^T) sharded over
ranks.

The sketch is linear in the entries of the tensor, so it splits over any partition of
them: each rank sketches its own share with the SAME hash tables and a sum all-reduce of
the m x s_n partial sketches gives Y_n.

* COO tensors: rank q of p takes the contiguous range of nonzeros
  [q nnz / p, (q + 1) nnz / p).
* Dense tensors: rank q takes the slab of mode-0 indices [q s_0 / p, (q + 1) s_0 / p) (a
  contiguous block of the C-order array).  For n != 0 the slab's mode-0 coordinates are
  local, so the mode-0 table is sliced to the slab; for n = 0 each rank owns whole
  columns of Y_0 (no sum needed: the partial of the other ranks is zero there).

Argument marshalling and partitioning only: the sketch of each share runs in the
library (tsketch.tensorsketch_input) unless the caller passes another ``sketch_fn``; the
reduction is torch.distributed's all_reduce (NCCL on GPUs, gloo on CPU ranks).
"""

from __future__ import annotations


def share_range(total: int, rank: int, world: int):
    """[begin, end) of rank's contiguous share of `total` items (balanced to one item)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError(f"rank {rank} of world {world}")
    return total * rank // world, total * (rank + 1) // world


def coo_share(idx, vals, rank: int, world: int):
    """Rank's contiguous share of a COO tensor's nonzeros: (idx[:, b:e], vals[b:e])."""
    b, e = share_range(int(vals.shape[0]), rank, world)
    return idx[:, b:e], vals[b:e]


def dense_slab(T, rank: int, world: int):
    """Rank's slab of mode-0 indices of a dense tensor: (T[b:e], b)."""
    b, e = share_range(int(T.shape[0]), rank, world)
    return T[b:e], b


def _library_sketch(X, mode, tables, m):
    from . import tsketch
    return tsketch.tensorsketch_input(X, mode, tables, m)


def partial_input_sketch(X, mode: int, tables, m: int, rank: int, world: int, sketch_fn=None):
    """This rank's partial Y_mode (m x dims[mode]): the sketch of its share of X.

    X is a dense torch tensor or a tsketch.Coo; tables[k] (k != mode) are the packed
    tables of the whole tensor (tables[mode] is ignored).  sketch_fn(X_share, mode,
    tables_share, m) computes the sketch of a share (default: the library)."""
    import torch
    from .tsketch import Coo
    fn = sketch_fn or _library_sketch
    if isinstance(X, Coo):
        idx, vals = coo_share(X.indices, X.values, rank, world)
        part = Coo(idx.contiguous(), vals.contiguous(), X.dims)
        return fn(part, mode, tables, m)
    slab, b = dense_slab(X, rank, world)
    e = b + slab.shape[0]
    tabs = list(tables)
    if mode != 0:
        tabs[0] = tables[0][b:e]
        return fn(slab.contiguous(), mode, tabs, m)
    # mode 0: this rank owns columns b..e-1 of Y_0
    Y = torch.zeros((m, X.shape[0]), dtype=X.dtype, device=X.device)
    if e > b:
        Y[:, b:e] = fn(slab.contiguous(), 0, tabs, m)
    return Y


def sharded_input_sketch(X, mode: int, tables, m: int, group=None, sketch_fn=None):
    """Y_mode over the ranks of `group` (the default process group when None): every rank
    passes the whole tensor's descriptor and tables, sketches its share, and all ranks
    receive the summed sketch."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    Y = partial_input_sketch(X, mode, tables, m, rank, world, sketch_fn)
    if world > 1:
        dist.all_reduce(Y, op=dist.ReduceOp.SUM, group=group)
    return Y
