"""Seeded synthetic tensors shaped like the paper's workloads (Sec. 7).

This module holds input generation only: none of the method's arithmetic.  It is
the one module shared by the CUDA-path tests, the oracle tests and the benchmark.
Randomness comes from numpy's PCG64 ``Generator`` (or, for the largest sparse
inputs, torch's device generator), never from the method's own generators.

Workloads
---------
dense_tucker     Tucker product of a Gaussian core with column-orthonormal factors
                 (QR of Gaussian matrices) plus Gaussian noise of a given relative
                 norm (the paper's Tensor 1 with alpha = 1, plus noise); optional
                 geometric decay of the core entries (weight**(i+j+k)).
dense_tucker_batch_torch
                 many dense_tucker tensors of uneven shapes and ranks, built on the
                 device with torch (the batched workload: mode sizes and one rank per
                 tensor drawn uniformly).
coo_zipf_tucker  COO tensor whose coordinates are i.i.d. Zipf(a) per mode truncated
                 to the mode size, values N(0,1) noise plus a planted Tucker
                 component sampled at the same coordinates, both of equal norm.
cp_collinear     sum of R rank-1 terms whose factor columns have unit norm and a
                 fixed pairwise cosine, plus Gaussian noise.
spiked_tucker    the paper's tensor with large coherence (Sec. 7, Tensor 4): a
                 dense_tucker tensor plus n entries at distinct random positions,
                 each N(||T||_F / sqrt(n), 1), so that E ||N|| / ||T|| is about 1.
"""

from __future__ import annotations

import numpy as np


def orthonormal(rng: np.random.Generator, s: int, R: int) -> np.ndarray:
    q, _ = np.linalg.qr(rng.standard_normal((s, R)))
    return q


def _tucker_product(core, factors):
    T = core
    for n, A in enumerate(factors):
        T = np.moveaxis(np.tensordot(A, T, axes=(1, n)), 0, n)
    return T


def dense_tucker(dims, ranks, noise: float, seed: int, core_decay: float | None = None,
                 dtype=np.float64):
    """Returns (T, core, factors); T has dtype ``dtype``, core/factors are float64."""
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(ranks))
    if core_decay is not None:
        w = np.ones(tuple(ranks))
        for n, R in enumerate(ranks):
            shape = [1] * len(ranks)
            shape[n] = R
            w = w * (core_decay ** np.arange(R)).reshape(shape)
        core = core * w
    factors = [orthonormal(rng, s, R) for s, R in zip(dims, ranks)]
    T = _tucker_product(core, factors)
    if noise > 0:
        E = rng.standard_normal(T.shape)
        T = T + E * (noise * np.linalg.norm(T) / np.linalg.norm(E))
    return np.ascontiguousarray(T.astype(dtype)), core, factors


def dense_tucker_batch_torch(count: int, size_range, rank_range, noise: float, seed: int,
                             device, dtype=None):
    """``count`` tensors as dense_tucker (Gaussian core, orthonormal factors, Gaussian
    noise of relative norm ``noise``), built on ``device``: mode sizes uniform in
    ``size_range`` (inclusive), one rank R uniform in ``rank_range`` per tensor.
    Returns (tensors, ranks): a list of contiguous torch tensors and [(R, R, R)]."""
    import torch
    dtype = dtype or torch.float32
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    tensors, ranks = [], []
    for _ in range(count):
        dims = [int(x) for x in rng.integers(size_range[0], size_range[1] + 1, size=3)]
        R = int(rng.integers(rank_range[0], rank_range[1] + 1))
        core = torch.from_numpy(rng.standard_normal((R, R, R))).to(device, torch.float64)
        A = [torch.from_numpy(orthonormal(rng, s, R)).to(device, torch.float64) for s in dims]
        T = torch.einsum("abc,ia,jb,kc->ijk", core, A[0], A[1], A[2])
        E = torch.randn(dims, generator=g, device=device, dtype=torch.float64)
        T = T + E * (noise * torch.linalg.norm(T) / torch.linalg.norm(E))
        tensors.append(T.to(dtype).contiguous())
        ranks.append((R, R, R))
    return tensors, ranks


def zipf_table(s: int, a: float) -> np.ndarray:
    """CDF of the Zipf(a) law truncated to {0, ..., s-1} (P(i) ~ (i+1)^-a)."""
    p = (np.arange(1, s + 1, dtype=np.float64)) ** (-a)
    c = np.cumsum(p)
    return c / c[-1]


def coo_zipf_tucker(dims, nnz: int, ranks, seed: int, zipf_a: float = 1.1,
                    val_dtype=np.float32):
    """Returns (idx int32 (N, nnz), vals, core, factors) generated on the host."""
    rng = np.random.default_rng(seed)
    N = len(dims)
    idx = np.empty((N, nnz), dtype=np.int32)
    for n, s in enumerate(dims):
        cdf = zipf_table(s, zipf_a)
        idx[n] = np.minimum(np.searchsorted(cdf, rng.random(nnz), side="right"), s - 1)
    core = rng.standard_normal(tuple(ranks))
    factors = [orthonormal(rng, s, R) for s, R in zip(dims, ranks)]
    planted = np.empty(nnz)
    chunk = 1 << 16
    for a in range(0, nnz, chunk):
        b = min(a + chunk, nnz)
        G = np.einsum("...r,cr->c...", core, factors[N - 1][idx[N - 1, a:b]])
        for n in range(N - 2, -1, -1):
            G = np.einsum("c...r,cr->c...", G, factors[n][idx[n, a:b]])
        planted[a:b] = G
    noise = rng.standard_normal(nnz)
    planted *= np.linalg.norm(noise) / max(np.linalg.norm(planted), 1e-300)
    vals = (planted + noise).astype(val_dtype)
    return idx, vals, core, factors


def coo_zipf_tucker_torch(dims, nnz: int, ranks, seed: int, device, zipf_a: float = 1.1):
    """Device-side generator of the same distribution as :func:`coo_zipf_tucker`.

    For inputs too large to build on the host quickly (1e8 nonzeros).  Returns
    (idx int32 tensor (N, nnz), vals float32 tensor) on ``device``.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    N = len(dims)
    idx = torch.empty((N, nnz), dtype=torch.int32, device=device)
    for n, s in enumerate(dims):
        cdf = torch.from_numpy(zipf_table(s, zipf_a)).to(device)
        u = torch.rand(nnz, generator=g, device=device, dtype=torch.float64)
        idx[n] = torch.clamp(torch.searchsorted(cdf, u, right=True), max=s - 1).to(torch.int32)
    rng = np.random.default_rng(seed)
    core = torch.from_numpy(rng.standard_normal(tuple(ranks))).to(device, torch.float32)
    factors = [torch.from_numpy(orthonormal(rng, s, R)).to(device, torch.float32)
               for s, R in zip(dims, ranks)]
    planted = torch.empty(nnz, dtype=torch.float32, device=device)
    chunk = 1 << 22
    for a in range(0, nnz, chunk):
        b = min(a + chunk, nnz)
        G = torch.einsum("...r,cr->c...", core, factors[N - 1][idx[N - 1, a:b].long()])
        for n in range(N - 2, -1, -1):
            G = torch.einsum("c...r,cr->c...", G, factors[n][idx[n, a:b].long()])
        planted[a:b] = G
    noise = torch.randn(nnz, generator=g, device=device, dtype=torch.float32)
    planted *= noise.norm() / planted.norm().clamp_min(1e-30)
    return idx, (planted + noise).contiguous()


def cp_collinear(dims, R: int, cosine: float, noise: float, seed: int, dtype=np.float64):
    """Returns (T, factors): unit columns with pairwise cosine ``cosine`` per mode."""
    rng = np.random.default_rng(seed)
    Gm = (1.0 - cosine) * np.eye(R) + cosine * np.ones((R, R))
    L = np.linalg.cholesky(Gm)
    factors = [orthonormal(rng, s, R) @ L.T for s in dims]
    T = 0.0
    for r in range(R):
        t = factors[0][:, r]
        for A in factors[1:]:
            t = np.multiply.outer(t, A[:, r])
        T = T + t
    if noise > 0:
        E = rng.standard_normal(T.shape)
        T = T + E * (noise * np.linalg.norm(T) / np.linalg.norm(E))
    return np.ascontiguousarray(T.astype(dtype)), factors


def spiked_tucker(dims, ranks, noise: float, seed: int, n_spikes: int = 10,
                  dtype=np.float64):
    """Returns (T + N, positions (n_spikes, N) int64, spike values).

    T is :func:`dense_tucker` (dims, ranks, noise, seed); N adds at ``n_spikes``
    distinct random linear positions values drawn from N(||T||_F / sqrt(n_spikes), 1).
    """
    T, _, _ = dense_tucker(dims, ranks, noise, seed)
    rng = np.random.default_rng(seed + 0x5EED)
    flat = T.reshape(-1).copy()
    lin = np.sort(rng.choice(flat.size, n_spikes, replace=False))
    vals = rng.normal(np.linalg.norm(flat) / np.sqrt(n_spikes), 1.0, n_spikes)
    flat[lin] += vals
    pos = np.stack(np.unravel_index(lin, tuple(dims)), axis=1).astype(np.int64)
    return np.ascontiguousarray(flat.reshape(tuple(dims)).astype(dtype)), pos, vals
