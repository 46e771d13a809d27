"""Random objects of the sketched Tucker-ALS method, from published definitions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper fixes what the random objects must satisfy but not how to draw them:

* Sec. 3.1, TensorSketch definition: each per-mode bucket map H_n is 3-wise
  independent on [s_n] -> [m] and each sign map S_n is 4-wise independent on
  [s_n] -> {-1, +1}.
* Sec. 5, composite sketching matrix: a Gaussian factor with variance 1/k1.
* Alg. 5: a Gaussian test matrix for the randomized SVD.
* Sec. 3.2, importance sampling: independent draws with replacement.

Reading adopted here (identical on the CUDA side, written independently there):

* Counter-based generator: splitmix64 (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014) used as a stateless mix of
  ``seed``, a 64-bit ``tag`` naming the object, and an element counter.
* Hash family: Carter-Wegman polynomials over the Mersenne prime p = 2^31 - 1
  (Carter & Wegman 1979; Thorup & Zhang 2012).  A random polynomial of degree
  d-1 with coefficients uniform in Z_p is d-wise independent on [0, p); degree 2
  gives the 3-wise bucket map, degree 3 the 4-wise sign map.  bucket =
  poly2(i) mod m; sign = +1 if poly3(i) is even else -1.
* Gaussians: Box-Muller in FP64 from two 53-bit uniforms.
"""

from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15          # splitmix64 increment (golden ratio)
MIX_M1 = 0xBF58476D1CE4E5B9        # splitmix64 finaliser multipliers
MIX_M2 = 0x94D049BB133111EB
P31 = (1 << 31) - 1                 # Mersenne prime of the hash family

# Purposes of random objects (the top byte of a tag).
PURPOSE_TS_HASH = 1        # TensorSketch bucket/sign maps H_{n,k}, S_{n,k}
PURPOSE_RRF_HASH = 2       # CountSketch factor of the composite sketch (Alg. 3)
PURPOSE_RRF_GAUSS = 3      # Gaussian factor G of the composite sketch
PURPOSE_RSVD_GAUSS = 4     # Gaussian test matrix of RSVD-LRLS (Alg. 5)
PURPOSE_LEV_UNIFORM = 5    # uniforms driving leverage-score sampling


def make_tag(purpose: int, sweep: int, n: int, k: int) -> int:
    """Pack (purpose, sweep, subproblem mode n, hashed mode k) into 64 bits."""
    assert 0 <= purpose < 256 and 0 <= sweep < (1 << 24)
    assert 0 <= n < 256 and 0 <= k < 256
    return (purpose << 56) | (sweep << 32) | (n << 16) | k


def _mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser on a uint64 array (wrap-around arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(MIX_M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(MIX_M2)
        z ^= z >> np.uint64(31)
    return z


def _mix64_int(z: int) -> int:
    z &= MASK64
    z ^= z >> 30
    z = (z * MIX_M1) & MASK64
    z ^= z >> 27
    z = (z * MIX_M2) & MASK64
    z ^= z >> 31
    return z


def rand64(seed: int, tag: int, idx) -> np.ndarray:
    """64 random bits for element ``idx`` of the object named ``tag``.

    rand64 = mix(mix(seed + GAMMA*(tag+1)) + GAMMA*(idx+1))   (mod 2^64)
    """
    key = _mix64_int((seed + GAMMA * (tag + 1)) & MASK64)
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + np.uint64(GAMMA) * (idx + np.uint64(1))
    return _mix64(z)


def uniform01(seed: int, tag: int, idx) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    r = rand64(seed, tag, idx)
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, tag: int, count: int) -> np.ndarray:
    """``count`` N(0,1) doubles; entry e uses counters 2e and 2e+1 (Box-Muller)."""
    e = np.arange(count, dtype=np.uint64)
    r1 = rand64(seed, tag, np.uint64(2) * e)
    r2 = rand64(seed, tag, np.uint64(2) * e + np.uint64(1))
    u1 = ((r1 >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u2 = (r2 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)          # [0, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def hash_coefficients(seed: int, tag: int):
    """Coefficients (a0, a1, a2) of the bucket polynomial and (b0..b3) of the sign polynomial."""
    c = rand64(seed, tag, np.arange(7, dtype=np.uint64)) % np.uint64(P31)
    return c[:3].copy(), c[3:].copy()


def poly_mod_p(coefs: np.ndarray, keys: np.ndarray) -> np.ndarray:
    """sum_j coefs[j] * keys^j mod p, by Horner's rule with a reduction after every step."""
    keys = np.asarray(keys, dtype=np.uint64)
    assert np.all(keys < np.uint64(P31)), "hash keys must lie in [0, 2^31 - 1)"
    acc = np.full(keys.shape, coefs[-1], dtype=np.uint64)
    for c in coefs[-2::-1]:
        acc = (acc * keys + np.uint64(c)) % np.uint64(P31)
    return acc


def hash_table(seed: int, purpose: int, sweep: int, n: int, k: int, size: int, nbins: int):
    """Bucket map and sign map on [0, size) for object (purpose, sweep, n, k).

    Returns (bins int64 in [0, nbins), signs float64 in {-1, +1}).
    """
    tag = make_tag(purpose, sweep, n, k)
    a, b = hash_coefficients(seed, tag)
    keys = np.arange(size, dtype=np.uint64)
    bins = (poly_mod_p(a, keys) % np.uint64(nbins)).astype(np.int64)
    odd = (poly_mod_p(b, keys) & np.uint64(1)).astype(np.int64)
    signs = 1.0 - 2.0 * odd.astype(np.float64)
    return bins, signs


def pack_table(bins: np.ndarray, signs: np.ndarray) -> np.ndarray:
    """int32 packing used at the C boundary: bucket in bits 0..30, bit 31 set for sign -1."""
    v = bins.astype(np.uint32) | ((signs < 0).astype(np.uint32) << np.uint32(31))
    return v.view(np.int32)


def unpack_table(packed: np.ndarray):
    u = np.asarray(packed).view(np.uint32)
    bins = (u & np.uint32(0x7FFFFFFF)).astype(np.int64)
    signs = np.where((u >> np.uint32(31)) != 0, -1.0, 1.0)
    return bins, signs
