"""Counter-based random numbers for the oracle (test infrastructure only).

Philox4x64-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 4x64-bit counter block is passed
through ten rounds of two 64x64->128-bit multiplies, with the 2x64-bit key
bumped by two Weyl constants between rounds.  The paper's method draws iid
N(0, dt) Brownian increments (Sec. 3.1.2: "whose prior distribution is iid
N(0, dt)"); every such draw here is keyed by (seed, purpose) and a counter
(block, step, particle, stream counter), so any draw can be recomputed in
isolation and in any order.

Normals use the Box-Muller transform on pairs of 53-bit uniforms:
u1 = (r1 >> 11 + 1) 2^-53 in (0, 1], u2 = (r2 >> 11) 2^-53 in [0, 1),
z1 = sqrt(-2 ln u1) cos(2 pi u2), z2 = sqrt(-2 ln u1) sin(2 pi u2).

Pinned by ``tests/test_oracle_rng.py`` against ``numpy.random.Philox``
(numpy's Philox4x64-10 bit generator) and by distribution tests.

The FP32 paths of the Matern noise, which draw one normal per cell and step, use
Philox4x32-10 from the same paper instead: a 4x32-bit counter block through ten rounds
of two 32x32->64-bit multiplies, the 2x32-bit key bumped by two 32-bit Weyl constants.
Its key is (seed mod 2^32, (seed >> 32) mod 2^16 + tag 2^16) and its counter (block,
step, particle, stream counter), each word mod 2^32; normals use Box-Muller on 32-bit
uniforms u1 = (r1 + 1) 2^-32 in (0, 1], u2 = r2 2^-32 in [0, 1).  Pinned by the known-
answer vectors published with the generator and by distribution tests.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B

MASK32 = (1 << 32) - 1
PHILOX32_M0 = 0xD2511F53
PHILOX32_M1 = 0xCD9E8D57
PHILOX32_W0 = 0x9E3779B9
PHILOX32_W1 = 0xBB67AE85

# purposes: the second key word; one independent stream per random choice
TAG_PRIOR_DW = 1     # forecast noise of a window    ctr = (block, step, particle, cycle)
TAG_PCN = 2          # PCN proposal noise            ctr = (block, step, particle, iter ctr)
TAG_PCN_ACCEPT = 3   # PCN accept uniform            ctr = (0, 0, particle, iter ctr)
TAG_RESAMPLE = 4     # systematic resampling offset  ctr = (0, 0, 0, stage ctr)
TAG_TRUTH = 5        # truth noise                   ctr = (block, step, 0, cycle)
TAG_OBS = 6          # observation noise             ctr = (block, 0, 0, cycle)
TAG_INIT = 7         # prior ensemble perturbation   ctr = (block, 0, particle, 0)
TAG_NUDGE = 8        # noise revealed during sequential nudging
TAG_MALA = 9         # MALA proposal noise           ctr = (block, step, particle, iter ctr)
TAG_MALA_ACCEPT = 10  # MALA accept uniform          ctr = (0, 0, particle, iter ctr)


def philox4x64_scalar(ctr, key):
    """One Philox4x64-10 block with Python integers (the definition, unvectorised)."""
    x0, x1, x2, x3 = (int(v) & MASK64 for v in ctr)
    k0, k1 = (int(v) & MASK64 for v in key)
    for _ in range(10):
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + PHILOX_W0) & MASK64
        k1 = (k1 + PHILOX_W1) & MASK64
    return (x0, x1, x2, x3)


def _mulhilo(a: np.ndarray, b: int):
    """Full 64x64 -> 128-bit product of uint64 arrays with a constant, by 32-bit halves."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    b0 = np.uint64(b & 0xFFFFFFFF)
    b1 = np.uint64(b >> 32)
    a0 = a & m32
    a1 = a >> s32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> s32) + (p01 & m32) + (p10 & m32)
    hi = p11 + (p01 >> s32) + (p10 >> s32) + (mid >> s32)
    lo = a * np.uint64(b)
    return hi, lo


def philox4x64(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x64-10 over broadcastable uint64 counter words."""
    with np.errstate(over="ignore"):
        x0, x1, x2, x3 = np.broadcast_arrays(*(np.asarray(v, dtype=np.uint64) for v in (c0, c1, c2, c3)))
        x0, x1, x2, x3 = (v.copy() for v in (x0, x1, x2, x3))
        k0 = int(k0) & MASK64
        k1 = int(k1) & MASK64
        for _ in range(10):
            hi0, lo0 = _mulhilo(x0, PHILOX_M0)
            hi1, lo1 = _mulhilo(x2, PHILOX_M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ np.uint64(k0), lo1, hi0 ^ x3 ^ np.uint64(k1), lo0
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
    return x0, x1, x2, x3


def u53_open0(r):
    """(r >> 11 + 1) * 2^-53: a uniform in (0, 1]."""
    return ((np.asarray(r, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def u53_open1(r):
    """(r >> 11) * 2^-53: a uniform in [0, 1)."""
    return (np.asarray(r, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def box_muller(r_a, r_b):
    """Two standard normals from two raw 64-bit words."""
    u1 = u53_open0(r_a)
    u2 = u53_open1(r_b)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def normals(seed: int, tag: int, count: int, c1, c2, c3) -> np.ndarray:
    """Standard normals z[..., k], k < count, keyed by (seed, tag) and counter (k//4, c1, c2, c3).

    c1, c2, c3 broadcast against each other; the result has their broadcast
    shape plus a trailing axis of length ``count``.  Normal k comes from block
    k // 4: words (r0, r1) give normals 0 and 1 of the block, (r2, r3) give 2 and 3.
    """
    c1, c2, c3 = np.broadcast_arrays(*(np.asarray(v, dtype=np.uint64) for v in (c1, c2, c3)))
    nblk = (count + 3) // 4
    blk = np.arange(nblk, dtype=np.uint64)
    shape = c1.shape + (nblk,)
    r0, r1, r2, r3 = philox4x64(np.broadcast_to(blk, shape), c1[..., None], c2[..., None], c3[..., None],
                                seed, tag)
    z0, z1 = box_muller(r0, r1)
    z2, z3 = box_muller(r2, r3)
    z = np.stack([z0, z1, z2, z3], axis=-1).reshape(c1.shape + (4 * nblk,))
    return z[..., :count]


def uniform_open0(seed: int, tag: int, c2, c3) -> np.ndarray:
    """Uniform in (0, 1] from word r0 of the block (0, 0, c2, c3)."""
    c2, c3 = np.broadcast_arrays(np.asarray(c2, dtype=np.uint64), np.asarray(c3, dtype=np.uint64))
    r0, _, _, _ = philox4x64(0, 0, c2, c3, seed, tag)
    return u53_open0(r0)


def u53_int(seed: int, tag: int, c3: int) -> int:
    """A 53-bit unsigned integer (r0 >> 11 of block (0, 0, 0, c3)), as a Python int."""
    r0, _, _, _ = philox4x64_scalar((0, 0, 0, c3), (seed, tag))
    return r0 >> 11


def philox4x32_scalar(ctr, key):
    """One Philox4x32-10 block with Python integers (the definition, unvectorised)."""
    x0, x1, x2, x3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for _ in range(10):
        p0 = PHILOX32_M0 * x0
        p1 = PHILOX32_M1 * x2
        x0, x1, x2, x3 = (p1 >> 32) ^ x1 ^ k0, p1 & MASK32, (p0 >> 32) ^ x3 ^ k1, p0 & MASK32
        k0 = (k0 + PHILOX32_W0) & MASK32
        k1 = (k1 + PHILOX32_W1) & MASK32
    return (x0, x1, x2, x3)


def philox4x32(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over broadcastable counter words (taken mod 2^32); uint64
    arrays holding 32-bit values."""
    m32 = np.uint64(MASK32)
    s32 = np.uint64(32)
    x0, x1, x2, x3 = np.broadcast_arrays(*(np.asarray(v, dtype=np.uint64) & m32 for v in (c0, c1, c2, c3)))
    x0, x1, x2, x3 = (v.copy() for v in (x0, x1, x2, x3))
    k0 = int(k0) & MASK32
    k1 = int(k1) & MASK32
    for _ in range(10):
        p0 = x0 * np.uint64(PHILOX32_M0)   # < 2^64: exact in uint64
        p1 = x2 * np.uint64(PHILOX32_M1)
        x0, x1, x2, x3 = (p1 >> s32) ^ x1 ^ np.uint64(k0), p1 & m32, (p0 >> s32) ^ x3 ^ np.uint64(k1), p0 & m32
        k0 = (k0 + PHILOX32_W0) & MASK32
        k1 = (k1 + PHILOX32_W1) & MASK32
    return x0, x1, x2, x3


def key32(seed: int, tag: int):
    """The Philox4x32 key of (seed, tag): distinct for seeds below 2^48 and tags below 2^16."""
    return int(seed) & MASK32, ((int(seed) >> 32) & 0xFFFF) | ((int(tag) & 0xFFFF) << 16)


def box_muller32(r_a, r_b):
    """Two standard normals from two raw 32-bit words (FP64 transform)."""
    u1 = (np.asarray(r_a, dtype=np.uint64).astype(np.float64) + 1.0) * 2.0 ** -32
    u2 = np.asarray(r_b, dtype=np.uint64).astype(np.float64) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def normals32(seed: int, tag: int, count: int, c1, c2, c3) -> np.ndarray:
    """As ``normals``, from Philox4x32-10 under key32(seed, tag) and counter (k//4, c1, c2, c3)
    mod 2^32: words (r0, r1) give normals 0 and 1 of a block, (r2, r3) give 2 and 3."""
    c1, c2, c3 = np.broadcast_arrays(*(np.asarray(v, dtype=np.uint64) for v in (c1, c2, c3)))
    nblk = (count + 3) // 4
    blk = np.arange(nblk, dtype=np.uint64)
    shape = c1.shape + (nblk,)
    r0, r1, r2, r3 = philox4x32(np.broadcast_to(blk, shape), c1[..., None], c2[..., None], c3[..., None],
                                *key32(seed, tag))
    z0, z1 = box_muller32(r0, r1)
    z2, z3 = box_muller32(r2, r3)
    z = np.stack([z0, z1, z2, z3], axis=-1).reshape(c1.shape + (4 * nblk,))
    return z[..., :count]


GEN64, GEN32 = "philox4x64", "philox4x32"


def window_increments(seed: int, tag: int, N: int, Ns: int, K: int, dt: float, c3: int,
                      particle0: int = 0, gen: str = GEN64) -> np.ndarray:
    """dW[p, s, k] ~ N(0, dt): block k//4, step s, particle particle0+p, stream counter c3,
    from Philox4x64-10 (``gen`` = GEN64) or Philox4x32-10 (GEN32)."""
    p = np.arange(particle0, particle0 + N, dtype=np.uint64)[:, None]
    s = np.arange(Ns, dtype=np.uint64)[None, :]
    draw = normals32 if gen == GEN32 else normals
    if gen not in (GEN64, GEN32):
        raise ValueError(gen)
    return np.sqrt(dt) * draw(seed, tag, K, s, p, np.uint64(c3))
