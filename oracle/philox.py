"""Philox4x32-10 counter-based generator and the method's random variates (oracle).

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter and a
2x32-bit key; each of the 10 rounds multiplies counter words 0 and 2 by
0xD2511F53 and 0xCD9E8D57 into 64-bit products (hi, lo) and outputs
(hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); between rounds the key is bumped by
the Weyl constants (0x9E3779B9, 0xBB67AE85).  Written here with numpy uint64
arithmetic, independently of the CUDA implementation.

Stream layout (the paper only says "draw a random number", Sec. 2.4):
  key          = (seed & 0xffffffff, seed >> 32)
  pair stream  = counter (id_i, id_j, step & 0xffffffff, (step >> 32) & 0x7fffffff)
                 -> 3 normals for the sampled gas velocity v^B_ij
  DM stream    = counter (id_i, 0, step & 0xffffffff, ((step >> 32) & 0x7fffffff) | 0x80000000)
                 -> words 0 and 3: selection uniform r_i with 52 random bits,
                    r_i = ((w0 << 20 | w3 >> 12) + 0.5) 2^-52 (exact in float64, and an
                    exact 64-bit fixed-point fraction);
                    word 1: cos(theta') = 2u - 1; word 2: phi' = 2 pi u (isotropic direction)
  Bernoulli    = counter (id_i, id_j, step & 0xffffffff, ((step >> 32) & 0x3fffffff) | 0x40000000)
                 (the per-pair variant of the Monte Carlo) -> words 0 and 3: r_ij with 52 bits as r_i;
                 word 1: cos(theta') = 2u - 1; word 2: phi' = 2 pi u
  uniform      = ((word >> 9) + 0.5) * 2^-23, in (0, 1) and exact in float32 and float64
  normals      = Box-Muller: z0, z1 = sqrt(-2 ln u0) (cos, sin)(2 pi u1),
                 z2 = sqrt(-2 ln u2) cos(2 pi u3)

Parity: pinned only statistically (uniformity chi^2, independence across
neighbouring counters, normal moments); published known-answer vectors are
not available here, so bit equality with the GPU is checked in the GPU tests.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four output words (uint64 arrays holding 32-bit values)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
        k0 = (k0 + W0) & MASK32
        k1 = (k1 + W1) & MASK32
    return c0, c1, c2, c3


def to_uniform(word):
    """((word >> 9) + 0.5) * 2^-23 in float64 (exactly representable in float32 too)."""
    return ((np.asarray(word, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def to_uniform52(w_hi, w_lo):
    """((w_hi << 20 | w_lo >> 12) + 0.5) * 2^-52: a float64 uniform in (0, 1) with 52 bits."""
    hi = np.asarray(w_hi, dtype=np.uint64)
    lo = np.asarray(w_lo, dtype=np.uint64)
    k = (hi << np.uint64(20)) | (lo >> np.uint64(12))
    return (k.astype(np.float64) + 0.5) * 2.0 ** -52


def _seed_key(seed):
    seed = int(seed)
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def pair_words(seed, step, id_i, id_j):
    k0, k1 = _seed_key(seed)
    step = int(step)
    return philox4x32_10(id_i, id_j, step & 0xFFFFFFFF, (step >> 32) & 0x7FFFFFFF, k0, k1)


def dm_words(seed, step, id_i):
    k0, k1 = _seed_key(seed)
    step = int(step)
    return philox4x32_10(id_i, 0, step & 0xFFFFFFFF, ((step >> 32) & 0x7FFFFFFF) | 0x80000000, k0, k1)


def pair_normals(seed, step, id_i, id_j):
    """Three standard normals per (i, j) pair by Box-Muller, shape (..., 3)."""
    w = pair_words(seed, step, id_i, id_j)
    u0, u1, u2, u3 = (to_uniform(x) for x in w)
    r0 = np.sqrt(-2.0 * np.log(u0))
    r2 = np.sqrt(-2.0 * np.log(u2))
    return np.stack([r0 * np.cos(2.0 * np.pi * u1), r0 * np.sin(2.0 * np.pi * u1),
                     r2 * np.cos(2.0 * np.pi * u3)], axis=-1)


def dm_uniforms(seed, step, id_i):
    """(r_i, cos theta', phi') per DM particle."""
    w = dm_words(seed, step, id_i)
    r = to_uniform52(w[0], w[3])
    cth = 2.0 * to_uniform(w[1]) - 1.0
    phi = 2.0 * np.pi * to_uniform(w[2])
    return r, cth, phi


def bern_words(seed, step, id_i, id_j):
    k0, k1 = _seed_key(seed)
    step = int(step)
    return philox4x32_10(id_i, id_j, step & 0xFFFFFFFF, ((step >> 32) & 0x3FFFFFFF) | 0x40000000, k0, k1)


def bern_uniforms(seed, step, id_i, id_j):
    """(r_ij, cos theta', phi') per pair of the per-pair Bernoulli stream."""
    w = bern_words(seed, step, id_i, id_j)
    return to_uniform52(w[0], w[3]), 2.0 * to_uniform(w[1]) - 1.0, 2.0 * np.pi * to_uniform(w[2])
