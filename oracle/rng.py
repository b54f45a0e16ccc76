"""Counter-based generators, from their published definitions (oracle).

TEST INFRASTRUCTURE ONLY.

SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output i of the stream seeded with s is
mix(s + (i + 1) * 0x9E3779B97F4A7C15) with the finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
It gives the sampler pre-compute its Rademacher probe: r_i = +1 if the low bit
of output i is 1, else -1 (the paper gives no probe for the Lanczos run of
Sec. 3.3).

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC 2011): 10 rounds on a 4 x 32-bit counter with a 2 x 32-bit key.
One round: (hi0, lo0) = M0 * x0, (hi1, lo1) = M1 * x2 (64-bit products),
x <- (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); between rounds the key is
bumped by the Weyl constants.  Normals come from Box-Muller on pairs of
uniforms u = (r + 0.5) / 2^32.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_output(seed: int, i: int) -> int:
    return splitmix64_mix((seed + (i + 1) * GOLDEN_GAMMA) & _M64)


def splitmix64_outputs(seed: int, count: int) -> np.ndarray:
    """Outputs 0..count-1 of the SplitMix64 stream (vectorised, uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & _M64) + i * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def rademacher_probe(seed: int, m: int) -> np.ndarray:
    """r_i = +1 if output i has its low bit set, else -1 (length m)."""
    z = splitmix64_outputs(seed, m)
    return np.where((z & np.uint64(1)) == np.uint64(1), 1.0, -1.0)


PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32-10 on uint32 arrays: ctr (..., 4), key (..., 2) -> (..., 4)."""
    x = [np.asarray(ctr[..., i], dtype=np.uint64) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64)
    k1 = np.asarray(key[..., 1], dtype=np.uint64)
    m32 = np.uint64(_M32)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & m32
            k1 = (k1 + np.uint64(PHILOX_W1)) & m32
        p0 = np.uint64(PHILOX_M0) * x[0]
        p1 = np.uint64(PHILOX_M1) * x[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & m32
        hi1, lo1 = p1 >> np.uint64(32), p1 & m32
        x = [(hi1 ^ x[1] ^ k0) & m32, lo1, (hi0 ^ x[3] ^ k1) & m32, lo0]
    return np.stack(x, axis=-1).astype(np.uint32)


def philox_normals(seed: int, count: int) -> np.ndarray:
    """count standard normals: element e uses counter (e // 4, 0, 0, 0) split
    into 32-bit words (lo, hi of the 64-bit block index), key = (seed lo, seed hi);
    the 4 outputs give two Box-Muller pairs (r0, r1) and (r2, r3) and element e
    takes component e % 4: (cos, sin) of pair 0, then of pair 1."""
    blocks = (count + 3) // 4
    b = np.arange(blocks, dtype=np.uint64)
    ctr = np.zeros((blocks, 4), dtype=np.uint64)
    ctr[:, 0] = b & np.uint64(_M32)
    ctr[:, 1] = b >> np.uint64(32)
    key = np.zeros((blocks, 2), dtype=np.uint64)
    key[:, 0] = seed & _M32
    key[:, 1] = (seed >> 32) & _M32
    r = philox4x32_10(ctr, key).astype(np.float64)
    u = (r + 0.5) / 4294967296.0
    out = np.zeros((blocks, 4))
    for p in range(2):
        u1, u2 = u[:, 2 * p], u[:, 2 * p + 1]
        rad = np.sqrt(-2.0 * np.log(u1))
        out[:, 2 * p] = rad * np.cos(2.0 * np.pi * u2)
        out[:, 2 * p + 1] = rad * np.sin(2.0 * np.pi * u2)
    return out.ravel()[:count]
