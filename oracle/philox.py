"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC 2011) and the Gaussian
block used to probe the inverse Hessian in Algorithm 3.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Round function (from the published definition): with multipliers
M0 = 0xD2511F53, M1 = 0xCD9E8D57 and key increments W0 = 0x9E3779B9,
W1 = 0xBB67AE85,
    (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2,
    c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
ten rounds, the key bumped by (W0, W1) between rounds.

Gaussian block X[p][n]: element i = row * n + col uses counter
(i // 4 low 32 bits, i // 4 high 32 bits, 0, 0) and key (seed low, seed high);
of the four words x0..x3, element i takes Box-Muller pair (x0, x1) when
i % 4 < 2 and (x2, x3) otherwise, with the 24-bit uniforms
u1 = ((a >> 8) + 1) / 2^24 in (0, 1] and u2 = (b >> 8) / 2^24 in [0, 1)
(exact in single and double precision), z = sqrt(-2 ln u1) * cos(2 pi u2)
for the even member and * sin(2 pi u2) for the odd one.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Vectorised Philox4x32-10.  ctr: uint64 array [..., 4] of 32-bit words,
    key: [..., 2].  Returns [..., 4] uint64 holding 32-bit words."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & MASK for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & MASK
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & MASK
    for r in range(10):
        p0 = np.uint64(M0) * c[0]
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        if r < 9:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
    return np.stack(c, axis=-1)


def gaussian_block(seed: int, p: int, n: int) -> np.ndarray:
    """Standard-normal X[p][n] from Philox4x32-10 + Box-Muller (FP64)."""
    total = p * n
    i = np.arange(total, dtype=np.uint64)
    blk = i // np.uint64(4)
    ctr = np.zeros((total, 4), dtype=np.uint64)
    ctr[:, 0] = blk & np.uint64(MASK)
    ctr[:, 1] = blk >> np.uint64(32)
    key = np.zeros((total, 2), dtype=np.uint64)
    key[:, 0] = np.uint64(seed & MASK)
    key[:, 1] = np.uint64((seed >> 32) & MASK)
    w = philox4x32_10(ctr, key)
    lane = (i % np.uint64(4)).astype(np.int64)
    pair = lane // 2
    a = np.where(pair == 0, w[:, 0], w[:, 2]) >> np.uint64(8)
    b = np.where(pair == 0, w[:, 1], w[:, 3]) >> np.uint64(8)
    u1 = (a.astype(np.float64) + 1.0) / 16777216.0
    u2 = b.astype(np.float64) / 16777216.0
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    z = np.where(lane % 2 == 0, rad * np.cos(ang), rad * np.sin(ang))
    return z.reshape(p, n)
