"""Philox counter-based RNG, written from Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC 2011).

TEST INFRASTRUCTURE ONLY (part of the oracle): imported by tests/, by the
smoke check and by the bench's CPU-baseline leg, never by the product path.

Philox-4xW-R maps a 4-word counter and a 2-word key through R rounds.  One
round multiplies words 0 and 2 by the constants M0 and M1 (full 2W-bit
products split into high and low halves) and permutes:
    out = (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0))
and the key is bumped by the Weyl constants (W0, W1) between rounds.  The
Weyl constants are the fractional parts of the golden ratio and of sqrt(3)
scaled to W bits; the multipliers are the ones published for each width.

Two implementations are kept on purpose:
  * ``philox_generic``: pure-Python integers, any width, used to pin the
    round structure against numpy's independent Philox-4x64-10;
  * ``philox4x32``: numpy-vectorised 4x32-10, used for bulk draws.
"""
from __future__ import annotations

import numpy as np

# Philox-4x32 multipliers and Weyl key increments.
M4x32 = (0xD2511F53, 0xCD9E8D57)
W32 = (0x9E3779B9, 0xBB67AE85)
# Philox-4x64 (only used by the pin against numpy's generator).
M4x64 = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
W64 = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)

ROUNDS = 10


def philox_generic(ctr, key, width=32, mult=M4x32, weyl=W32, rounds=ROUNDS):
    """One Philox-4xW block with Python integers (slow, obviously correct)."""
    mask = (1 << width) - 1
    x0, x1, x2, x3 = (int(c) & mask for c in ctr)
    k0, k1 = (int(k) & mask for k in key)
    for _ in range(rounds):
        p0 = mult[0] * x0
        p1 = mult[1] * x2
        hi0, lo0 = p0 >> width, p0 & mask
        hi1, lo1 = p1 >> width, p1 & mask
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + weyl[0]) & mask
        k1 = (k1 + weyl[1]) & mask
    return (x0, x1, x2, x3)


def philox4x32(ctr: np.ndarray, key) -> np.ndarray:
    """Vectorised Philox-4x32-10.  ctr: uint32 [..., 4]; key: (k0, k1)."""
    c = np.asarray(ctr, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    x0, x1, x2, x3 = (c[..., i].copy() for i in range(4))
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    m0, m1 = np.uint64(M4x32[0]), np.uint64(M4x32[1])
    lo_mask = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    for _ in range(ROUNDS):
        p0 = m0 * x0            # < 2^64: exact in uint64
        p1 = m1 * x2
        hi0, lo0 = p0 >> s32, p0 & lo_mask
        hi1, lo1 = p1 >> s32, p1 & lo_mask
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + np.uint64(W32[0])) & lo_mask
        k1 = (k1 + np.uint64(W32[1])) & lo_mask
    return np.stack([x0, x1, x2, x3], -1).astype(np.uint32)


def seed_key(seed: int):
    """Philox key from a 64-bit seed: (low word, high word)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


# Stream tags (low 4 bits of counter word 3); block index sits above them.
TAG_WRS = 0
TAG_WORLD = 1
TAG_SCREEN = 2
TAG_SHADE = 3
TAG_RIS = 4        # clustered sampling: candidates in a cluster and their pick
TAG_CLUSTER = 5    # clustered training targets: a member light per cluster
TAG_TEMPORAL = 6   # temporal resampling: the pick between the current and previous reservoir


def stream_words(ids: np.ndarray, frame: int, view: int, tag: int,
                 n_words: int, seed: int) -> np.ndarray:
    """uint32 [len(ids), n_words]: word j of stream (id, frame, view, tag).

    Counter = (id, frame, view, (block << 4) | tag); word j comes from block
    j // 4, lane j % 4.
    """
    ids = np.asarray(ids, dtype=np.uint64)
    n_blocks = (n_words + 3) // 4
    out = np.empty((ids.shape[0], n_blocks * 4), np.uint32)
    key = seed_key(seed)
    for b in range(n_blocks):
        ctr = np.empty((ids.shape[0], 4), np.uint64)
        ctr[:, 0] = ids & np.uint64(0xFFFFFFFF)
        ctr[:, 1] = np.uint64(frame & 0xFFFFFFFF)
        ctr[:, 2] = np.uint64(view & 0xFFFFFFFF)
        ctr[:, 3] = np.uint64(((b << 4) | tag) & 0xFFFFFFFF)
        out[:, 4 * b:4 * b + 4] = philox4x32(ctr, key)
    return out[:, :n_words]


def uniform24(r: np.ndarray) -> np.ndarray:
    """float32 in [0, 1): the top 24 bits of a uint32 word times 2^-24."""
    return ((np.asarray(r, np.uint32) >> np.uint32(8)).astype(np.float32)
            * np.float32(2.0 ** -24))
