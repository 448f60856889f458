"""Counter-based random numbers written from their published definitions.

* Philox-4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11.  A 4x32-bit counter is mixed with a 2x32-bit key by ten
  rounds; each round takes two 32x32->64 bit products of counter words with the
  multipliers 0xD2511F53 and 0xCD9E8D57, XORs the high halves with the other
  two counter words and the key, and permutes the words.  The key is bumped by
  the Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
* SplitMix64: Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA'14 (the finaliser with shifts 30/27/31).

Everything is vectorised numpy on uint32/uint64 and bit-reproducible on any
host.  This module contains no part of the predistortion method.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox-4x32 with 10 rounds.

    ctr: uint32 array [..., 4]; key: uint32 array broadcastable to [..., 2].
    Returns uint32 [..., 4].
    """
    ctr = np.asarray(ctr, dtype=np.uint32)
    key = np.asarray(key, dtype=np.uint32)
    c0, c1, c2, c3 = (ctr[..., i].astype(np.uint64) for i in range(4))
    k0 = np.broadcast_to(key[..., 0], c0.shape).astype(np.uint32)
    k1 = np.broadcast_to(key[..., 1], c0.shape).astype(np.uint32)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd:
                k0 = (k0 + _W0).astype(np.uint32)
                k1 = (k1 + _W1).astype(np.uint32)
            p0 = _M0 * c0
            p1 = _M1 * c2
            hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
            hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
            c0, c1, c2, c3 = (hi1 ^ c1 ^ k0.astype(np.uint64),
                              lo1,
                              hi0 ^ c3 ^ k1.astype(np.uint64),
                              lo0)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state x (the state is advanced first)."""
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _tag_hash(tag: str) -> int:
    """FNV-1a 64-bit of the tag text, so that named streams are independent."""
    h = 0xCBF29CE484222325
    for b in tag.encode():
        h = ((h ^ b) * 0x100000001B3) & ((1 << 64) - 1)
    return h


class Stream:
    """A named, seeded stream: key = SplitMix64(seed, tag), counter = index.

    Every draw advances a 64-bit block counter held in counter words 0-1, so
    the n-th value of a stream never depends on how earlier draws were split.
    """

    def __init__(self, seed: int, tag: str):
        k = splitmix64((int(seed) * 0x9E3779B97F4A7C15 ^ _tag_hash(tag)) & ((1 << 64) - 1))
        self.key = np.array([k & 0xFFFFFFFF, k >> 32], dtype=np.uint32)
        self.block = 0

    def u32(self, n: int) -> np.ndarray:
        """n uniform 32-bit words."""
        nblk = (n + 3) // 4
        idx = np.arange(self.block, self.block + nblk, dtype=np.uint64)
        self.block += nblk
        ctr = np.zeros((nblk, 4), dtype=np.uint32)
        ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
        ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
        return philox4x32_10(ctr, self.key).reshape(-1)[:n]

    def uniform(self, n: int) -> np.ndarray:
        """n doubles uniform on the open interval (0, 1), 53-bit resolution."""
        w = self.u32(2 * n).astype(np.uint64).reshape(n, 2)
        bits = ((w[:, 0] << np.uint64(21)) ^ (w[:, 1] >> np.uint64(11))) & np.uint64((1 << 53) - 1)
        return (bits.astype(np.float64) + 0.5) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n standard normal doubles by the Box-Muller transform."""
        m = (n + 1) // 2
        u = self.uniform(2 * m).reshape(m, 2)
        r = np.sqrt(-2.0 * np.log(u[:, 0]))
        t = 2.0 * np.pi * u[:, 1]
        return np.stack([r * np.cos(t), r * np.sin(t)], axis=1).reshape(-1)[:n]
