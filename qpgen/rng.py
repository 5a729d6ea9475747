"""Seeded counter-based random streams for the synthetic QP inputs.

Every random quantity of a problem (a matrix pattern, its values, a vector)
draws from its own stream, keyed by ``(seed, tag)``, so that adding a new
quantity never shifts the draws of an existing one.  The bit source is the
Philox-4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11) as shipped in numpy;
its raw 64-bit output is a pure integer function of key and counter, so the
bits are identical on every platform.  The transforms to uniform, normal,
Bernoulli-pattern and integer draws below are written here.

This module holds no solver arithmetic: it only produces inputs.
"""
from __future__ import annotations

import zlib

import numpy as np

_TWO_M53 = 1.0 / 9007199254740992.0  # 2**-53


def _tag_key(tag: str) -> int:
    return zlib.crc32(tag.encode("utf-8")) & 0xFFFFFFFF


class Stream:
    """One independent stream of draws, keyed by ``(seed, tag)``."""

    def __init__(self, seed: int, tag: str):
        self.seed = int(seed)
        self.tag = tag
        self._bits = np.random.Philox(key=[self.seed & 0xFFFFFFFFFFFFFFFF, _tag_key(tag)])

    def raw(self, k: int) -> np.ndarray:
        return self._bits.random_raw(int(k)).astype(np.uint64, copy=False)

    def uniform(self, k: int) -> np.ndarray:
        """k draws from U[0, 1): the top 53 bits of each raw word."""
        return (self.raw(k) >> np.uint64(11)).astype(np.float64) * _TWO_M53

    def uniform_open0(self, k: int) -> np.ndarray:
        """k draws from U(0, 1]."""
        return 1.0 - self.uniform(k)

    def normal(self, k: int, mean: float = 0.0, std: float = 1.0) -> np.ndarray:
        """k draws from N(mean, std^2) by the Box-Muller transform (one
        output per pair of uniforms)."""
        u1 = self.uniform_open0(k)
        u2 = self.uniform(k)
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
        return mean + std * z

    def permutation(self, k: int) -> np.ndarray:
        """A uniformly random permutation of range(k) (argsort of uniform keys;
        ties broken by index, which makes the result deterministic)."""
        return np.argsort(self.uniform(k), kind="stable")


def bernoulli_pattern(stream: Stream, nrows: int, ncols: int, density: float):
    """Positions of the ones of an nrows x ncols iid Bernoulli(density) grid.

    Returns (rows, cols) int64 arrays in row-major order.  The gaps between
    consecutive ones of a flattened iid Bernoulli(p) sequence are iid
    Geometric(p) on {1, 2, ...}; drawing the gaps costs one uniform per one
    instead of one per grid cell, which matters for the 1% x (200000 x 20000)
    grids.  Gap = 1 + floor(log(u) / log(1 - p)) with u ~ U(0, 1].
    """
    total = int(nrows) * int(ncols)
    if total == 0 or density <= 0.0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    if density >= 1.0:
        flat = np.arange(total, dtype=np.int64)
        return flat // ncols, flat % ncols
    log1mp = np.log1p(-density)
    chunks = []
    pos = -1
    block = max(1024, int(total * density * 1.02) + 1024)
    while True:
        u = stream.uniform_open0(block)
        gaps = 1 + np.floor(np.log(u) / log1mp).astype(np.int64)
        p = pos + np.cumsum(gaps)
        keep = p[p < total]
        chunks.append(keep)
        if keep.size < p.size:
            break
        pos = int(p[-1])
        block = max(1024, block // 4)
    flat = np.concatenate(chunks)
    return flat // ncols, flat % ncols
