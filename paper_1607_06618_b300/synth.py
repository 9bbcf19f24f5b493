"""Seeded synthetic read sets (stand-ins for the paper's sequencing data sets).

This module holds no arithmetic of the counting method: it only draws reads.  Every random
number comes from one counter-based generator, SplitMix64 (Steele, Lea & Flood, 2014):

    key(seed, stream) = mix64(seed * GOLDEN + stream)
    r(seed, stream, i) = mix64(key(seed, stream) + (i + 1) * GOLDEN)      (mod 2**64)

with GOLDEN = 0x9E3779B97F4A7C15 and mix64 the SplitMix64 output function, so any draw can
be recomputed from (seed, stream, index) alone.  A probability p is tested as
(r >> 32) < floor(p * 2**32).

Reads come back as ASCII bytes (``seq``, uint8) plus ``offsets`` (uint64, nreads + 1); read i
is ``seq[offsets[i]:offsets[i+1]]``.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_ASCII = np.frombuffer(b"ACGT", dtype=np.uint8)
_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        z = np.array([seed], dtype=np.uint64) * GOLDEN + np.uint64(stream)
    return _mix64(z)[0]


def draws(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """r(seed, stream, i) for i in [start, start + n) as uint64."""
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_key(seed, stream) + idx * GOLDEN)


def threshold(p: float) -> np.uint64:
    return np.uint64(int(math.floor(p * 2 ** 32)))


def genome(size: int, seed: int) -> np.ndarray:
    """Uniform random genome as base codes 0..3 (A, C, G, T)."""
    out = np.empty(size, dtype=np.uint8)
    for s in range(0, size, _CHUNK):
        n = min(_CHUNK, size - s)
        out[s:s + n] = (draws(seed, 0, s, n) & np.uint64(3)).astype(np.uint8)
    return out


def uniform_reads(nreads: int, length: int, p_n: float, seed: int):
    """i.i.d. uniform ACGT reads of fixed length, each base N with probability p_n."""
    total = nreads * length
    seq = np.empty(total, dtype=np.uint8)
    tn = threshold(p_n)
    for s in range(0, total, _CHUNK):
        n = min(_CHUNK, total - s)
        r = draws(seed, 0, s, n)
        b = _ASCII[(r & np.uint64(3)).astype(np.intp)]
        b[(r >> np.uint64(32)) < tn] = ord("N")
        seq[s:s + n] = b
    offsets = np.arange(nreads + 1, dtype=np.uint64) * np.uint64(length)
    return seq, offsets


def sampled_reads(gen: np.ndarray, nreads: int, length: int, p_sub: float, seed: int,
                  both_strands: bool = True, p_n: float = 0.0, read_base: int = 0):
    """Fixed-length reads at uniform start positions of ``gen`` (base codes).

    Streams of ``seed``: 0 start position, 1 strand, 2 substitution draw per base,
    3 N draw per base.  A reverse-strand read is the reverse complement of its window.  A
    substituted base becomes one of the other three with equal probability.  ``read_base``
    offsets the read index so that a read set can be drawn in slices.
    """
    G = gen.size
    total = nreads * length
    seq = np.empty(total, dtype=np.uint8)
    ts, tn = threshold(p_sub), threshold(p_n)
    per = max(1, _CHUNK // length)
    cols = np.arange(length, dtype=np.int64)
    for j0 in range(0, nreads, per):
        nr = min(per, nreads - j0)
        starts = (draws(seed, 0, read_base + j0, nr) % np.uint64(G - length + 1)).astype(np.int64)
        codes = gen[starts[:, None] + cols[None, :]]
        if both_strands:
            rev = (draws(seed, 1, read_base + j0, nr) >> np.uint64(63)).astype(bool)
            codes[rev] = 3 - codes[rev, ::-1]
        base_idx = (read_base + j0) * length
        r = draws(seed, 2, base_idx, nr * length).reshape(nr, length)
        hit = (r >> np.uint64(32)) < ts
        shift = (np.uint64(1) + (r & np.uint64(0xFFFF)) % np.uint64(3)).astype(np.uint8)
        codes = np.where(hit, (codes + shift) & 3, codes).astype(np.uint8)
        b = _ASCII[codes.astype(np.intp)]
        if p_n > 0:
            rn = draws(seed, 3, base_idx, nr * length).reshape(nr, length)
            b[(rn >> np.uint64(32)) < tn] = ord("N")
        seq[j0 * length:(j0 + nr) * length] = b.reshape(-1)
    offsets = np.arange(nreads + 1, dtype=np.uint64) * np.uint64(length)
    return seq, offsets


def tiled_reads(gen: np.ndarray, length: int, step: int):
    """Error-free forward-strand reads of ``length`` starting at every ``step``-th position."""
    starts = np.arange(0, gen.size - length + 1, step, dtype=np.int64)
    codes = gen[starts[:, None] + np.arange(length)[None, :]]
    seq = _ASCII[codes.astype(np.intp)].reshape(-1)
    offsets = np.arange(starts.size + 1, dtype=np.uint64) * np.uint64(length)
    return seq, offsets


def random_small(nreads: int, min_len: int, max_len: int, p_n: float, seed: int,
                 lowercase: bool = False):
    """Tiny read sets of mixed lengths (tests): uniform lengths, uniform bases, N w.p. p_n."""
    lens = (draws(seed, 10, 0, nreads) % np.uint64(max_len - min_len + 1)).astype(np.int64) + min_len
    offsets = np.zeros(nreads + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(lens).astype(np.uint64)
    total = int(offsets[-1])
    r = draws(seed, 11, 0, total)
    seq = _ASCII[(r & np.uint64(3)).astype(np.intp)].copy()
    seq[(r >> np.uint64(32)) < threshold(p_n)] = ord("N")
    if lowercase:
        low = ((r >> np.uint64(8)) & np.uint64(7)) == np.uint64(0)
        isb = seq != ord("N")
        seq[low & isb] += 32
    return seq, offsets


# --- the measured workloads ---------------------------------------------------------------

WORKLOADS = {
    # 20,000 reads x 150 bp, i.i.d. uniform bases, 0.5% N (seed 1); k=32, m=7, 64 bins, min 1
    "uniform-20k-k32": dict(k=32, m=7, nbins=64, min_count=1),
    # 5 Mbp uniform genome (seed 2001); 1e6 x 150 bp reads (30x), both strands, 0.5%
    # substitutions (seed 2002); k=65, m=9, 256 bins, min 2
    "genome5M-30x-k65": dict(k=65, m=9, nbins=256, min_count=2),
}


def workload(name: str, scale: float = 1.0):
    """(seq, offsets, params) of a named workload; ``scale`` < 1 keeps a prefix of the reads."""
    p = dict(WORKLOADS[name])
    if name == "uniform-20k-k32":
        n = max(1, int(round(20000 * scale)))
        seq, off = uniform_reads(n, 150, 0.005, seed=1)
    elif name == "genome5M-30x-k65":
        gen = genome(5_000_000, seed=2001)
        n = max(1, int(round(1_000_000 * scale)))
        seq, off = sampled_reads(gen, n, 150, 0.005, seed=2002)
    else:
        raise KeyError(name)
    return seq, off, p
