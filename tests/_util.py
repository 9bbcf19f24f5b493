"""Shared helpers for the tests (no method arithmetic: sorting, string conversion, filters)."""
from __future__ import annotations

import numpy as np


def sort_rows(keys: np.ndarray, counts: np.ndarray):
    """Sort (keys[n, W], counts[n]) by key, word 0 most significant."""
    counts = np.asarray(counts).astype(np.uint64)
    keys = np.asarray(keys, dtype=np.uint64)
    if len(counts) == 0:
        return keys.reshape(0, keys.shape[-1] if keys.ndim == 2 else 0), counts
    keys = keys.reshape(len(counts), -1)
    order = np.lexsort(keys.T[::-1])
    return keys[order], counts[order]


def assert_same_rows(got, want):
    gk, gc = sort_rows(*got)
    wk, wc = sort_rows(*want)
    assert gk.shape == wk.shape, f"row count {gk.shape[0]} != {wk.shape[0]}"
    assert np.array_equal(gk, wk), "keys differ"
    assert np.array_equal(gc, wc), "counts differ"


def keys_to_ascii(keys: np.ndarray, k: int) -> np.ndarray:
    """[n, W] keys -> [n, k] ASCII bytes (A=0 C=1 G=2 T=3, first base most significant)."""
    keys = np.asarray(keys, dtype=np.uint64)
    n, W = keys.shape
    out = np.empty((n, k), dtype=np.uint8)
    lut = np.frombuffer(b"ACGT", dtype=np.uint8)
    for i in range(k):
        bit = 2 * (k - 1 - i)          # bit offset of base i in the 64W-bit integer
        word = W - 1 - bit // 64
        sh = np.uint64(bit % 64)
        out[:, i] = lut[((keys[:, word] >> sh) & np.uint64(3)).astype(np.intp)]
    return out


def fnv1a64_rows(ascii_rows: np.ndarray) -> np.ndarray:
    """FNV-1a 64 of each row of bytes (the oracle's pass filter, vectorised)."""
    h = np.full(ascii_rows.shape[0], 0xcbf29ce484222325, dtype=np.uint64)
    prime = np.uint64(0x100000001b3)
    with np.errstate(over="ignore"):
        for i in range(ascii_rows.shape[1]):
            h ^= ascii_rows[:, i].astype(np.uint64)
            h *= prime
    return h


def reads_from_strings(strings):
    seq = np.frombuffer("".join(strings).encode("latin-1"), dtype=np.uint8).copy()
    offs = np.zeros(len(strings) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(s) for s in strings])
    return seq, offs


def revcomp_reads(seq: np.ndarray, offs: np.ndarray):
    """Reverse-complement every read (bytes other than ACGTacgt kept as they are)."""
    table = np.arange(256, dtype=np.uint8)
    for a, b in zip(b"ACGTacgt", b"TGCAtgca"):
        table[a] = b
    comp = table[seq]
    out = np.empty_like(seq)
    o = offs.astype(np.int64)
    for i in range(len(o) - 1):
        out[o[i]:o[i + 1]] = comp[o[i]:o[i + 1]][::-1]
    return out, offs


_FNV_BASIS = 0xcbf29ce484222325 - (1 << 64)  # as a signed 64-bit integer
_FNV_PRIME = 0x100000001b3


def fnv1a64_device(keys, k: int, rows_per_chunk: int = 1 << 25):
    """FNV-1a 64 of every key's ASCII string (the oracle's pass filter), for keys int64[n, W]
    on a CUDA device; int64[n] (two's complement of the unsigned hash).  Torch wraps int64
    products modulo 2^64, which is the hash's arithmetic."""
    import torch
    n, W = keys.shape
    lut = torch.tensor([ord(c) for c in "ACGT"], dtype=torch.int64, device=keys.device)
    out = torch.empty(n, dtype=torch.int64, device=keys.device)
    for a in range(0, n, rows_per_chunk):
        kk = keys[a:a + rows_per_chunk]
        h = torch.full((kk.shape[0],), _FNV_BASIS, dtype=torch.int64, device=keys.device)
        for i in range(k):
            bit = 2 * (k - 1 - i)
            base = (kk[:, W - 1 - bit // 64] >> (bit % 64)) & 3  # masked: the shift's sign bits go
            h = (h ^ lut[base]) * _FNV_PRIME
        out[a:a + kk.shape[0]] = h
    return out


def device_pass_rows(keys, counts, k: int, npass: int, pass_index: int = 0):
    """Host copies of the device rows whose key is in the oracle's pass (npass a power of two,
    so the unsigned residue is the low bits of the signed hash)."""
    import torch
    assert npass & (npass - 1) == 0
    h = fnv1a64_device(keys, k)
    sel = torch.nonzero((h & (npass - 1)) == pass_index).flatten()
    return (keys[sel].cpu().numpy().view(np.uint64),
            counts[sel].cpu().numpy().view(np.uint32).astype(np.uint64))


def device_digest(keys, counts, k: int):
    """Order-independent digest of device rows: (rows, sum of counts, wrapping sum of
    FNV(key) * (count + 1)).  Equal results give equal digests in any row order."""
    import torch
    h = fnv1a64_device(keys, k)
    c = counts.to(torch.int64) & 0xFFFFFFFF
    return (int(keys.shape[0]), int(c.sum().item()), int((h * (c + 1)).sum().item()))
