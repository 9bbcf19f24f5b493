"""CPU oracle for Gerbil's k-mer counting path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline legs (the
cpu_baseline of its line and its sample check, the reference arm, the oracle rate and sample
check of each workload of its configs block, and the per-k oracle rate and sample check of
``--ksweep``) may import this package.  The product library (``paper_1607_06618_b300``) never imports it and
shares no code with it.

``kmer_oracle.cpp`` holds the plain definitions (a ``std::map`` over k-mer strings, the
minimizer partition by its definition, the App. C record encoder); this module compiles it
with g++ and wraps it with ctypes.  ``brute.py`` is a second, pure-Python implementation used
only to pin the C++ oracle on tiny inputs.

Parity status: pinned (see tests/test_oracle_pins.py) -- worked examples of Fig. 1,
Sec. 2.4.2 and App. C, brute force on tiny inputs, closed-form totals and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmer_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

ORDER_KMC2 = 0
ORDER_LEX = 1
ORDER_CGAT = 2
ORDER_ROBERTS = 3
ORDER_RANDOM = 4
ORDER_DFP = 5


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree with g++ (plain -O2, no vectorisation tricks needed)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        vpp = ctypes.POINTER(ctypes.c_void_p)
        lib.oracle_windows.restype = ctypes.c_uint64
        lib.oracle_windows.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int]
        lib.oracle_count.restype = ctypes.c_int
        lib.oracle_count.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, vpp]
        lib.oracle_count_size.restype = ctypes.c_uint64
        lib.oracle_count_size.argtypes = [ctypes.c_void_p]
        lib.oracle_count_copy.restype = None
        lib.oracle_count_copy.argtypes = [ctypes.c_void_p, u64p, u64p]
        lib.oracle_count_free.restype = None
        lib.oracle_count_free.argtypes = [ctypes.c_void_p]
        lib.oracle_partition.restype = ctypes.c_int
        lib.oracle_partition.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_uint32, u32p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_uint32, vpp]
        lib.oracle_partition_size.restype = ctypes.c_uint64
        lib.oracle_partition_dfp.restype = ctypes.c_int
        lib.oracle_partition_dfp.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_uint32, u32p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_uint32, ctypes.c_float, ctypes.c_uint32,
                                             ctypes.POINTER(ctypes.c_void_p)]
        lib.oracle_dfp_ranks.restype = ctypes.c_int
        lib.oracle_dfp_ranks.argtypes = [u8p, u64p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_float, ctypes.c_uint32, u32p]
        lib.oracle_partition_size.argtypes = [ctypes.c_void_p]
        lib.oracle_partition_copy.restype = None
        lib.oracle_partition_copy.argtypes = [ctypes.c_void_p, u64p, u32p, u32p, u64p]
        lib.oracle_partition_free.restype = None
        lib.oracle_partition_free.argtypes = [ctypes.c_void_p]
        lib.oracle_mmer_rank.restype = ctypes.c_uint64
        lib.oracle_mmer_rank.argtypes = [ctypes.c_char_p, ctypes.c_int]
        lib.oracle_bin_of.restype = ctypes.c_uint32
        lib.oracle_bin_of.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u32p]
        lib.oracle_encode_record.restype = ctypes.c_int
        lib.oracle_encode_record.argtypes = [ctypes.c_char_p, ctypes.c_uint32, u8p, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _reads(seq, offsets):
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    if seq.size == 0:
        seq = np.zeros(1, dtype=np.uint8)
    return seq, offsets


def words_for_k(k: int) -> int:
    return (2 * k + 63) // 64


def windows(seq, offsets, k: int) -> int:
    """Number of windows of k determined bases (the closed-form total at min_count=1)."""
    seq, offsets = _reads(seq, offsets)
    return int(_load().oracle_windows(_ptr(seq, ctypes.c_uint8), _ptr(offsets, ctypes.c_uint64),
                                      offsets.size - 1, k))


def count(seq, offsets, k: int, canonical: bool = True, min_count: int = 1,
          npass: int = 1, pass_index: int = 0):
    """Exact k-mer histogram: (keys uint64[n, W], counts uint64[n]) in ascending key order.

    Keys use the base-4 big-integer layout: A=0 C=1 G=2 T=3, first base most significant,
    W = ceil(2k/64) words with word 0 most significant.
    """
    seq, offsets = _reads(seq, offsets)
    lib = _load()
    h = ctypes.c_void_p()
    rc = lib.oracle_count(_ptr(seq, ctypes.c_uint8), _ptr(offsets, ctypes.c_uint64),
                          offsets.size - 1, k, 1 if canonical else 0, min_count, npass,
                          pass_index, ctypes.byref(h))
    if rc != 0:
        raise ValueError("oracle_count rejected its arguments")
    try:
        n = int(lib.oracle_count_size(h))
        W = words_for_k(k)
        keys = np.zeros((n, W), dtype=np.uint64)
        counts = np.zeros(n, dtype=np.uint64)
        if n:
            lib.oracle_count_copy(h, _ptr(keys, ctypes.c_uint64), _ptr(counts, ctypes.c_uint64))
    finally:
        lib.oracle_count_free(h)
    return keys, counts


def dfp_ranks(seq, offsets, m: int, p: float = 0.5, every: int = 16, canonical_min: bool = True):
    """dfp(p) rank of every m-mer value (Sec. 3.1), frequencies from every `every`-th read."""
    seq, offsets = _reads(seq, offsets)
    out = np.zeros(4 ** m, np.uint32)
    rc = _load().oracle_dfp_ranks(_ptr(seq, ctypes.c_uint8), _ptr(offsets, ctypes.c_uint64),
                                  offsets.size - 1, m, 1 if canonical_min else 0, p, every,
                                  _ptr(out, ctypes.c_uint32))
    if rc != 0:
        raise ValueError("oracle_dfp_ranks rejected its arguments")
    return out


def partition(seq, offsets, k: int, m: int, nbins: int, bounds=None, ordering: int = ORDER_KMC2,
              canonical_min: bool = True, lmax: int = 256, dfp_p: float = 0.5, dfp_every: int = 16):
    """Super-mers by definition: dict of arrays pos, nkmers, bin, minimizer (input order)."""
    seq, offsets = _reads(seq, offsets)
    lib = _load()
    bptr = None
    if bounds is not None:
        bounds = np.ascontiguousarray(bounds, dtype=np.uint32)
        bptr = _ptr(bounds, ctypes.c_uint32)
    h = ctypes.c_void_p()
    rc = lib.oracle_partition_dfp(_ptr(seq, ctypes.c_uint8), _ptr(offsets, ctypes.c_uint64),
                                  offsets.size - 1, k, m, nbins, bptr, ordering,
                                  1 if canonical_min else 0, lmax, dfp_p, dfp_every, ctypes.byref(h))
    if rc != 0:
        raise ValueError("oracle_partition rejected its arguments")
    try:
        n = int(lib.oracle_partition_size(h))
        out = {"pos": np.zeros(n, np.uint64), "nkmers": np.zeros(n, np.uint32),
               "bin": np.zeros(n, np.uint32), "minimizer": np.zeros(n, np.uint64)}
        if n:
            lib.oracle_partition_copy(h, _ptr(out["pos"], ctypes.c_uint64),
                                      _ptr(out["nkmers"], ctypes.c_uint32),
                                      _ptr(out["bin"], ctypes.c_uint32),
                                      _ptr(out["minimizer"], ctypes.c_uint64))
    finally:
        lib.oracle_partition_free(h)
    return out


def mmer_rank(s: str, ordering: int = ORDER_KMC2) -> int:
    return int(_load().oracle_mmer_rank(s.encode(), ordering))


def bin_of(minimizer: int, nbins: int, bounds=None) -> int:
    bptr = None
    if bounds is not None:
        bounds = np.ascontiguousarray(bounds, dtype=np.uint32)
        bptr = _ptr(bounds, ctypes.c_uint32)
    return int(_load().oracle_bin_of(minimizer, nbins, bptr))


def encode_record(kmer: str, count: int) -> bytes:
    """App. C output record of one (k-mer, count) pair."""
    buf = np.zeros(8 + len(kmer), dtype=np.uint8)
    n = _load().oracle_encode_record(kmer.encode(), count, _ptr(buf, ctypes.c_uint8), buf.size)
    if n < 0:
        raise ValueError("invalid k-mer")
    return bytes(buf[:n])


def key_to_string(words, k: int) -> str:
    """Inverse of the key layout (for reading results in tests)."""
    v = 0
    for w in words:
        v = (v << 64) | int(w)
    return "".join("ACGT"[(v >> (2 * (k - 1 - i))) & 3] for i in range(k))
