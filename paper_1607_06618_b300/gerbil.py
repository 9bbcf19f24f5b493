"""Thin ctypes binding of ``libgerbil.so`` (include/gerbil.h) -- argument marshalling only.

Every step of the path runs in the CUDA library; this module passes pointers and sizes.
Device memory and streams come from PyTorch (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``).  There is no CPU fallback: if the library is
missing or no CUDA device is usable, calls raise ``GerbilError``.

The module-level functions carry the C-ABI's names; ``Context``/``Bins``/``Counts`` wrap the
handles for convenient lifetime management.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgerbil.so")

GERBIL_OK = 0
GERBIL_E_INVAL = 1
GERBIL_E_UNSUPPORTED = 2
GERBIL_E_NOMEM = 3
GERBIL_E_OVERFLOW = 4
GERBIL_E_TIMEOUT = 5
GERBIL_E_CUDA = 6
GERBIL_E_STATE = 7
GERBIL_ORDER_KMC2 = 0
GERBIL_ORDER_LEX = 1

# every symbol the header declares (checked by tests/test_abi.py)
ABI_SYMBOLS = (
    "gerbil_wait_selftest", "gerbil_opts_default", "gerbil_strerror", "gerbil_last_error", "gerbil_create",
    "gerbil_destroy", "gerbil_partition", "gerbil_bins_info", "gerbil_bin_stats",
    "gerbil_bins_export", "gerbil_bins_free", "gerbil_count", "gerbil_count_batch",
    "gerbil_counts_info", "gerbil_counts_view", "gerbil_counts_to_host", "gerbil_counts_free",
    "gerbil_profile", "gerbil_get_phase_times", "gerbil_count_small_noalloc", "gerbil_membench",
    "gerbil_trim", "gerbil_device_bytes", "gerbil_server_create", "gerbil_server_submit",
    "gerbil_server_wait", "gerbil_server_get_stats", "gerbil_server_destroy",
    "gerbil_autotune", "gerbil_set_tuning", "gerbil_get_tuning", "gerbil_encode_records",
    "gerbil_forget_ratio", "gerbil_probe_stats", "gerbil_get_probe_stats",
    "gerbil_server_last_error",
)


class GerbilError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class gerbil_reads(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("nreads", ctypes.c_uint64), ("on_device", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class gerbil_opts(ctypes.Structure):
    _fields_ = [("canonical", ctypes.c_int32), ("ordering", ctypes.c_int32),
                ("canonical_minimizer", ctypes.c_int32), ("supermer_cap", ctypes.c_uint32),
                ("bin_bounds", ctypes.c_void_p), ("max_probes", ctypes.c_uint32),
                ("load_factor", ctypes.c_float), ("distinct_ratio", ctypes.c_float),
                ("overflow_slots", ctypes.c_uint32), ("persistent", ctypes.c_int32),
                ("ring_slots", ctypes.c_uint32), ("fused", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("max_table_mib", ctypes.c_uint32),
                ("autotune", ctypes.c_uint32), ("graph", ctypes.c_uint32),
                ("dfp_pivot", ctypes.c_float), ("dfp_sample", ctypes.c_uint32),
                ("probe_scheme", ctypes.c_int32), ("item_kmers", ctypes.c_uint32),
                ("sorted_output", ctypes.c_int32), ("claim_first", ctypes.c_int32)]


TUNE_CLASSES = 4


class gerbil_tuning(ctypes.Structure):
    _fields_ = [("load_factor", ctypes.c_float * TUNE_CLASSES),
                ("class_bytes", ctypes.c_uint64 * (TUNE_CLASSES - 1)),
                ("fused", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("k_words", ctypes.c_int32), ("samples", ctypes.c_uint32),
                ("ns_per_kmer", ctypes.c_double),
                ("probe_scheme", ctypes.c_int32), ("item_kmers", ctypes.c_uint32)]

    def as_dict(self):
        return {"load_factor": [float(x) for x in self.load_factor],
                "class_bytes": [int(x) for x in self.class_bytes],
                "fused": int(self.fused), "schedule": int(self.schedule),
                "k_words": int(self.k_words), "samples": int(self.samples),
                "ns_per_kmer": float(self.ns_per_kmer),
                "probe_scheme": int(self.probe_scheme), "item_kmers": int(self.item_kmers)}

    @classmethod
    def from_dict(cls, d):
        t = cls()
        for i, x in enumerate(d["load_factor"]):
            t.load_factor[i] = x
        for i, x in enumerate(d.get("class_bytes", [])):
            t.class_bytes[i] = x
        t.fused, t.schedule = d["fused"], d["schedule"]
        t.k_words, t.samples = d.get("k_words", 0), d.get("samples", 0)
        t.ns_per_kmer = d.get("ns_per_kmer", 0.0)
        t.probe_scheme = d.get("probe_scheme", 0)
        t.item_kmers = d.get("item_kmers", 256)
        return t


class gerbil_count_stats(ctypes.Structure):
    _fields_ = [("occurrences", ctypes.c_uint64), ("distinct", ctypes.c_uint64),
                ("emitted", ctypes.c_uint64), ("overflowed", ctypes.c_uint64),
                ("table_slots", ctypes.c_uint64), ("retries", ctypes.c_uint32),
                ("bins", ctypes.c_uint32), ("groups", ctypes.c_uint32), ("sorted", ctypes.c_uint32)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class gerbil_phase_times(ctypes.Structure):
    _fields_ = [("encode_ms", ctypes.c_double), ("supermer_ms", ctypes.c_double),
                ("clear_ms", ctypes.c_double), ("insert_ms", ctypes.c_double),
                ("compact_ms", ctypes.c_double), ("overflow_ms", ctypes.c_double),
                ("insert_launches", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("calls", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64)]

    def as_dict(self):
        return {name: (float if t is ctypes.c_double else int)(getattr(self, name))
                for name, t in self._fields_}


class gerbil_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("kmers", ctypes.c_uint64),
                ("max_concurrent", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("kernel_launches", ctypes.c_uint64)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_ if name != "reserved"}


class gerbil_job_times(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("worker", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {"queue_ms": self.queue_ms, "run_ms": self.run_ms, "latency_ms": self.latency_ms,
                "worker": int(self.worker)}


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy


def slot_bytes(k: int) -> int:
    """Bytes of one hash-table slot at k (include/gerbil.h table layout): the meta word with
    the key's low 30 bits, then the rest of the key in 63-bit chunks, rounded to 16 bytes."""
    ws = 1 if 2 * k <= 30 + 63 else (2 * k - 30 + 62) // 63
    return 8 * ((ws + 2) & ~1)
_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree CUDA library (built by ``build.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise GerbilError(GERBIL_E_CUDA, "libgerbil.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    P, U64, U32, I32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "gerbil_opts_default": (None, [ctypes.POINTER(gerbil_opts)]),
        "gerbil_strerror": (ctypes.c_char_p, [I32]),
        "gerbil_last_error": (ctypes.c_char_p, [P]),
        "gerbil_create": (I32, [PP, I32, U64, P]),
        "gerbil_destroy": (None, [P]),
        "gerbil_partition": (I32, [P, ctypes.POINTER(gerbil_reads), I32, I32, I32,
                                   ctypes.POINTER(gerbil_opts), PP]),
        "gerbil_bins_info": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                   ctypes.POINTER(I32), ctypes.POINTER(U64), ctypes.POINTER(U64)]),
        "gerbil_bin_stats": (I32, [P, I32, ctypes.POINTER(U64), ctypes.POINTER(U64),
                                   ctypes.POINTER(U64)]),
        "gerbil_bins_export": (I32, [P, P, P, P, U64]),
        "gerbil_bins_free": (None, [P]),
        "gerbil_count": (I32, [P, P, I32, I32, U32, ctypes.POINTER(gerbil_opts), PP]),
        "gerbil_count_batch": (I32, [P, P, P, I32, I32, U32, ctypes.POINTER(gerbil_opts), PP]),
        "gerbil_counts_info": (I32, [P, ctypes.POINTER(U64), ctypes.POINTER(I32),
                                     ctypes.POINTER(gerbil_count_stats)]),
        "gerbil_counts_view": (I32, [P, ctypes.POINTER(U64), ctypes.POINTER(I32), PP, PP]),
        "gerbil_counts_to_host": (I32, [P, P, P, U64]),
        "gerbil_counts_free": (None, [P]),
        "gerbil_profile": (I32, [P, I32]),
        "gerbil_trim": (I32, [P]),
        "gerbil_forget_ratio": (I32, [P]),
        "gerbil_probe_stats": (I32, [P, I32]),
        "gerbil_get_probe_stats": (I32, [P, ctypes.POINTER(U64), ctypes.POINTER(U64)]),
        "gerbil_encode_records": (I32, [P, I32, P, U64, I32, ctypes.POINTER(U64)]),
        "gerbil_autotune": (I32, [P, P, I32, U32, ctypes.POINTER(gerbil_opts),
                                  ctypes.POINTER(gerbil_tuning)]),
        "gerbil_set_tuning": (I32, [P, I32, ctypes.POINTER(gerbil_tuning)]),
        "gerbil_get_tuning": (I32, [P, I32, ctypes.POINTER(gerbil_tuning)]),
        "gerbil_device_bytes": (U64, [P]),
        "gerbil_server_create": (I32, [PP, I32, U64, I32]),
        "gerbil_server_submit": (I32, [P, ctypes.POINTER(gerbil_reads), I32, I32, I32, U32,
                                       ctypes.POINTER(gerbil_opts), ctypes.POINTER(U64)]),
        "gerbil_server_wait": (I32, [P, U64, ctypes.c_int64, PP, ctypes.POINTER(gerbil_job_times)]),
        "gerbil_server_get_stats": (I32, [P, ctypes.POINTER(gerbil_server_stats)]),
        "gerbil_server_destroy": (None, [P]),
        "gerbil_server_last_error": (ctypes.c_char_p, [P]),
        "gerbil_membench": (I32, [P, U64, I32, U64, ctypes.POINTER(ctypes.c_double)]),
        "gerbil_wait_selftest": (I32, [P, U64]),
        "gerbil_count_small_noalloc": (I32, [P, P, U64, U64, I32, U32, I32, P, P, U64,
                                             ctypes.POINTER(U64), P]),
        "gerbil_get_phase_times": (I32, [P, ctypes.POINTER(gerbil_phase_times)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != GERBIL_OK:
        lib = load()
        msg = lib.gerbil_strerror(status).decode()
        if ctx:
            detail = lib.gerbil_last_error(ctx).decode()
            if detail:
                msg += ": " + detail
        raise GerbilError(status, msg)


def default_opts(**kw) -> gerbil_opts:
    o = gerbil_opts()
    load().gerbil_opts_default(ctypes.byref(o))
    for key, val in kw.items():
        if key == "bin_bounds":
            continue
        setattr(o, key, val)
    return o


# ---- C-ABI names ------------------------------------------------------------------------
def gerbil_create(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int | None = None):
    h = ctypes.c_void_p()
    _check(load().gerbil_create(ctypes.byref(h), device, hbm_budget_bytes, cuda_stream))
    return h


def gerbil_destroy(ctx):
    load().gerbil_destroy(ctx)


def gerbil_profile(ctx, enable: bool):
    _check(load().gerbil_profile(ctx, 1 if enable else 0), ctx)


def gerbil_get_phase_times(ctx):
    t = gerbil_phase_times()
    _check(load().gerbil_get_phase_times(ctx, ctypes.byref(t)), ctx)
    return t.as_dict()


def gerbil_membench(ctx, nbytes: int, op: int, per_thread: int) -> float:
    g = ctypes.c_double()
    _check(load().gerbil_membench(ctx, nbytes, op, per_thread, ctypes.byref(g)), ctx)
    return g.value


def _reads_struct(seq, offsets):
    """Marshal reads: torch CUDA tensors (device pointers) or numpy arrays (host pointers)."""
    r = gerbil_reads()
    keep = (seq, offsets)
    if hasattr(seq, "data_ptr"):
        r.seq, r.offsets, r.on_device = seq.data_ptr(), offsets.data_ptr(), 1 if seq.is_cuda else 0
        r.nreads = offsets.numel() - 1
    else:
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        keep = (seq, offsets)
        r.seq, r.offsets, r.on_device = seq.ctypes.data, offsets.ctypes.data, 0
        r.nreads = offsets.size - 1
    return r, keep


def gerbil_partition(ctx, seq, offsets, k: int, m: int, nbins: int, opts: gerbil_opts | None = None,
                     bin_bounds=None):
    r, keep = _reads_struct(seq, offsets)
    o = opts if opts is not None else default_opts()
    bb = None
    if bin_bounds is not None:
        bb = np.ascontiguousarray(bin_bounds, dtype=np.uint32)
        o.bin_bounds = bb.ctypes.data
    h = ctypes.c_void_p()
    st = load().gerbil_partition(ctx, ctypes.byref(r), k, m, nbins, ctypes.byref(o), ctypes.byref(h))
    o.bin_bounds = None
    del keep, bb
    _check(st, ctx)
    return h


def gerbil_bins_info(bins):
    k, m, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ns, nk = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().gerbil_bins_info(bins, ctypes.byref(k), ctypes.byref(m), ctypes.byref(nb),
                                   ctypes.byref(ns), ctypes.byref(nk)))
    return {"k": k.value, "m": m.value, "nbins": nb.value, "n_supermers": ns.value,
            "n_kmers": nk.value}


def gerbil_bin_stats(bins, b: int):
    ns, nbases, nk = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().gerbil_bin_stats(bins, b, ctypes.byref(ns), ctypes.byref(nbases), ctypes.byref(nk)))
    return ns.value, nbases.value, nk.value


def gerbil_bins_export(bins):
    n = gerbil_bins_info(bins)["n_supermers"]
    pos = np.zeros(max(n, 1), np.uint64)
    nk = np.zeros(max(n, 1), np.uint32)
    b = np.zeros(max(n, 1), np.uint32)
    _check(load().gerbil_bins_export(bins, pos.ctypes.data, nk.ctypes.data, b.ctypes.data, pos.size))
    return {"pos": pos[:n], "nkmers": nk[:n], "bin": b[:n]}


def gerbil_bins_free(bins):
    load().gerbil_bins_free(bins)


def gerbil_count(ctx, bins, b: int, k: int, min_count: int, opts: gerbil_opts | None = None):
    o = opts if opts is not None else default_opts()
    h = ctypes.c_void_p()
    _check(load().gerbil_count(ctx, bins, b, k, min_count, ctypes.byref(o), ctypes.byref(h)), ctx)
    return h


def gerbil_count_batch(ctx, bins, bin_list, k: int, min_count: int, opts: gerbil_opts | None = None):
    o = opts if opts is not None else default_opts()
    h = ctypes.c_void_p()
    if bin_list is None:
        st = load().gerbil_count_batch(ctx, bins, None, 0, k, min_count, ctypes.byref(o), ctypes.byref(h))
    else:
        arr = np.ascontiguousarray(bin_list, dtype=np.int32)
        st = load().gerbil_count_batch(ctx, bins, arr.ctypes.data, arr.size, k, min_count,
                                       ctypes.byref(o), ctypes.byref(h))
    _check(st, ctx)
    return h


def gerbil_counts_info(counts):
    n, w = ctypes.c_uint64(), ctypes.c_int()
    s = gerbil_count_stats()
    _check(load().gerbil_counts_info(counts, ctypes.byref(n), ctypes.byref(w), ctypes.byref(s)))
    return n.value, w.value, s.as_dict()


def gerbil_counts_view(counts):
    """(rows, key words, keys device pointer, counts device pointer) of a result."""
    n, w = ctypes.c_uint64(), ctypes.c_int()
    kp, cp = ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().gerbil_counts_view(counts, ctypes.byref(n), ctypes.byref(w), ctypes.byref(kp),
                                     ctypes.byref(cp)))
    return n.value, w.value, kp.value or 0, cp.value or 0


def gerbil_counts_to_host(counts, keys_out=None, counts_out=None):
    n, W, _ = gerbil_counts_info(counts)
    keys = keys_out if keys_out is not None else np.zeros((max(n, 1), W), np.uint64)
    cnt = counts_out if counts_out is not None else np.zeros(max(n, 1), np.uint32)
    _check(load().gerbil_counts_to_host(counts, keys.ctypes.data, cnt.ctypes.data, min(len(cnt), len(keys))))
    return keys[:n], cnt[:n]


def gerbil_counts_free(counts):
    load().gerbil_counts_free(counts)


def gerbil_count_small_noalloc(seq, offsets, k: int, min_count: int, canonical: bool,
                               keys_out, counts_out, stream: int | None = None):
    """Counts a small read set with no device allocation inside the library.

    seq (uint8[n]) and offsets (int64[nreads + 1]) are contiguous torch CUDA tensors;
    keys_out (int64, at least cap * W elements, W = ceil(2k/64)) and counts_out (int32[cap])
    are caller-allocated contiguous CUDA tensors on the same device.  Returns the number of
    rows.  Tensors of another shape, type or device raise ValueError before the call, since
    the library writes up to cap * W key words and reads offsets[nreads] bases.
    """
    import torch
    W = (2 * k + 63) // 64
    need = ((seq, torch.uint8, "seq"), (offsets, torch.int64, "offsets"),
            (keys_out, torch.int64, "keys_out"), (counts_out, torch.int32, "counts_out"))
    for t, dt, name in need:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.dtype != dt:
            raise ValueError("%s must be %s, not %s" % (name, dt, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if t.device != seq.device:
            raise ValueError("%s is on %s, seq on %s" % (name, t.device, seq.device))
    if offsets.dim() != 1 or offsets.numel() < 1:
        raise ValueError("offsets must hold nreads + 1 >= 1 entries")
    cap = counts_out.numel()
    if keys_out.numel() < cap * W:
        raise ValueError("keys_out holds %d words; %d rows of %d words need %d"
                         % (keys_out.numel(), cap, W, cap * W))
    nreads = offsets.numel() - 1
    first, nbases = (int(x) for x in offsets[[0, -1]].tolist())
    if first < 0 or nbases > seq.numel():
        raise ValueError("offsets run outside seq (%d..%d of %d bases)" % (first, nbases, seq.numel()))
    n = ctypes.c_uint64()
    st = load().gerbil_count_small_noalloc(seq.data_ptr(), offsets.data_ptr(), nreads, nbases, k,
                                           min_count, 1 if canonical else 0, keys_out.data_ptr(),
                                           counts_out.data_ptr(), cap, ctypes.byref(n), stream)
    _check(st)
    return n.value


def gerbil_autotune(ctx, bins, k: int, min_count: int, opts: gerbil_opts | None = None) -> dict:
    t = gerbil_tuning()
    o = opts if opts is not None else default_opts()
    _check(load().gerbil_autotune(ctx, bins, k, min_count, ctypes.byref(o), ctypes.byref(t)), ctx)
    return t.as_dict()


def gerbil_set_tuning(ctx, k: int, tuning: dict | None):
    t = gerbil_tuning.from_dict(tuning) if tuning is not None else None
    _check(load().gerbil_set_tuning(ctx, k, ctypes.byref(t) if t is not None else None), ctx)


def gerbil_get_tuning(ctx, k: int) -> dict | None:
    t = gerbil_tuning()
    st = load().gerbil_get_tuning(ctx, k, ctypes.byref(t))
    if st == GERBIL_E_STATE:
        return None
    _check(st, ctx)
    return t.as_dict()


def gerbil_encode_records(counts, k: int, out=None, cap: int = 0, out_on_device: int = 0) -> int:
    """App. C records of a result into ``out`` (a pointer), or only their size when out is None."""
    nb = ctypes.c_uint64()
    _check(load().gerbil_encode_records(counts, k, out, cap, out_on_device, ctypes.byref(nb)))
    return nb.value


def gerbil_wait_selftest(ctx, wait_ns: int) -> int:
    """Status of one bounded wait on a flag that nothing sets (GERBIL_E_TIMEOUT expected)."""
    return load().gerbil_wait_selftest(ctx, wait_ns)


def gerbil_trim(ctx):
    _check(load().gerbil_trim(ctx), ctx)


def gerbil_device_bytes(ctx) -> int:
    return int(load().gerbil_device_bytes(ctx))


def gerbil_server_create(device: int, hbm_budget_bytes: int, slots: int):
    h = ctypes.c_void_p()
    _check(load().gerbil_server_create(ctypes.byref(h), device, hbm_budget_bytes, slots))
    return h


def gerbil_server_submit(server, seq, offsets, k, m, nbins, min_count, opts=None, bin_bounds=None):
    r, keep = _reads_struct(seq, offsets)
    o = opts if opts is not None else default_opts()
    bb = None
    if bin_bounds is not None:
        bb = np.ascontiguousarray(bin_bounds, dtype=np.uint32)
        o.bin_bounds = bb.ctypes.data
    jid = ctypes.c_uint64()
    st = load().gerbil_server_submit(server, ctypes.byref(r), k, m, nbins, min_count,
                                     ctypes.byref(o), ctypes.byref(jid))
    o.bin_bounds = None
    _check(st)
    return jid.value


def gerbil_server_wait(server, job_id: int, timeout_ms: int = -1):
    h = ctypes.c_void_p()
    t = gerbil_job_times()
    st = load().gerbil_server_wait(server, job_id, timeout_ms, ctypes.byref(h), ctypes.byref(t))
    if st not in (GERBIL_OK, GERBIL_E_TIMEOUT):
        raise GerbilError(st, load().gerbil_server_last_error(server).decode())
    _check(st)
    return h, t.as_dict()


def gerbil_server_get_stats(server):
    s = gerbil_server_stats()
    _check(load().gerbil_server_get_stats(server, ctypes.byref(s)))
    return s.as_dict()


def gerbil_server_destroy(server):
    load().gerbil_server_destroy(server)


# ---- handle wrappers ----------------------------------------------------------------------
class _DeviceArray:
    """Exposes a device pointer to torch through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (ptr, False), "version": 2, "strides": None}
        self._owner = owner


class Counts:
    def __init__(self, handle, ctx):
        self.handle, self.ctx = handle, ctx
        ctx._children.add(self)

    def info(self):
        return gerbil_counts_info(self.handle)

    def __len__(self):
        return self.info()[0]

    def to_host(self):
        return gerbil_counts_to_host(self.handle)

    def encode_records(self, k: int, device: bool = False):
        """App. C output records of every row: a numpy uint8 array, or a torch uint8 CUDA
        tensor with device=True."""
        n = gerbil_encode_records(self.handle, k)
        if device:
            import torch
            buf = torch.empty(max(1, n), dtype=torch.uint8, device=torch.device("cuda", self.ctx.device))
            gerbil_encode_records(self.handle, k, buf.data_ptr(), n, 1)
            return buf[:n]
        buf = np.empty(max(1, n), dtype=np.uint8)
        gerbil_encode_records(self.handle, k, buf.ctypes.data, n, 0)
        return buf[:n]

    def torch_views(self):
        """(keys int64[n, W], counts int32[n]) torch views of the device result (no copy)."""
        import torch
        n, W, _ = self.info()
        _, _, kp, cp = gerbil_counts_view(self.handle)
        if n == 0:
            dev = torch.device("cuda", self.ctx.device)
            return (torch.zeros((0, W), dtype=torch.int64, device=dev),
                    torch.zeros(0, dtype=torch.int32, device=dev))
        keys = torch.as_tensor(_DeviceArray(kp, (n, W), "<i8", self), device="cuda")
        cnts = torch.as_tensor(_DeviceArray(cp, (n,), "<i4", self), device="cuda")
        return keys, cnts

    def free(self):
        # a context frees its children before it is destroyed (include/gerbil.h ownership)
        if self.handle and self.ctx.handle:
            gerbil_counts_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _ServerOwner:
    """Stands in for a Context as the owner of results handed over by a Server."""

    def __init__(self, server):
        self._server = server
        self._children = weakref.WeakSet()

    @property
    def handle(self):
        return self._server.handle

    @property
    def device(self):
        return self._server.device


class Server:
    """Counting jobs served continuously under an HBM budget (see gerbil_server_create)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, slots: int = 4):
        self.device = device
        self.handle = gerbil_server_create(device, hbm_budget_bytes, slots)
        self._owner = _ServerOwner(self)
        self._keep = {}

    def submit(self, seq, offsets, k, m, nbins, min_count, opts=None, bin_bounds=None) -> int:
        if hasattr(seq, "data_ptr") and seq.is_cuda:
            import torch
            torch.cuda.current_stream(seq.device).synchronize()  # the workers' streams do not wait
        jid = gerbil_server_submit(self.handle, seq, offsets, k, m, nbins, min_count, opts, bin_bounds)
        if hasattr(seq, "data_ptr") and seq.is_cuda:
            self._keep[jid] = (seq, offsets)  # device reads stay alive until the job is waited for
        return jid

    def wait(self, job_id: int, timeout_ms: int = -1):
        h, times = gerbil_server_wait(self.handle, job_id, timeout_ms)
        self._keep.pop(job_id, None)
        return Counts(h, self._owner), times

    def stats(self):
        return gerbil_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            for child in list(self._owner._children):
                child.free()
            gerbil_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Bins:
    def __init__(self, handle, ctx):
        self.handle, self.ctx = handle, ctx
        ctx._children.add(self)

    def info(self):
        return gerbil_bins_info(self.handle)

    def stats(self, b: int):
        return gerbil_bin_stats(self.handle, b)

    def export(self):
        return gerbil_bins_export(self.handle)

    def free(self):
        if self.handle and self.ctx.handle:
            gerbil_bins_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        if not stream:
            # torch's default stream is the legacy default stream (handle 0); a NULL handle
            # would make the context create a stream of its own that does not wait for it
            stream = CUDA_STREAM_LEGACY
        self.device = device
        self._children = weakref.WeakSet()
        self.handle = gerbil_create(device, hbm_budget_bytes, stream)

    def partition(self, seq, offsets, k, m, nbins, opts=None, bin_bounds=None) -> Bins:
        return Bins(gerbil_partition(self.handle, seq, offsets, k, m, nbins, opts, bin_bounds), self)

    def count(self, bins: Bins, b: int, k: int, min_count: int, opts=None) -> Counts:
        return Counts(gerbil_count(self.handle, bins.handle, b, k, min_count, opts), self)

    def probe_stats(self, enable: bool = True):
        _check(load().gerbil_probe_stats(self.handle, 1 if enable else 0), self.handle)

    def get_probe_stats(self):
        """(slots, lines) histograms: index i < 32 = placed after i+1 slots read / lines
        touched, 32 = more, 33 = sent to the overflow area."""
        a = (ctypes.c_uint64 * 34)()
        b = (ctypes.c_uint64 * 34)()
        _check(load().gerbil_get_probe_stats(self.handle, a, b), self.handle)
        return np.array(a[:], dtype=np.uint64), np.array(b[:], dtype=np.uint64)

    def forget_ratio(self):
        _check(load().gerbil_forget_ratio(self.handle), self.handle)

    def autotune(self, bins: Bins, k: int, min_count: int, opts=None) -> dict:
        return gerbil_autotune(self.handle, bins.handle, k, min_count, opts)

    def set_tuning(self, k: int, tuning: dict | None):
        gerbil_set_tuning(self.handle, k, tuning)

    def get_tuning(self, k: int) -> dict | None:
        return gerbil_get_tuning(self.handle, k)

    def count_batch(self, bins: Bins, bin_list, k: int, min_count: int, opts=None) -> Counts:
        return Counts(gerbil_count_batch(self.handle, bins.handle, bin_list, k, min_count, opts), self)

    def profile(self, enable: bool = True):
        gerbil_profile(self.handle, enable)

    def phase_times(self):
        return gerbil_get_phase_times(self.handle)

    def close(self):
        if self.handle:
            for child in list(self._children):
                child.free()
            gerbil_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
