"""The CPU oracle over large read sets: its key-pass filter (keys whose FNV-1a hash is
pass_index mod npass) run on disjoint slices of the reads in spawned processes, the slices'
counts added per key.

Counts are additive over reads -- every window lies in exactly one read -- so the sum over the
slices is the oracle's count over the whole read set, restricted to the pass's keys.  The pool
is started with ``spawn``: a process forked after CUDA was initialised can hang.  The slices'
reads are sent to the workers by pickling (no shared memory or temporary files needed).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _count_slice(args):
    seq, offs, k, canonical, npass, pass_index = args
    import oracle
    return oracle.count(seq, offs, k, canonical=canonical, min_count=1, npass=npass,
                        pass_index=pass_index)


def read_slices(offs: np.ndarray, nslices: int):
    """[r0, r1) read ranges of about equal base counts."""
    offs = np.asarray(offs, dtype=np.uint64)
    nreads = offs.size - 1
    if nreads <= 0:
        return []
    cuts = np.searchsorted(offs, np.linspace(0, int(offs[-1]), nslices + 1)[1:-1].astype(np.uint64))
    bounds = np.unique(np.concatenate([[0], np.clip(cuts, 0, nreads), [nreads]]))
    return [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


def merge(keys: np.ndarray, counts: np.ndarray):
    """Rows with equal keys summed; ascending key order."""
    keys = np.asarray(keys, dtype=np.uint64)
    counts = np.asarray(counts, dtype=np.uint64)
    if counts.size == 0:
        return keys.reshape(0, keys.shape[-1] if keys.ndim == 2 else 0), counts
    order = np.lexsort(keys.T[::-1])
    keys, counts = keys[order], counts[order]
    new = np.ones(counts.size, dtype=bool)
    new[1:] = np.any(keys[1:] != keys[:-1], axis=1)
    starts = np.flatnonzero(new)
    return keys[starts], np.add.reduceat(counts, starts)


class PassCount:
    """Starts the workers at once (so that the caller can do GPU work meanwhile); ``result()``
    waits and returns (keys uint64[n, W], counts uint64[n]) in ascending key order."""

    def __init__(self, jobs, procs: int | None = None, slices_per_proc: int = 4):
        """jobs: list of (seq, offs, k, canonical, npass, pass_index); one result per job."""
        import oracle
        oracle.build()  # once, before the workers load it
        procs = max(1, min(procs or os.cpu_count() or 1, 64))
        tasks, self._owner = [], []
        for j, (seq, offs, k, canonical, npass, pidx) in enumerate(jobs):
            offs = np.asarray(offs, dtype=np.uint64)
            for r0, r1 in read_slices(offs, procs * slices_per_proc):
                a, b = int(offs[r0]), int(offs[r1])
                tasks.append((seq[a:b], offs[r0:r1 + 1] - np.uint64(a), k, canonical, npass, pidx))
                self._owner.append(j)
        self._words = [(2 * job[2] + 63) // 64 for job in jobs]
        self._njobs = len(jobs)
        self.procs = procs
        self._pool = mp.get_context("spawn").Pool(procs)
        self._async = self._pool.map_async(_count_slice, tasks, chunksize=1)

    def result(self):
        try:
            parts = self._async.get()
        finally:
            self._pool.close()
            self._pool.join()
        out = []
        for j in range(self._njobs):
            mine = [p for p, o in zip(parts, self._owner) if o == j]
            if not mine:
                out.append((np.zeros((0, self._words[j]), np.uint64), np.zeros(0, np.uint64)))
                continue
            out.append(merge(np.concatenate([p[0] for p in mine]),
                             np.concatenate([p[1] for p in mine])))
        return out
