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


# --- torch generators (any device, bit-identical on CPU and GPU) ---------------------------
# Same SplitMix64 counter as above, in int64 arithmetic: products wrap modulo 2**64 and right
# shifts are made logical with a mask.  A uniform integer below M is (r >>> 11) % M; a
# probability p is tested as (r >>> 32) < floor(p * 2**32).

def _s64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


_TG = _s64(0x9E3779B97F4A7C15)
_TM1 = _s64(0xBF58476D1CE4E5B9)
_TM2 = _s64(0x94D049BB133111EB)


def _shr(z, s: int):
    return (z >> s) & ((1 << (64 - s)) - 1)


def _t_mix64(z):
    z = (z ^ _shr(z, 30)) * _TM1
    z = (z ^ _shr(z, 27)) * _TM2
    return z ^ _shr(z, 31)


def t_draws(seed: int, stream: int, start: int, n: int, device="cpu"):
    """r(seed, stream, i) for i in [start, start + n) as an int64 tensor (two's complement)."""
    import torch
    key = _t_mix64(torch.tensor([_s64((seed * 0x9E3779B97F4A7C15 + stream) % (1 << 64))],
                                dtype=torch.int64, device=device))
    idx = torch.arange(start + 1, start + n + 1, dtype=torch.int64, device=device)
    return _t_mix64(key + idx * _TG)


def _t_below(r, m: int):
    return _shr(r, 11) % m


def _t_hit(r, p: float):
    return _shr(r, 32) < int(math.floor(p * 2 ** 32))


def t_genome(size: int, seed: int, device="cpu"):
    import torch
    out = torch.empty(size, dtype=torch.uint8, device=device)
    step = 1 << 24
    for s in range(0, size, step):
        n = min(step, size - s)
        out[s:s + n] = (t_draws(seed, 0, s, n, device) & 3).to(torch.uint8)
    return out


def t_genome_with_repeats(size: int, seed: int, repeat_frac: float = 0.2, unit_min: int = 2000,
                          unit_max: int = 10000, copies_min: int = 5, copies_max: int = 50,
                          device="cpu"):
    """Uniform genome, then repeat units (a random segment of length U[unit_min, unit_max]
    copied U{copies_min..copies_max} times to uniform positions, overwriting) until
    repeat_frac of the genome has been written by copies.  Streams 20..23 of ``seed``."""
    g = t_genome(size, seed, device)
    copied, u = 0, 0
    while copied < repeat_frac * size:
        r = t_draws(seed, 20, 3 * u, 3, "cpu")
        L = unit_min + int(_t_below(r[0:1], unit_max - unit_min + 1))
        src = int(_t_below(r[1:2], size - L + 1))
        c = copies_min + int(_t_below(r[2:3], copies_max - copies_min + 1))
        unit = g[src:src + L].clone()
        dst = _t_below(t_draws(seed, 23, 64 * u, c, "cpu"), size - L + 1)
        for d in dst.tolist():
            g[d:d + L] = unit
        copied += c * L
        u += 1
    return g


_T_ASCII = None


def _ascii(device):
    import torch
    return torch.tensor(list(b"ACGT"), dtype=torch.uint8, device=device)


def t_sampled_reads(gen, nreads: int, length: int, p_sub: float, seed: int,
                    both_strands: bool = True, p_n: float = 0.0):
    """Fixed-length reads at uniform starts of ``gen`` (codes, a torch tensor), reverse strand
    with p = 1/2, substitutions with p_sub, N with p_n.  Streams 0..3 of ``seed``.  Returns
    (seq uint8 ASCII, offsets int64) on gen's device."""
    import torch
    dev = gen.device
    G = gen.numel()
    seq = torch.empty(nreads * length, dtype=torch.uint8, device=dev)
    per = max(1, (1 << 22) // length)
    cols = torch.arange(length, device=dev)
    lut = _ascii(dev)
    for j0 in range(0, nreads, per):
        nr = min(per, nreads - j0)
        starts = _t_below(t_draws(seed, 0, j0, nr, dev), G - length + 1)
        codes = gen[starts[:, None] + cols[None, :]].to(torch.int64)
        if both_strands:
            rev = _shr(t_draws(seed, 1, j0, nr, dev), 63).bool()
            codes = torch.where(rev[:, None], 3 - codes.flip(1), codes)
        base = j0 * length
        r = t_draws(seed, 2, base, nr * length, dev).view(nr, length)
        shift = 1 + (r & 0xFFFF) % 3
        codes = torch.where(_t_hit(r, p_sub), (codes + shift) & 3, codes)
        b = lut[codes]
        if p_n > 0:
            rn = t_draws(seed, 3, base, nr * length, dev).view(nr, length)
            b = torch.where(_t_hit(rn, p_n), torch.full_like(b, ord("N")), b)
        seq[base:base + nr * length] = b.reshape(-1)
    offsets = torch.arange(nreads + 1, dtype=torch.int64, device=dev) * length
    return seq, offsets


def t_long_reads(gen, coverage: float, median: float, sigma: float, lmin: int, lmax: int,
                 p_err: float, seed: int):
    """Reads of log-normal length (median, sigma; clipped to [lmin, lmax]) at uniform starts
    until coverage x genome bases are drawn; reverse strand with p = 1/2; per template base an
    error with p_err: substitution 60%, insertion of a random base before it 20%, deletion 20%.
    Streams 30..36 of ``seed``."""
    import torch
    dev = gen.device
    G = gen.numel()
    target = int(coverage * G)
    lens, total, i = [], 0, 0
    while total < target:
        n = 1 << 16
        u1 = (_shr(t_draws(seed, 30, i, n, "cpu"), 11).double() + 0.5) / float(1 << 53)
        u2 = (_shr(t_draws(seed, 31, i, n, "cpu"), 11).double() + 0.5) / float(1 << 53)
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)  # Box-Muller
        L = torch.clamp(torch.round(median * torch.exp(sigma * z)), lmin, min(lmax, G)).to(torch.int64)
        cs = torch.cumsum(L, 0)
        need = int(torch.searchsorted(cs, torch.tensor([target - total])).item()) + 1
        L = L[:need]
        lens.append(L)
        total += int(L.sum())
        i += n
    L = torch.cat(lens).to(dev)
    nreads = L.numel()
    starts = _t_below(t_draws(seed, 32, 0, nreads, dev), 1 << 62) % (G - L + 1)
    rev = _shr(t_draws(seed, 33, 0, nreads, dev), 63).bool()
    tpl_off = torch.zeros(nreads + 1, dtype=torch.int64, device=dev)
    tpl_off[1:] = torch.cumsum(L, 0)
    ntpl = int(tpl_off[-1])
    lut = _ascii(dev)
    pieces, out_lens = [], torch.zeros(nreads, dtype=torch.int64, device=dev)
    step = 1 << 24
    read_of = torch.repeat_interleave(torch.arange(nreads, device=dev), L)
    for s in range(0, ntpl, step):
        n = min(step, ntpl - s)
        rid = read_of[s:s + n]
        within = torch.arange(s, s + n, device=dev) - tpl_off[rid]
        # template base: forward from the start, or the reverse complement of the window
        fpos = starts[rid] + torch.where(rev[rid], L[rid] - 1 - within, within)
        code = gen[fpos].to(torch.int64)
        code = torch.where(rev[rid], 3 - code, code)
        e = t_draws(seed, 34, s, n, dev)
        hit = _t_hit(e, p_err)
        kind = (e & 0xFF) % 10  # 0-5 substitution, 6-7 insertion, 8-9 deletion
        sub = hit & (kind < 6)
        ins = hit & (kind >= 6) & (kind < 8)
        dele = hit & (kind >= 8)
        code = torch.where(sub, (code + 1 + (_shr(e, 8) & 0xFFFF) % 3) & 3, code)
        rb = t_draws(seed, 35, s, n, dev) & 3
        emit = 1 + ins.to(torch.int64) - dele.to(torch.int64)  # bases written per template base
        first = torch.where(ins, rb, code)     # an inserted base comes before the template base
        second = code
        both = torch.stack([first, second], 1).reshape(-1)
        keep = torch.stack([emit >= 1, emit == 2], 1).reshape(-1)
        pieces.append(lut[both[keep]])
        out_lens.index_add_(0, rid, emit)
    seq = torch.cat(pieces)
    offsets = torch.zeros(nreads + 1, dtype=torch.int64, device=dev)
    offsets[1:] = torch.cumsum(out_lens, 0)
    return seq, offsets


def lognormal_bounds(nbins: int, sigma: float, seed: int):
    """nbins-1 ascending split points over [0, 2**32) for per-bin weights LogNormal(0, sigma)."""
    import torch
    u1 = (_shr(t_draws(seed, 40, 0, nbins, "cpu"), 11).double() + 0.5) / float(1 << 53)
    u2 = (_shr(t_draws(seed, 41, 0, nbins, "cpu"), 11).double() + 0.5) / float(1 << 53)
    z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
    w = torch.exp(sigma * z).numpy()
    cum = np.cumsum(w) / w.sum()
    return np.minimum(np.floor(cum[:-1] * 2 ** 32), 2 ** 32 - 1).astype(np.uint32)


TORCH_WORKLOADS = {
    # 100 Mbp genome, 20% repeats (2-10 kbp units copied 5-50x; seeds 3001/3002), 12e6 reads of
    # 250 bp (30x), both strands, 0.3% substitutions (seed 3003); k=99, m=9, 1024 bins with
    # log-normal (sigma 1) shares of the minimizer space (seed 3004), min 2
    "genome100M-repeats-30x-k99": dict(k=99, m=9, nbins=1024, min_count=2),
    # 50 Mbp genome (seed 4001); reads of log-normal length (median 10 kbp, sigma 0.7, clipped
    # to [200, 100000]) to 20x, 10% errors (60/20/20 sub/ins/del), both strands (seed 4002);
    # k=200, m=11, 512 bins, min 2
    "genome50M-longreads-20x-k200": dict(k=200, m=11, nbins=512, min_count=2),
}


def torch_workload(name: str, scale: float = 1.0, device="cpu"):
    """(seq uint8, offsets int64, params) as torch tensors on ``device``; ``scale`` shrinks the
    genome and the read count together (same structure, smaller)."""
    p = dict(TORCH_WORKLOADS[name])
    if name == "genome100M-repeats-30x-k99":
        G = max(20000, int(100_000_000 * scale))
        gen = t_genome_with_repeats(G, 3001, device=device)
        nreads = max(1, int(round(30 * G / 250)))
        seq, off = t_sampled_reads(gen, nreads, 250, 0.003, 3003)
        p["bin_bounds"] = lognormal_bounds(p["nbins"], 1.0, 3004)
    elif name == "genome50M-longreads-20x-k200":
        G = max(200000, int(50_000_000 * scale))
        gen = t_genome(G, 4001, device)
        seq, off = t_long_reads(gen, 20.0, 10000.0, 0.7, 200, 100000, 0.10, 4002)
    else:
        raise KeyError(name)
    return seq, off, p


# Serving stream: Poisson arrivals (mean `rate` jobs/s); each job a 150 bp read set drawn from
# a random genome of log-uniform size in [1, 200] Mbp at a coverage uniform in [10, 40], both
# strands, 0.5% substitutions and 0.5% N; k uniform over {32, 65, 127} with m = 7, 9, 11;
# bins = the power of two nearest to windows / 1e6, clamped to [64, 1024]; min_count 1.
# Job parameters use streams 50..54 of ``seed``; job j's genome and reads use seeds
# 100000 + 2j and 100001 + 2j.
SERVING_K = ((32, 7), (65, 9), (127, 11))


def _unit(seed: int, stream: int, n: int):
    return (draws(seed, stream, 0, n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def serving_jobs(n_jobs: int, rate: float = 20.0, seed: int = 5, g_min: float = 1e6,
                 g_max: float = 200e6, read_len: int = 150):
    """Parameters of ``n_jobs`` jobs: dicts with arrival_s, genome, coverage, nreads, k, m,
    nbins, min_count, seeds."""
    u_gap, u_g, u_cov, u_k = (_unit(seed, 50 + i, n_jobs) for i in range(4))
    t, jobs = 0.0, []
    for j in range(n_jobs):
        t += -math.log(1.0 - u_gap[j]) / rate
        G = int(round(math.exp(math.log(g_min) + u_g[j] * (math.log(g_max) - math.log(g_min)))))
        cov = 10.0 + 30.0 * u_cov[j]
        k, m = SERVING_K[min(2, int(u_k[j] * 3))]
        nreads = max(1, int(round(cov * G / read_len)))
        nwin = nreads * (read_len - k + 1)
        nbins = 1 << max(0, int(round(math.log2(max(1.0, nwin / 1e6)))))
        nbins = min(1024, max(64, nbins))
        jobs.append(dict(arrival_s=t, genome=G, coverage=cov, nreads=nreads, read_len=read_len,
                         k=k, m=m, nbins=nbins, min_count=1,
                         genome_seed=100000 + 2 * j, read_seed=100001 + 2 * j))
    return jobs


def t_serving_reads(job: dict, device="cuda", scale: float = 1.0):
    """(seq, offsets) of one serving job on ``device`` (``scale`` shrinks genome and reads)."""
    G = max(4 * job["read_len"], int(job["genome"] * scale))
    nreads = max(1, int(round(job["nreads"] * scale)))
    gen = t_genome(G, job["genome_seed"], device)
    seq, off = t_sampled_reads(gen, nreads, job["read_len"], 0.005, job["read_seed"], p_n=0.005)
    del gen
    return seq, off
