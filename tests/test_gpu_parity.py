"""Parity of the CUDA path (through the C ABI) with the CPU oracle -- needs a B300.

Counts are integers, so every comparison is bit-exact: same set of keys, same counts.  Bins
are compared as sets of (global start, k-mers, bin) rows, since their order within a bin is
free.
"""
import numpy as np
import pytest

import oracle
from paper_1607_06618_b300 import synth
from tests._util import (assert_same_rows, fnv1a64_rows, keys_to_ascii, reads_from_strings,
                         revcomp_reads, sort_rows)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_06618_b300 import gerbil
    ctx = gerbil.Context(0)
    yield gerbil, ctx, torch
    ctx.close()


def _dev(torch, seq, offs):
    return (torch.from_numpy(np.ascontiguousarray(seq)).cuda(),
            torch.from_numpy(np.ascontiguousarray(offs).view(np.int64)).cuda())


def _gpu_count(g, seq, offs, k, m, nbins, min_count, on_device=True, batch=True, **opt):
    gerbil, ctx, torch = g
    o = gerbil.default_opts(**opt)
    s, of = _dev(torch, seq, offs) if on_device else (seq, offs)
    bins = ctx.partition(s, of, k, m, nbins, o, opt.get("bin_bounds"))
    if batch:
        res = ctx.count_batch(bins, None, k, min_count, o)
        keys, counts = res.to_host()
        stats = res.info()[2]
        res.free()
    else:
        ks, cs = [], []
        stats = {"overflowed": 0, "retries": 0}
        for b in range(nbins):
            r = ctx.count(bins, b, k, min_count, o)
            kk, cc = r.to_host()
            ks.append(kk)
            cs.append(cc)
            stats["overflowed"] += r.info()[2]["overflowed"]
            stats["retries"] += r.info()[2]["retries"]
            r.free()
        W = (2 * k + 63) // 64
        keys = np.concatenate(ks) if ks else np.zeros((0, W), np.uint64)
        counts = np.concatenate(cs) if cs else np.zeros(0, np.uint32)
    bins.free()
    return (keys, counts), stats


# ---- phase one -------------------------------------------------------------------------

def _gpu_bins(g, seq, offs, k, m, nbins, **opt):
    gerbil, ctx, torch = g
    o = gerbil.default_opts(**opt)
    s, of = _dev(torch, seq, offs)
    bins = ctx.partition(s, of, k, m, nbins, o, opt.get("bin_bounds"))
    ex = bins.export()
    info = bins.info()
    stats = [bins.stats(b) for b in range(nbins)]
    bins.free()
    return ex, info, stats


def _rows(part):
    return sorted(zip(part["pos"].tolist(), part["nkmers"].tolist(), part["bin"].tolist()))


@pytest.mark.parametrize("k,m,lmax,ordering", [
    (32, 7, 256, 0), (32, 7, 7, 0), (65, 9, 256, 0), (65, 9, 1024, 1), (8, 3, 5, 1),
    (99, 9, 64, 0), (200, 11, 256, 0), (256, 15, 300, 0), (33, 1, 256, 1),
    (32, 7, 256, 2), (65, 9, 256, 3), (65, 9, 256, 4), (99, 11, 128, 2), (127, 15, 256, 3),
    (200, 13, 256, 4), (12, 1, 256, 3), (10, 2, 3, 4)])
def test_partition_matches_oracle(g, k, m, lmax, ordering):
    nreads = 700 if k < 100 else 120
    seq, offs = synth.random_small(nreads, k - 3, k + 400, p_n=0.004, seed=k * 31 + m)
    nbins = 37
    ex, info, stats = _gpu_bins(g, seq, offs, k, m, nbins, supermer_cap=lmax, ordering=ordering)
    want = oracle.partition(seq, offs, k, m, nbins, ordering=ordering, lmax=lmax)
    assert _rows(ex) == _rows(want)
    assert info["n_kmers"] == oracle.windows(seq, offs, k)
    for b in range(nbins):
        sel = want["bin"] == b
        assert stats[b][0] == int(sel.sum())
        assert stats[b][2] == int(want["nkmers"][sel].sum())


def test_partition_config1_full_and_bounds(g):
    seq, offs, p = synth.workload("uniform-20k-k32")
    bounds = np.sort(np.random.default_rng(3).integers(0, 2 ** 32, p["nbins"] - 1)).astype(np.uint32)
    for bb in (None, bounds):
        ex, _, _ = _gpu_bins(g, seq, offs, p["k"], p["m"], p["nbins"], bin_bounds=bb)
        want = oracle.partition(seq, offs, p["k"], p["m"], p["nbins"], bounds=bb)
        assert _rows(ex) == _rows(want)


def test_partition_edge_reads(g):
    k, m = 12, 5
    reads = ["", "ACGT", "A" * 12, "acgtACGTacgtN", "N" * 40, "ACGTNACGTACGTACGTTT", "",
             "GATTACA" * 9, "ACGTRYACGTACGTACGTACGT\n", "T" * 11, "C" * 13]
    seq, offs = reads_from_strings(reads)
    for lmax in (1, 3, 256):
        ex, _, _ = _gpu_bins(g, seq, offs, k, m, 4, supermer_cap=lmax)
        want = oracle.partition(seq, offs, k, m, 4, lmax=lmax)
        assert _rows(ex) == _rows(want)
    # forward minimizers in lexicographic order: Fig. 1's example
    seq, offs = reads_from_strings(["CAAGAACAGTG" * 3])
    ex, _, _ = _gpu_bins(g, seq, offs, 8, 3, 1, ordering=1, canonical_minimizer=0, canonical=0)
    want = oracle.partition(seq, offs, 8, 3, 1, ordering=1, canonical_min=False)
    assert _rows(ex) == _rows(want)


@pytest.mark.parametrize("k,m", [(32, 7), (65, 9)])
def test_every_byte_value_in_reads(g, k, m):
    """Sec. 2.4.1: only ACGTacgt are bases.  Each of the 256 byte values replaces twenty bases
    at random positions of ragged reads (so both the 32-byte vector path and the scalar tail of
    the encoder see it); bins and counts match the oracle."""
    rng = np.random.default_rng(k)
    seq, offs = synth.random_small(2000, k - 2, k + 600, p_n=0.0, seed=k + 7, lowercase=True)
    seq = seq.copy()
    hit = rng.choice(seq.size, 256 * 20, replace=False)
    seq[hit] = np.tile(np.arange(256, dtype=np.uint8), 20)
    ex, _, _ = _gpu_bins(g, seq, offs, k, m, 16)
    assert _rows(ex) == _rows(oracle.partition(seq, offs, k, m, 16))
    got, _ = _gpu_count(g, seq, offs, k, m, 16, 1)
    assert_same_rows(got, oracle.count(seq, offs, k, min_count=1))


# ---- phase two -------------------------------------------------------------------------

# the first and last k of every (key words, stored chunks) pair from k = 8 to the paper's 479:
# the key's low 30 bits sit in the meta word, the rest in max(1, ceil((2k - 30) / 63)) chunks
@pytest.mark.parametrize("k", [8, 15, 16, 31, 32, 33, 46, 47, 64, 65, 78, 79, 96, 97, 99, 109,
                               110, 128, 129, 141, 142, 160, 161, 172, 173, 192, 193, 200, 204,
                               205, 224, 225, 235, 236, 256, 257, 267, 268, 288, 289, 298, 299,
                               320, 321, 330, 331, 352, 353, 361, 362, 384, 385, 393, 394, 416,
                               417, 424, 425, 448, 449, 456, 457, 479])
def test_count_matches_oracle_all_word_counts(g, k):
    m = min(11, k - 1)
    seq, offs = synth.random_small(400, max(1, k - 4), k + 300, p_n=0.003, seed=1000 + k,
                                   lowercase=(k % 2 == 1))
    # add repeated content so that counts above 1 occur
    seq = np.concatenate([seq, seq[: int(offs[50])]])
    offs = np.concatenate([offs, offs[1:51] + offs[-1]])
    for mc in (1, 2):
        got, _ = _gpu_count(g, seq, offs, k, m, 16, mc)
        assert_same_rows(got, oracle.count(seq, offs, k, canonical=True, min_count=mc))


# both probe schemes (linear; the paper's windowed double hashing) and every work-item size on
# the same inputs, with and without forced overflow (theta = 1), over the slot sizes 16..112 B
@pytest.mark.parametrize("k", [8, 32, 33, 64, 65, 97, 99, 127, 200, 400])
def test_probe_schemes_and_item_sizes(g, k):
    m = min(11, k - 1)
    seq, offs = synth.random_small(500, max(1, k - 4), k + 300, p_n=0.003, seed=3000 + k)
    seq = np.concatenate([seq, seq[: int(offs[120])]])
    offs = np.concatenate([offs, offs[1:121] + offs[-1]])
    gerbil, ctx, torch = g
    combos = ((0, 256), (1, 256), (0, 128), (1, 64), (0, 64), (1, 128))
    if k > 128:  # items of 64 and 128 k-mers are built for keys of up to four words
        for scheme, ik in combos[2:]:
            with pytest.raises(gerbil.GerbilError) as e:
                _gpu_count(g, seq, offs, k, m, 16, 1, probe_scheme=scheme, item_kmers=ik)
            assert e.value.status == gerbil.GERBIL_E_UNSUPPORTED
        combos = combos[:2]
    for mc in (1, 2):
        want = oracle.count(seq, offs, k, canonical=True, min_count=mc)
        for scheme, ik in combos:
            ctx.forget_ratio()  # tables sized for all-distinct keys: nothing overflows
            got, st = _gpu_count(g, seq, offs, k, m, 16, mc, probe_scheme=scheme, item_kmers=ik)
            assert st["overflowed"] == 0
            assert_same_rows(got, want)
            if ik != 256 and mc == 2:
                continue
            got, st = _gpu_count(g, seq, offs, k, m, 16, mc, probe_scheme=scheme, item_kmers=ik,
                                 max_probes=1, distinct_ratio=0.05, overflow_slots=1 << 22)
            assert st["overflowed"] > 0
            assert_same_rows(got, want)
            got, st = _gpu_count(g, seq, offs, k, m, 16, mc, probe_scheme=scheme, item_kmers=ik,
                                 persistent=0, schedule=0)
            assert_same_rows(got, want)


# both probe orders (claim first / read first, gerbil_opts.claim_first) on the same inputs, with
# and without forced overflow (theta = 1), in the capped and the uncapped (tables beyond L2)
# forms of the kernel
@pytest.mark.parametrize("k", [21, 32, 65, 99, 200, 479])
def test_claim_first_and_read_first_probe_orders(g, k):
    gerbil, ctx, torch = g
    m = min(11, k - 1)
    seq, offs = synth.random_small(500, max(1, k - 4), k + 300, p_n=0.003, seed=3500 + k)
    seq = np.concatenate([seq, seq[: int(offs[120])]])
    offs = np.concatenate([offs, offs[1:121] + offs[-1]])
    for mc in (1, 2):
        want = oracle.count(seq, offs, k, canonical=True, min_count=mc)
        for cf in (1, 2):
            ctx.forget_ratio()
            got, st = _gpu_count(g, seq, offs, k, m, 16, mc, claim_first=cf)
            assert st["overflowed"] == 0
            assert_same_rows(got, want)
            got, st = _gpu_count(g, seq, offs, k, m, 16, mc, claim_first=cf, max_probes=1,
                                 distinct_ratio=0.05, overflow_slots=1 << 22)
            assert st["overflowed"] > 0
            assert_same_rows(got, want)
    if k in (200, 479):  # one table larger than L2: the uncapped form of the kernel
        seq, offs = synth.uniform_reads(2500, 1000, 0.0, seed=7500 + k)
        want = oracle.count(seq, offs, k, canonical=True, min_count=1)
        for cf in (1, 2):
            ctx.forget_ratio()
            got, st = _gpu_count(g, seq, offs, k, 11, 1, 1, claim_first=cf)
            assert_same_rows(got, want)


def test_bad_probe_scheme_and_item_size_rejected(g):
    gerbil, ctx, torch = g
    seq, offs = synth.random_small(20, 40, 60, p_n=0.0, seed=1)
    for bad in (dict(probe_scheme=2), dict(item_kmers=96), dict(item_kmers=512),
                dict(claim_first=3), dict(claim_first=-1)):
        with pytest.raises(gerbil.GerbilError) as e:
            _gpu_count(g, seq, offs, 21, 7, 4, 1, **bad)
        assert e.value.status == gerbil.GERBIL_E_INVAL


# keys of six or more words in one table larger than the L2 cache: the insert kernel's form
# without the register cap
@pytest.mark.parametrize("k", [200, 400, 479])
def test_count_wide_keys_tables_beyond_l2(g, k):
    gerbil, ctx, torch = g
    seq, offs = synth.uniform_reads(2500, 1000, 0.0, seed=7000 + k)
    seq = np.concatenate([seq, seq[: int(offs[300])]])  # 300 reads twice: counts of 2
    offs = np.concatenate([offs, offs[1:301] + offs[-1]])
    ctx.forget_ratio()
    got, st = _gpu_count(g, seq, offs, k, 11, 1, 1)
    slot = gerbil.slot_bytes(k)
    assert st["table_slots"] * slot > torch.cuda.get_device_properties(0).L2_cache_size
    assert_same_rows(got, oracle.count(seq, offs, k, canonical=True, min_count=1))


def test_count_config1_full_batch_grid_and_per_bin(g):
    seq, offs, p = synth.workload("uniform-20k-k32")
    want = oracle.count(seq, offs, p["k"], min_count=1)
    assert int(want[1].sum()) == oracle.windows(seq, offs, p["k"])
    for batch, persistent, fused in ((True, 1, 0), (True, 0, 0), (True, 1, 1), (True, 1, 2),
                                     (False, 1, 0), (False, 1, 1), (False, 1, 2)):
        got, _ = _gpu_count(g, seq, offs, p["k"], p["m"], p["nbins"], 1, batch=batch,
                            persistent=persistent, fused=fused)
        assert_same_rows(got, want)


def test_fused_ring_wrap_dedicated_and_classic(g):
    """Fused form with a tiny table ring: ring regions are reused many times (each reuse waits
    for the previous tenant's compaction) and the larger bins get dedicated tables; waves of
    several sizes; the two-kernel form."""
    seq, offs = synth.random_small(3000, 100, 300, p_n=0.002, seed=21)
    seq = np.concatenate([seq, seq[: int(offs[800])]])
    offs = np.concatenate([offs, offs[1:801] + offs[-1]])
    k = 45
    want = oracle.count(seq, offs, k, min_count=2)
    for ring in (3000, 20000, 40000, 0):
        got, st = _gpu_count(g, seq, offs, k, 9, 97, 2, fused=1, ring_slots=ring)
        assert st["overflowed"] == 0
        assert_same_rows(got, want)
    got, _ = _gpu_count(g, seq, offs, k, 9, 97, 2, fused=0, persistent=0)
    assert_same_rows(got, want)
    # a two-kernel call leaves tables in the arena; the next fused call must clear them
    got, _ = _gpu_count(g, seq, offs, k, 9, 97, 2, fused=1, ring_slots=20000)
    assert_same_rows(got, want)
    for wave in (3000, 20000, 0):
        got, st = _gpu_count(g, seq, offs, k, 9, 97, 2, fused=2, ring_slots=wave)
        assert_same_rows(got, want)
    # forced overflow in the fused form falls back to the overflow recount
    got, st = _gpu_count(g, seq, offs, k, 9, 97, 2, fused=1, max_probes=1, distinct_ratio=0.05,
                         overflow_slots=1 << 22)
    assert st["overflowed"] > 0
    assert_same_rows(got, want)


def test_count_host_buffers_path(g):
    seq, offs = synth.random_small(300, 50, 400, p_n=0.01, seed=5)
    got, _ = _gpu_count(g, seq, offs, 41, 9, 8, 1, on_device=False)
    assert_same_rows(got, oracle.count(seq, offs, 41))


def test_count_noncanonical(g):
    seq, offs = synth.random_small(300, 50, 400, p_n=0.01, seed=6)
    for k in (21, 77):
        got, _ = _gpu_count(g, seq, offs, k, 7, 8, 1, canonical=0)
        assert_same_rows(got, oracle.count(seq, offs, k, canonical=False))


def test_count_edge_cases(g):
    k = 16
    reads = ["", "A" * 15, "A" * 16, "A" * 200, "T" * 100, "ACGTACGTACGTACGTACGT",
             "NNNNNNNNNNNNNNNNNNNNNNNN", "acgtacgtacgtacgtAC", "GGGGCCCC" * 10]
    seq, offs = reads_from_strings(reads)
    for mc in (1, 2, 3, 100):
        got, _ = _gpu_count(g, seq, offs, k, 5, 3, mc)
        assert_same_rows(got, oracle.count(seq, offs, k, min_count=mc))
    # no windows at all
    seq, offs = reads_from_strings(["ACG", "", "NNNN"])
    got, _ = _gpu_count(g, seq, offs, k, 5, 3, 1)
    assert got[1].size == 0


def test_forced_overflow_recount_is_exact(g):
    # theta = 1 and a tiny table send most k-mers to the overflow area
    seq, offs = synth.random_small(500, 100, 300, p_n=0.002, seed=8)
    seq = np.concatenate([seq, seq])
    offs = np.concatenate([offs, offs[1:] + offs[-1]])
    for k in (32, 65, 200):
        want = oracle.count(seq, offs, k, min_count=2)
        kw = dict(max_probes=1, distinct_ratio=0.05, overflow_slots=1 << 22)
        got, st = _gpu_count(g, seq, offs, k, 9, 4, 2, **kw)
        assert st["overflowed"] > 0 and st["retries"] == 0
        assert_same_rows(got, want)
        # per-bin path with the same forcing
        got, st = _gpu_count(g, seq, offs, k, 9, 4, 2, batch=False, **kw)
        assert st["overflowed"] > 0
        assert_same_rows(got, want)


def test_overflow_area_full_retries(g):
    seq, offs = synth.random_small(200, 100, 200, p_n=0.0, seed=9)
    got, st = _gpu_count(g, seq, offs, 33, 7, 2, 1, max_probes=1, distinct_ratio=0.01,
                         overflow_slots=16)
    assert st["retries"] > 0
    assert_same_rows(got, oracle.count(seq, offs, 33))


def test_invariants_on_gpu(g):
    seq, offs = synth.random_small(800, 100, 300, p_n=0.005, seed=10)
    base, _ = _gpu_count(g, seq, offs, 45, 9, 64, 1)
    rc, _ = _gpu_count(g, *revcomp_reads(seq, offs), 45, 9, 64, 1)
    assert_same_rows(rc, base)
    for nb, m in ((1, 9), (7, 5), (1000, 11)):
        other, _ = _gpu_count(g, seq, offs, 45, m, nb, 1)
        assert_same_rows(other, base)


# ---- the measured workload at full size ----------------------------------------------------

@pytest.fixture(scope="module")
def genome5m():
    return synth.workload("genome5M-30x-k65")


def test_genome5m_full_size_sampled_parity(g, genome5m):
    """Full-size k=65 workload, batched persistent launch as timed by bench.py: the keys with
    FNV-1a(key) = 0 (mod 64) must match the oracle's pass 0 of 64 exactly."""
    seq, offs, p = genome5m
    got, st = _gpu_count(g, seq, offs, p["k"], p["m"], p["nbins"], p["min_count"])
    keys, counts = got
    h = fnv1a64_rows(keys_to_ascii(keys, p["k"]))
    sel = (h % np.uint64(64)) == np.uint64(0)
    want = oracle.count(seq, offs, p["k"], min_count=p["min_count"], npass=64, pass_index=0)
    assert_same_rows((keys[sel], counts[sel]), want)
    assert st["occurrences"] == oracle.windows(seq, offs, p["k"])


def test_genome5m_full_size_total(g, genome5m):
    """At min_count = 1 the counts sum to the number of N-free windows (closed form)."""
    seq, offs, p = genome5m
    got, st = _gpu_count(g, seq, offs, p["k"], p["m"], p["nbins"], 1)
    k = p["k"]
    total_windows = (offs.size - 1) * (150 - k + 1)  # no N in this workload
    assert int(got[1].astype(np.uint64).sum()) == total_windows
    assert st["distinct"] == got[1].size
    # each key once
    sk, _ = sort_rows(*got)
    assert not np.any(np.all(sk[1:] == sk[:-1], axis=1))


def test_counts_do_not_depend_on_the_ordering(g):
    """The six orderings move k-mers between bins, never change a count (Sec. 2.1)."""
    seq, offs = synth.random_small(500, 60, 260, p_n=0.003, seed=4242)
    seq = np.concatenate([seq, seq[: int(offs[80])]])
    offs = np.concatenate([offs, offs[1:81] + offs[-1]])
    want = oracle.count(seq, offs, 41, min_count=1)
    for ordering in range(6):
        got, _ = _gpu_count(g, seq, offs, 41, 9, 23, 1, ordering=ordering)
        assert_same_rows(got, want)


@pytest.mark.parametrize("k,m,p,every", [(32, 7, 0.5, 16), (65, 9, 0.0, 4), (65, 9, 1.0, 1),
                                         (99, 11, 0.8, 8), (20, 6, 0.5, 3), (127, 12, 0.3, 5)])
def test_partition_dfp_ordering_matches_oracle(g, k, m, p, every):
    """dfp(p) (Sec. 3.1): frequencies sampled on the GPU, rank table built by the library; the
    bins equal the oracle's, which samples and ranks by its own code."""
    seq, offs = synth.random_small(600, k - 3, k + 300, p_n=0.004, seed=k * 7 + m)
    seq = np.concatenate([seq, seq[: int(offs[100])]])  # repeats: uneven m-mer frequencies
    offs = np.concatenate([offs, offs[1:101] + offs[-1]])
    ex, _, _ = _gpu_bins(g, seq, offs, k, m, 29, ordering=5, dfp_pivot=p, dfp_sample=every)
    want = oracle.partition(seq, offs, k, m, 29, ordering=5, dfp_p=p, dfp_every=every)
    assert _rows(ex) == _rows(want)


def test_bounded_wait_runs_out_and_context_stays_usable(g):
    """Every device wait is bounded: a wait on a flag that nothing sets ends after its limit
    with GERBIL_E_TIMEOUT, and the same context counts exactly afterwards."""
    gerbil, ctx, torch = g
    import time
    t0 = time.perf_counter()
    assert gerbil.gerbil_wait_selftest(ctx.handle, 50_000_000) == gerbil.GERBIL_E_TIMEOUT
    assert 0.04 < time.perf_counter() - t0 < 5.0
    assert gerbil.gerbil_wait_selftest(ctx.handle, 0) == gerbil.GERBIL_E_INVAL
    seq, offs = synth.random_small(50, 40, 120, p_n=0.01, seed=77)
    got, _ = _gpu_count(g, seq, offs, 31, 7, 8, 1)
    assert_same_rows(got, oracle.count(seq, offs, 31))


# ---- sorted output ---------------------------------------------------------------------

@pytest.mark.parametrize("k", [20, 32, 65, 99, 200, 479])
def test_sorted_output_equals_oracle_in_order(g, k):
    """gerbil_opts.sorted_output: the rows come back in ascending key order -- compared with the
    oracle's rows (ascending by construction) position by position, with no host sort -- for
    key widths of 1, 1, 3, 4, 7 and 15 words, from the batch and from a grouped batch."""
    gerbil, ctx, torch = g
    m = min(11, k - 1)
    seq, offs = synth.random_small(700, max(1, k - 4), k + 300, p_n=0.003, seed=4000 + k)
    seq = np.concatenate([seq, seq[: int(offs[150])]])
    offs = np.concatenate([offs, offs[1:151] + offs[-1]])
    for mc, extra in ((1, {}), (2, {}), (1, {"max_table_mib": 1})):
        wk, wc = oracle.count(seq, offs, k, canonical=True, min_count=mc)
        o = gerbil.default_opts(sorted_output=1, **extra)
        s, of = _dev(torch, seq, offs)
        bins = ctx.partition(s, of, k, m, 16, o)
        res = ctx.count_batch(bins, None, k, mc, o)
        keys, counts = res.to_host()
        st = res.info()[2]
        res.free()
        bins.free()
        assert st["sorted"] == 1
        if extra:
            assert st["groups"] > 1
        assert np.array_equal(np.asarray(keys, np.uint64).reshape(wk.shape), wk)
        assert np.array_equal(np.asarray(counts, np.uint64), wc)


def test_sorted_output_many_rows_and_per_bin(g):
    """A larger sort (several hundred tiles of 2048 rows, equal high digits everywhere) and the
    single-bin call."""
    gerbil, ctx, torch = g
    seq, offs = synth.uniform_reads(6000, 150, 0.002, seed=77)
    k = 31
    wk, wc = oracle.count(seq, offs, k, canonical=True, min_count=1)
    assert len(wc) > 600_000
    o = gerbil.default_opts(sorted_output=1)
    s, of = _dev(torch, seq, offs)
    bins = ctx.partition(s, of, k, 7, 8, o)
    res = ctx.count_batch(bins, None, k, 1, o)
    keys, counts = res.to_host()
    res.free()
    assert np.array_equal(np.asarray(keys, np.uint64).reshape(wk.shape), wk)
    assert np.array_equal(np.asarray(counts, np.uint64), wc)
    one = ctx.count(bins, 3, k, 1, o)
    kk, cc = one.to_host()
    one.free()
    bins.free()
    kk = np.asarray(kk, np.uint64).reshape(-1, 1)
    assert len(cc) > 1000 and np.all(kk[1:, 0] > kk[:-1, 0])
