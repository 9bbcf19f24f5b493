"""Autotuner: the settings it picks are in range, are kept per key width, and counting with
them -- or with any other settings in the search space -- gives the oracle's rows exactly."""
import numpy as np
import pytest

import oracle
from paper_1607_06618_b300 import synth
from tests._util import assert_same_rows

pytestmark = pytest.mark.gpu

K, M, NBINS = 65, 9, 64


@pytest.fixture(scope="module")
def data():
    import torch
    from paper_1607_06618_b300 import gerbil
    gen = synth.genome(400_000, 7101)
    seq, offs = synth.sampled_reads(gen, 30_000, 150, 0.005, 7102)
    want = oracle.count(seq, offs, K, min_count=2)
    s = torch.from_numpy(seq).cuda()
    o = torch.from_numpy(offs.view(np.int64)).cuda()
    ctx = gerbil.Context(0)
    bins = ctx.partition(s, o, K, M, NBINS)
    yield gerbil, ctx, bins, want
    bins.free()
    ctx.close()


def _rows(ctx, bins, opts):
    res = ctx.count_batch(bins, None, K, 2, opts)
    got = res.to_host()
    res.free()
    return got


def test_autotune_picks_valid_settings_and_counts_match(data):
    gerbil, ctx, bins, want = data
    assert ctx.get_tuning(K) is None
    t = ctx.autotune(bins, K, 2)
    assert t["fused"] in (0, 1, 2) and t["schedule"] in (0, 1)
    assert all(a in (0.35, 0.5, 0.65, 0.8) for a in (round(x, 2) for x in t["load_factor"]))
    assert t["probe_scheme"] in (0, 1) and t["item_kmers"] in (64, 128, 256)
    assert t["k_words"] == 3 and t["samples"] >= 4 and t["ns_per_kmer"] > 0
    assert ctx.get_tuning(K) == t and ctx.get_tuning(96) == t  # same key width (3 words)
    assert ctx.get_tuning(64) is None  # 2 words
    assert ctx.get_tuning(31) is None
    assert_same_rows(_rows(ctx, bins, gerbil.default_opts(autotune=1)), want)


@pytest.mark.parametrize("fused,schedule,alpha,scheme,ik", [
    (0, 1, 0.8, 0, 256), (0, 0, 0.35, 1, 128), (1, 1, 0.65, 0, 256), (2, 1, 0.8, 0, 256),
    (0, 1, 0.8, 1, 64), (0, 1, 0.35, 0, 64), (0, 1, 0.65, 1, 256)])
def test_every_setting_of_the_search_space_counts_exactly(data, fused, schedule, alpha, scheme, ik):
    gerbil, ctx, bins, want = data
    n = gerbil.TUNE_CLASSES
    ctx.set_tuning(K, {"load_factor": [alpha] * n, "fused": fused, "schedule": schedule,
                       "probe_scheme": scheme, "item_kmers": ik})
    assert_same_rows(_rows(ctx, bins, gerbil.default_opts(autotune=1)), want)
    ctx.set_tuning(K, None)
    assert ctx.get_tuning(K) is None


def test_tuned_on_first_use_and_rejects_bad_settings(data):
    gerbil, ctx, bins, want = data
    ctx.set_tuning(K, None)
    assert_same_rows(_rows(ctx, bins, gerbil.default_opts(autotune=1)), want)
    assert ctx.get_tuning(K) is not None  # tuned by the first call with autotune set
    with pytest.raises(gerbil.GerbilError):
        ctx.set_tuning(K, {"load_factor": [0.99] * 4, "fused": 0, "schedule": 1})
    with pytest.raises(gerbil.GerbilError):
        ctx.set_tuning(K, {"load_factor": [0.5] * 4, "fused": 3, "schedule": 1})


def test_graph_form_counts_exactly_and_is_reused(data):
    """Graph form: the captured batch gives the oracle's rows; the second batch of the same shape
    updates the instantiated graph, a batch of another shape builds a new one."""
    gerbil, ctx, bins, want = data
    ctx.profile(True)
    opts = gerbil.default_opts(graph=1)
    for _ in range(3):
        assert_same_rows(_rows(ctx, bins, opts), want)
    t = ctx.phase_times()
    assert t["graph_launches"] == 3 and t["insert_launches"] == 3
    assert t["insert_ms"] > 0 and t["compact_ms"] > 0  # phase events recorded inside the graph
    # a subset of the bins (another shape), then the full batch again
    sub = list(range(0, NBINS, 3))
    res = ctx.count_batch(bins, sub, K, 2, opts)
    part = res.to_host()
    res.free()
    res = ctx.count_batch(bins, sub, K, 2, gerbil.default_opts())
    assert_same_rows(part, res.to_host())
    res.free()
    assert_same_rows(_rows(ctx, bins, opts), want)
    ctx.profile(False)


def test_graph_form_with_overflow_and_retry(data):
    """Graph form, then the overflow recount after it (theta = 1, small tables), and a retry
    after the overflow area ran full (a new graph shape)."""
    gerbil, ctx, bins, want = data
    opts = gerbil.default_opts(graph=1, max_probes=1, distinct_ratio=0.05, overflow_slots=1 << 22)
    res = ctx.count_batch(bins, None, K, 2, opts)
    st = res.info()[2]
    assert st["overflowed"] > 0 and st["retries"] == 0
    assert_same_rows(res.to_host(), want)
    res.free()
    opts = gerbil.default_opts(graph=1, max_probes=1, distinct_ratio=0.01, overflow_slots=16)
    res = ctx.count_batch(bins, None, K, 2, opts)
    assert res.info()[2]["retries"] > 0
    assert_same_rows(res.to_host(), want)
    res.free()


@pytest.mark.parametrize("scheme", [0, 1])
def test_probe_statistics_account_for_every_kmer(data, scheme):
    """Probe histograms (Sec. 3.3): every inserted k-mer is recorded once (placed after some
    number of slots, or sent to the overflow area); lines (scheme 0) or windows (scheme 1)
    never exceed slots read; the statistics change no count."""
    gerbil, ctx, bins, want = data
    ctx.probe_stats(True)
    got = _rows(ctx, bins, gerbil.default_opts(probe_scheme=scheme))
    slots, lines = ctx.get_probe_stats()
    occ = bins.info()["n_kmers"]
    assert int(slots.sum()) == occ and int(lines.sum()) == occ
    assert slots[33] == lines[33] == 0  # nothing overflowed at theta 1024
    # lines <= slots for every k-mer: the cumulative line histogram dominates the slot one
    assert np.all(np.cumsum(lines[:33]) >= np.cumsum(slots[:33]))
    assert slots[0] > occ // 2
    ctx.probe_stats(False)
    with pytest.raises(gerbil.GerbilError):
        ctx.get_probe_stats()
    assert_same_rows(got, want)
    # theta = 1 with small tables: k-mers that found no room are counted in the last bucket
    ctx.probe_stats(True)
    res = ctx.count_batch(bins, None, K, 2, gerbil.default_opts(max_probes=1, distinct_ratio=0.05,
                                                                 overflow_slots=1 << 22,
                                                                 probe_scheme=scheme))
    st = res.info()[2]
    res.free()
    slots, lines = ctx.get_probe_stats()
    assert int(slots[33]) == st["overflowed"] > 0 and int(slots[:33].sum()) + int(slots[33]) == occ
    ctx.probe_stats(False)


def test_ratio_learned_from_a_batch_that_overflowed(data):
    """Sec. 3.4 sizing: a ratio learned on a repetitive input sizes the tables of a more diverse
    one too small; that batch spills (and stays exact), and the ratio it measured sizes the
    next batch, which must not spill again."""
    gerbil, ctx, _, _ = data
    import torch
    rep, roffs = synth.uniform_reads(500, 150, 0.0, seed=7301)
    rep = np.tile(rep, 8)  # every read 8 times: about 1/8 of the k-mers distinct
    roffs = np.arange(8 * 500 + 1, dtype=np.uint64) * 150
    uni, uoffs = synth.uniform_reads(4000, 150, 0.0, seed=7302)  # nearly all distinct
    want = oracle.count(uni, uoffs, 32, min_count=1)
    opts = gerbil.default_opts(overflow_slots=1 << 24)
    ctx.forget_ratio()

    def count(seq, offs):
        s = torch.from_numpy(seq).cuda()
        o = torch.from_numpy(offs.view(np.int64)).cuda()
        bins = ctx.partition(s, o, 32, 7, 16, opts)
        res = ctx.count_batch(bins, None, 32, 1, opts)
        got, st = res.to_host(), res.info()[2]
        res.free()
        bins.free()
        return got, st

    _, st = count(rep, roffs)
    assert st["distinct"] * 6 < st["occurrences"]
    got, st = count(uni, uoffs)
    assert st["overflowed"] > 0 and st["retries"] == 0
    assert_same_rows(got, want)
    got, st = count(uni, uoffs)
    assert st["overflowed"] == 0
    assert_same_rows(got, want)
    ctx.forget_ratio()
