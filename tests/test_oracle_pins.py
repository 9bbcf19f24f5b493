"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties the oracle to something other than itself: a worked example printed in the
paper (tests/golden/), brute force on tiny inputs (oracle/brute.py, pure Python), a closed
form, or an invariant that must hold for the exact histogram.
"""
import collections
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1607_06618_b300 import synth
from tests._util import revcomp_reads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _reads(strings):
    seq = np.frombuffer("".join(strings).encode(), dtype=np.uint8).copy()
    offs = np.zeros(len(strings) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(s) for s in strings])
    return seq, offs


def _as_dict(keys, counts, k):
    return {oracle.key_to_string(keys[i], k): int(counts[i]) for i in range(len(counts))}


# ---- worked examples ------------------------------------------------------------------

def test_fig1_supermers_worked_example():
    rows = {r[0]: r[1:] for r in _golden("fig1_supermers.txt") if r[0] != "supermer"}
    expect = [r[1] for r in _golden("fig1_supermers.txt") if r[0] == "supermer"]
    s, k, m = rows["sequence"][0], int(rows["k"][0]), int(rows["m"][0])
    seq, offs = _reads([s])
    part = oracle.partition(seq, offs, k, m, nbins=1, ordering=oracle.ORDER_LEX,
                            canonical_min=False, lmax=1 << 30)
    got = [s[int(p):int(p) + int(n) + k - 1] for p, n in zip(part["pos"], part["nkmers"])]
    assert got == expect
    # the brute force reaches the same five super-mers
    assert [x[1] for x in brute.supermers(s, k, m, ordering="lex", canonical_min=False)] == expect


def test_canonical_worked_example():
    rows = {r[0]: r[1] for r in _golden("canonical_example.txt")}
    assert brute.revcomp(rows["kmer"]) == rows["revcomp"]
    seq, offs = _reads([rows["kmer"], rows["revcomp"], "NNNN"])
    keys, counts = oracle.count(seq, offs, 4, canonical=True)
    assert _as_dict(keys, counts, 4) == {rows["canonical"]: 2}
    keys, counts = oracle.count(seq, offs, 4, canonical=False)
    assert _as_dict(keys, counts, 4) == {rows["kmer"]: 1, rows["revcomp"]: 1}


def test_appc_record_worked_examples():
    for row in _golden("appc_records.txt"):
        count, kmer, bits = int(row[0]), row[1], row[2:]
        expect = bytes(int(b, 2) for b in bits)
        assert oracle.encode_record(kmer, count) == expect
    # boundary of the one-byte counter: 254 fits, 255 takes the escape
    assert oracle.encode_record("ACGT", 254) == bytes([254, 0b00011011])
    assert oracle.encode_record("ACGT", 255) == bytes([0xFF, 0, 0, 0, 255, 0b00011011])


# ---- key layout and the KMC2 ordering reading -----------------------------------------

def test_key_layout_numeric_equals_lexicographic():
    rng = np.random.default_rng(5)
    for k in (3, 31, 32, 33, 64, 65, 100):
        strs = ["".join("ACGT"[i] for i in rng.integers(0, 4, k)) for _ in range(40)]
        seq, offs = _reads(strs)
        keys, counts = oracle.count(seq, offs, k, canonical=False)
        got = [oracle.key_to_string(w, k) for w in keys]
        assert got == sorted(set(strs))  # ascending key order == lexicographic order
        # unused high bits of word 0 are zero
        spare = 64 * keys.shape[1] - 2 * k
        if spare:
            assert np.all(keys[:, 0] >> np.uint64(64 - spare) == 0)


def test_kmc2_ordering_cases():
    four7 = 4 ** 7
    cases = {  # m-mer -> demoted?
        "AAACGTC": True,   # starts with AAA
        "ACAGTCG": True,   # starts with ACA
        "CAAGTCG": True,   # AA at position 1
        "CGTCGAA": True,   # AA at the end
        "AACGTCG": False,  # AA only at the very beginning
        "CGTACGT": False,
        "TTTTTTT": False,
    }
    for s, demoted in cases.items():
        v = brute.value(s)
        assert oracle.mmer_rank(s, oracle.ORDER_KMC2) == v + (four7 if demoted else 0), s
        assert oracle.mmer_rank(s, oracle.ORDER_LEX) == v
    # every demoted m-mer ranks after every kept one
    assert oracle.mmer_rank("TTTTTTT") < oracle.mmer_rank("AAAAAAA")


def test_bin_map_reading():
    # fmix32 of MurmurHash3 (published constants); known values of the finalizer
    assert oracle.bin_of(0, 1 << 31) == 0
    assert oracle.bin_of(1, 2 ** 32 - 1) == 0x514E28B7 % (2 ** 32 - 1)
    bounds = np.array([1 << 30, 1 << 31, 3 << 30], dtype=np.uint32)
    for v in range(200):
        h = oracle.bin_of(v, 2 ** 32 - 1)  # raw hash (below the modulus)
        assert oracle.bin_of(v, 4, bounds) == int(np.searchsorted(bounds, h, side="right"))


# ---- brute force on tiny inputs -------------------------------------------------------

KS = [3, 4, 5, 8, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 300, 479]


@pytest.mark.parametrize("k", KS)
def test_count_equals_brute_force(k):
    for seed in range(3):
        seq, offs = synth.random_small(30, max(1, k - 5), k + 120, p_n=0.02, seed=100 * k + seed,
                                       lowercase=(seed == 1))
        reads = brute.reads_from(seq.tobytes(), offs)
        for canonical in (True, False):
            for mc in (1, 2):
                keys, counts = oracle.count(seq, offs, k, canonical=canonical, min_count=mc)
                assert _as_dict(keys, counts, k) == brute.count(reads, k, canonical, mc)


def test_count_low_complexity_and_palindromes():
    # even k admits palindromes x == revcomp(x): one count per occurrence, not two
    reads = ["ACGTACGTACGT", "AAAAAAAAAAAA", "TTTTTTTT", "ACGT", "GGCC" * 5, "NNNN", ""]
    seq, offs = _reads(reads)
    for k in (2, 4, 6):
        keys, counts = oracle.count(seq, offs, k)
        assert _as_dict(keys, counts, k) == brute.count(reads, k)
    keys, counts = oracle.count(seq, offs, 4)
    d = _as_dict(keys, counts, 4)
    assert d["ACGT"] == 4  # three in read 0, one in read 3 (palindrome)
    assert d["AAAA"] == 9 + 5  # AAAA in read 1 and its reverse complement TTTT in read 2


@pytest.mark.parametrize("k,m", [(8, 3), (15, 5), (32, 7), (33, 9), (65, 9)])
def test_partition_equals_brute_force(k, m):
    for seed in range(2):
        seq, offs = synth.random_small(25, k - 2, k + 90, p_n=0.01, seed=7 * k + seed)
        reads = brute.reads_from(seq.tobytes(), offs)
        for ordering, oname in ((oracle.ORDER_KMC2, "kmc2"), (oracle.ORDER_LEX, "lex")):
            for lmax in (10 ** 6, 7):
                part = oracle.partition(seq, offs, k, m, nbins=16, ordering=ordering, lmax=lmax)
                got = [(int(p), int(n), int(b), int(z)) for p, n, b, z in
                       zip(part["pos"], part["nkmers"], part["bin"], part["minimizer"])]
                want = []
                for i, r in enumerate(reads):
                    for g, s, mz in brute.supermers(r, k, m, oname, True, lmax, int(offs[i])):
                        v = brute.value(mz)
                        want.append((g, len(s) - k + 1, oracle.bin_of(v, 16), v))
                assert got == want


# ---- closed forms ---------------------------------------------------------------------

def test_total_equals_nfree_windows_config1_scale():
    seq, offs, p = synth.workload("uniform-20k-k32", scale=0.25)
    keys, counts = oracle.count(seq, offs, p["k"])
    total = int(counts.sum())
    # independent count in numpy: windows whose k bases are all in ACGT
    good = np.isin(seq, np.frombuffer(b"ACGT", np.uint8)).astype(np.int64).reshape(-1, 150)
    csum = np.concatenate([np.zeros((good.shape[0], 1), np.int64), np.cumsum(good, 1)], 1)
    k = p["k"]
    expect = int(((csum[:, k:] - csum[:, :-k]) == k).sum())
    assert total == expect == oracle.windows(seq, offs, k)
    # and it is close to the closed-form expectation 150-k+1 windows x 0.995^k per read
    exp_mean = good.shape[0] * (150 - k + 1) * 0.995 ** k
    assert abs(total - exp_mean) < 0.01 * exp_mean


def test_tiling_closed_form():
    # error-free forward reads at every s-th position: count(x) = number of reads covering x
    gen = synth.genome(3000, seed=77)
    L, s, k = 60, 7, 21
    seq, offs = synth.tiled_reads(gen, L, s)
    keys, counts = oracle.count(seq, offs, k, canonical=False)
    got = _as_dict(keys, counts, k)
    gstr = "".join("ACGT"[c] for c in gen)
    expect = collections.Counter()
    nreads = len(offs) - 1
    for i in range(gen.size - k + 1):
        cover = sum(1 for j in range(nreads) if j * s <= i and i + k <= j * s + L)
        if cover:
            expect[gstr[i:i + k]] += cover
    assert got == dict(expect)


# ---- invariants of the exact histogram --------------------------------------------------

def _revcomp_reads(seq, offs):
    reads = brute.reads_from(seq.tobytes(), offs)
    table = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")
    rr = [r.encode("latin-1").translate(table)[::-1].decode("latin-1") for r in reads]
    return _reads(rr)


@pytest.mark.parametrize("k", [25, 32, 65])
def test_invariant_reverse_complementing_reads(k):
    seq, offs = synth.random_small(200, 20, 300, p_n=0.01, seed=k)
    a = oracle.count(seq, offs, k)
    b = oracle.count(*_revcomp_reads(seq, offs), k)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("k", [24, 33])
def test_invariant_noncanonical_sums_to_canonical(k):
    seq, offs = synth.random_small(200, 20, 200, p_n=0.01, seed=3 + k)
    can = _as_dict(*oracle.count(seq, offs, k, canonical=True), k)
    raw = _as_dict(*oracle.count(seq, offs, k, canonical=False), k)
    for x, c in can.items():
        r = brute.revcomp(x)
        expect = raw.get(x, 0) + (raw.get(r, 0) if r != x else 0)
        assert c == expect


def test_invariant_read_permutation_and_passes():
    seq, offs = synth.random_small(150, 30, 200, p_n=0.01, seed=9)
    reads = brute.reads_from(seq.tobytes(), offs)
    perm = np.random.default_rng(1).permutation(len(reads))
    a = oracle.count(seq, offs, 31)
    b = oracle.count(*_reads([reads[i] for i in perm]), 31)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # the G-pass split of the oracle is a partition of the same histogram
    parts = [oracle.count(seq, offs, 31, npass=4, pass_index=g) for g in range(4)]
    keys = np.concatenate([p[0] for p in parts])
    counts = np.concatenate([p[1] for p in parts])
    order = np.lexsort(keys.T[::-1])
    assert np.array_equal(keys[order], a[0]) and np.array_equal(counts[order], a[1])


def test_invariant_partition_covers_windows_and_bins_agree():
    k, m, nb = 31, 7, 32
    seq, offs = synth.random_small(120, 25, 250, p_n=0.01, seed=4)
    part = oracle.partition(seq, offs, k, m, nb, lmax=40)
    s = seq.tobytes().decode()
    # the k-mers of all super-mers are exactly the N-free windows (as a multiset)
    from_parts = collections.Counter()
    for p, n in zip(part["pos"], part["nkmers"]):
        for i in range(int(n)):
            from_parts[s[int(p) + i:int(p) + i + k]] += 1
    windows = collections.Counter()
    for r in brute.reads_from(seq.tobytes(), offs):
        for i in range(len(r) - k + 1):
            if all(c in "ACGT" for c in r[i:i + k]):
                windows[r[i:i + k]] += 1
    assert from_parts == windows
    assert int(part["nkmers"].max()) <= 40
    # with canonical minimizers a k-mer and its reverse complement fall into one bin
    bin_of_kmer = {}
    for p, n, b in zip(part["pos"], part["nkmers"], part["bin"]):
        for i in range(int(n)):
            bin_of_kmer[s[int(p) + i:int(p) + i + k]] = int(b)
    for x, b in bin_of_kmer.items():
        mz = brute.minimizer(brute.revcomp(x), m)
        assert oracle.bin_of(brute.value(mz), nb) == b


# ---- the other orderings of Sec. 3.1 -----------------------------------------------------

def _all_mmers(m):
    return ["".join(t) for t in itertools.product("ACGT", repeat=m)]


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_cgat_ordering_is_lexicographic_in_c_g_a_t(m):
    mm = _all_mmers(m)
    by_rank = sorted(mm, key=lambda s: oracle.mmer_rank(s, oracle.ORDER_CGAT))
    assert by_rank == sorted(mm, key=lambda s: ["CGAT".index(c) for c in s])


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_roberts_ordering_complements_even_positions(m):
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}

    def key(s):
        t = [comp[c] if i % 2 == 1 else c for i, c in enumerate(s)]  # 2nd, 4th, ... base
        return ["CATG".index(c) for c in t]

    mm = _all_mmers(m)
    assert sorted(mm, key=lambda s: oracle.mmer_rank(s, oracle.ORDER_ROBERTS)) == sorted(mm, key=key)
    # the property Sec. 3.1 states: rare minimizers like CGCGCG are preferred -- it is the
    # smallest m-mer of all (it maps to CCCCCC)
    assert oracle.mmer_rank("CG" * 3, oracle.ORDER_ROBERTS) == 0


@pytest.mark.parametrize("m", [1, 2, 3, 5, 7])
def test_random_ordering_is_a_permutation(m):
    ranks = sorted(oracle.mmer_rank(s, oracle.ORDER_RANDOM) for s in _all_mmers(m))
    assert ranks == list(range(4 ** m))


@pytest.mark.parametrize("ordering", [0, 1, 2, 3, 4])
def test_partition_covers_every_window_under_every_ordering(ordering):
    """Every ordering gives super-mers whose k-mers are exactly the N-free windows, and x and
    revcomp(x) land in one bin (canonical minimizers)."""
    seq, offs = synth.random_small(60, 20, 120, p_n=0.01, seed=77 + ordering)
    k, m = 15, 5
    part = oracle.partition(seq, offs, k, m, 7, ordering=ordering)
    assert int(part["nkmers"].sum()) == oracle.windows(seq, offs, k)
    rseq, roffs = revcomp_reads(seq, offs)
    rpart = oracle.partition(rseq, roffs, k, m, 7, ordering=ordering)
    assert np.array_equal(np.bincount(part["bin"], weights=part["nkmers"], minlength=7),
                          np.bincount(rpart["bin"], weights=rpart["nkmers"], minlength=7))


def test_dfp_ordering_follows_frequencies_and_pivot():
    """dfp(p) (Sec. 3.1): a permutation; p = 0 ranks the rarest m-mers first, p = 1 the most
    frequent, p = 0.5 those of middle frequency (checked against a count written here)."""
    seq, offs = synth.random_small(400, 40, 120, p_n=0.02, seed=909)
    m, every = 3, 4
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}
    freq = collections.Counter()
    text = seq.tobytes().decode()
    for r in range(0, len(offs) - 1, every):
        read = text[int(offs[r]):int(offs[r + 1])].upper()
        for q in range(len(read) - m + 1):
            s = read[q:q + m]
            if set(s) <= set("ACGT"):
                rc = "".join(comp[c] for c in reversed(s))
                freq[min(s, rc)] += 1
    mm = sorted(_all_mmers(m), key=lambda s: (freq[s], brute.value(s)))  # ascending frequency
    for p, first in ((0.0, mm[0]), (1.0, mm[-1]), (0.5, mm[len(mm) // 2])):
        ranks = oracle.dfp_ranks(seq, offs, m, p=p, every=every)
        assert sorted(ranks.tolist()) == list(range(4 ** m))
        assert ranks[brute.value(first)] == 0
    ranks = oracle.dfp_ranks(seq, offs, m, p=0.0, every=every)
    assert [s for s in sorted(mm, key=lambda s: ranks[brute.value(s)])] == mm
