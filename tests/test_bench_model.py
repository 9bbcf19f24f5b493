"""Host-side arithmetic of bench.py: the insert kernel's algorithmic byte model, the bounded
samples the oracle is timed on, and the k sweep's range (no GPU)."""
import numpy as np

import bench


def test_insert_byte_model_steps_with_the_sector_rounded_slot():
    """P(W) = 32 * ceil((8W + 8) / 32) + 32: a slot read rounded up to 32-byte sectors plus one
    dirty sector written back -- 64 B up to 3 key words, 96 B up to 7, 128 B up to 11, 160 B
    up to 15."""
    want = {1: 64, 2: 64, 3: 64, 4: 96, 5: 96, 6: 96, 7: 96, 8: 128, 9: 128, 10: 128, 11: 128,
            12: 160, 13: 160, 14: 160, 15: 160}
    for W, p in want.items():
        insert, step = bench._model_bytes(occ=1000, n_bases=0, distinct=0, emitted=0, W=W)
        assert insert == 1000 * p
        assert step == insert
    # b_in is a quarter byte per base of the super-mers; compaction reads 8W+8 bytes per live
    # entry and writes 8W+4 per output row
    insert, step = bench._model_bytes(occ=10, n_bases=400, distinct=7, emitted=3, W=3)
    assert insert == 100 + 10 * 64
    assert step == insert + 7 * 32 + 3 * 28


def test_oracle_sample_holds_the_requested_windows():
    # reads of 150, 10 (shorter than k), 150 and 200 bases at k = 65: 86, 0, 86, 136 windows
    lens = np.array([150, 10, 150, 200], dtype=np.uint64)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    assert bench._reads_for_windows(offs, 65, 1) == 1
    assert bench._reads_for_windows(offs, 65, 86) == 1
    assert bench._reads_for_windows(offs, 65, 87) == 3
    assert bench._reads_for_windows(offs, 65, 172) == 3
    assert bench._reads_for_windows(offs, 65, 173) == 4
    assert bench._reads_for_windows(offs, 65, 10 ** 9) == 4  # never past the last read


def test_k_sweep_spans_every_key_width_band_up_to_479():
    ks = bench.KSWEEP
    assert list(ks) == sorted(ks) and ks[0] == 32 and ks[-1] == 479
    widths = {(2 * k + 63) // 64 for k in ks}
    assert {1, 3, 4, 7, 8, 15} <= widths


def test_traffic_only_from_a_profile_of_the_current_source():
    """The bench line carries the DRAM bytes of the committed config-2 insert summary only while
    that summary was taken on the current kernel source; otherwise null, with the reason."""
    traffic, src = bench._traffic_and_source("genome5M-30x-k65")
    if bench._src_sha() in src:
        assert traffic is not None and 2e9 < traffic < 6e9, src
    else:
        assert traffic is None and "another kernel source" in src, src
    assert bench._traffic_and_source("no-such-workload") == (None, "no ncu summary for this workload")
