"""The sliced, pooled oracle equals one oracle call over the whole read set (counts are additive
over reads), and the device-side FNV filter equals the host one (both on the CPU here)."""
import numpy as np

import oracle
from paper_1607_06618_b300 import synth
from tests._oracle_pool import PassCount, read_slices
from tests._util import assert_same_rows, fnv1a64_device, fnv1a64_rows, keys_to_ascii


def test_read_slices_cover_every_read_once():
    _, offs = synth.random_small(300, 10, 500, p_n=0.0, seed=9)
    sl = read_slices(offs, 7)
    assert sl[0][0] == 0 and sl[-1][1] == offs.size - 1
    assert all(a[1] == b[0] for a, b in zip(sl[:-1], sl[1:]))


def test_pooled_slices_equal_one_oracle_call():
    seq, offs = synth.random_small(400, 40, 400, p_n=0.01, seed=21)
    seq = np.concatenate([seq, seq[: int(offs[150])]])  # repeats across slices
    offs = np.concatenate([offs, offs[1:151] + offs[-1]])
    jobs = [(seq, offs, 33, True, 4, 1), (seq, offs, 70, False, 1, 0), (seq[:0], offs[:1], 21, True, 1, 0)]
    got = PassCount(jobs, procs=3, slices_per_proc=3).result()
    assert_same_rows(got[0], oracle.count(seq, offs, 33, npass=4, pass_index=1))
    assert_same_rows(got[1], oracle.count(seq, offs, 70, canonical=False))
    assert got[2][0].shape == (0, 1) and got[2][1].size == 0


def test_device_fnv_equals_host_fnv():
    import torch
    seq, offs = synth.random_small(50, 120, 200, p_n=0.0, seed=5)
    for k in (5, 32, 33, 65, 127, 200):
        keys, _ = oracle.count(seq, offs, k)
        want = fnv1a64_rows(keys_to_ascii(keys, k))
        got = fnv1a64_device(torch.from_numpy(keys.view(np.int64)), k, rows_per_chunk=97)
        assert np.array_equal(got.numpy().view(np.uint64), want)
