"""The two generator implementations agree (no GPU): torch draws equal the numpy draws, on
CPU, for the same (seed, stream, index)."""
import numpy as np

from paper_1607_06618_b300 import synth


def test_torch_draws_equal_numpy_draws():
    for seed, stream, start, n in ((1, 0, 0, 1000), (3003, 2, 123456789, 777), (5000 + 17, 34, 5, 64)):
        a = synth.draws(seed, stream, start, n)
        b = synth.t_draws(seed, stream, start, n).numpy().view(np.uint64)
        assert np.array_equal(a, b)


def test_torch_generators_are_deterministic_and_well_formed():
    s1, o1, p = synth.torch_workload("genome100M-repeats-30x-k99", scale=0.0005)
    s2, o2, _ = synth.torch_workload("genome100M-repeats-30x-k99", scale=0.0005)
    assert bytes(s1.numpy()) == bytes(s2.numpy()) and np.array_equal(o1.numpy(), o2.numpy())
    assert set(np.unique(s1.numpy()).tolist()) <= set(b"ACGT")
    assert int(o1[-1]) == s1.numel() and (o1[1:] - o1[:-1]).eq(250).all()
    b = p["bin_bounds"]
    assert b.size == p["nbins"] - 1 and np.all(np.diff(b.astype(np.int64)) >= 0)
    s, o, _ = synth.torch_workload("genome50M-longreads-20x-k200", scale=0.002)
    L = (o[1:] - o[:-1]).numpy()
    assert int(o[-1]) == s.numel() and L.min() >= 150 and L.max() <= 110000
    assert 0.15e6 * 20 * 0.9 < s.numel() < 0.2e6 * 20 * 1.3
