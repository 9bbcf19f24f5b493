"""The no-allocation entry point against the regular one and the oracle (runs after every other
test).

gerbil_count_small_noalloc serves callers that cannot allocate device memory -- code whose
device memory belongs to another component (a framework's caching allocator, a fixed budget) or
that cannot take the device synchronisation cudaMalloc/cudaFree imply: its scratch is a fixed
device array inside the library.  Its rows must equal those of the regular path
(gerbil_partition + gerbil_count_batch) and the CPU oracle's exactly -- counts are integers --
on two calls in a row, since the second call reuses the array the first one left behind.
"""
import numpy as np
import pytest

import oracle
from paper_1607_06618_b300 import synth
from tests._util import assert_same_rows

pytestmark = pytest.mark.gpu


def _regular(gerbil, ctx, s, o, k, m, nbins, min_count, canonical):
    opts = gerbil.default_opts(canonical=1 if canonical else 0)
    bins = ctx.partition(s, o, k, m, nbins, opts)
    res = ctx.count_batch(bins, None, k, min_count, opts)
    keys, counts = res.to_host()
    res.free()
    bins.free()
    return keys, counts


@pytest.mark.parametrize("k,min_count,canonical", [(31, 1, True), (65, 2, True), (40, 1, False)])
def test_noalloc_matches_regular_path_and_oracle_twice(k, min_count, canonical):
    import torch
    from paper_1607_06618_b300 import gerbil

    assert torch.cuda.is_available()
    seq, offs = synth.random_small(600, 80, 300, p_n=0.003, seed=77 + k)
    seq = np.concatenate([seq, seq[: int(offs[200])]])  # repeats, so counts above 1 occur
    offs = np.concatenate([offs, offs[1:201] + offs[-1]])
    s = torch.from_numpy(seq).cuda()
    o = torch.from_numpy(offs.view(np.int64)).cuda()
    ctx = gerbil.Context(0)
    try:
        want = _regular(gerbil, ctx, s, o, k, 7, 16, min_count, canonical)
    finally:
        ctx.close()
    assert_same_rows(want, oracle.count(seq, offs, k, canonical=canonical, min_count=min_count))
    W = (2 * k + 63) // 64
    cap = int(seq.size)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        keys = torch.full((cap, W), -1, dtype=torch.int64, device="cuda")
        counts = torch.zeros(cap, dtype=torch.int32, device="cuda")
        n = gerbil.gerbil_count_small_noalloc(s, o, k, min_count, canonical, keys, counts, stream)
        got = (keys[:n].cpu().numpy().view(np.uint64), counts[:n].cpu().numpy().view(np.uint32))
        assert_same_rows(got, want)


def test_noalloc_size_limits_and_argument_checks():
    import torch
    from paper_1607_06618_b300 import gerbil

    keys = torch.zeros((1, 3), dtype=torch.int64, device="cuda")
    counts = torch.zeros(1, dtype=torch.int32, device="cuda")
    # more windows than the scratch table holds (524 thousand at k = 65): rejected by the
    # library before any GPU work
    s = torch.full((600_000,), ord("A"), dtype=torch.uint8, device="cuda")
    o = torch.tensor([0, 600_000], dtype=torch.int64, device="cuda")
    with pytest.raises(gerbil.GerbilError) as e:
        gerbil.gerbil_count_small_noalloc(s, o, 65, 1, True, keys, counts, None)
    assert e.value.status == gerbil.GERBIL_E_INVAL
    # an output buffer that is too small is reported with the size it needed
    seq, offs = synth.random_small(50, 100, 120, p_n=0.0, seed=3)
    s = torch.from_numpy(seq).cuda()
    o = torch.from_numpy(offs.view(np.int64)).cuda()
    with pytest.raises(gerbil.GerbilError) as e:
        gerbil.gerbil_count_small_noalloc(s, o, 65, 1, True, keys, counts, None)
    assert e.value.status == gerbil.GERBIL_E_INVAL
    # buffers the library would write past, or read outside of, never reach it
    big = torch.zeros(4096, dtype=torch.int32, device="cuda")
    narrow = torch.zeros((4096, 1), dtype=torch.int64, device="cuda")  # k = 65 needs 3 words
    bad = [
        (s, o, narrow, big),                                            # keys_out too narrow
        (s, o, torch.zeros((4096, 6), dtype=torch.int64, device="cuda")[:, ::2], big),  # strided
        (s, o, torch.zeros((4096, 3), dtype=torch.int32, device="cuda"), big),  # wrong dtype
        (s, o, torch.zeros((4096, 3), dtype=torch.int64), big),          # host tensor
        (s, o, torch.zeros((4096, 3), dtype=torch.int64, device="cuda"),
         torch.zeros(4096, dtype=torch.int64, device="cuda")),          # counts not int32
        (s, o[:0], torch.zeros((4096, 3), dtype=torch.int64, device="cuda"), big),  # no offsets
        (s[:10], o, torch.zeros((4096, 3), dtype=torch.int64, device="cuda"), big),  # offsets past seq
    ]
    for args in bad:
        with pytest.raises(ValueError):
            gerbil.gerbil_count_small_noalloc(args[0], args[1], 65, 1, True, args[2], args[3], None)
    # zero reads (offsets = [0]) is a valid, empty input
    n = gerbil.gerbil_count_small_noalloc(s, o[:1], 65, 1, True,
                                          torch.zeros((4096, 3), dtype=torch.int64, device="cuda"),
                                          big, None)
    assert n == 0
