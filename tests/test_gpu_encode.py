"""App. C output records written on the GPU equal the oracle's encoder row by row (bytes, no
tolerance), for one-byte and five-byte counts, every key width, host and device output (host
output with and without room for the longest records), and a result joined from bin groups."""
import numpy as np
import pytest

import oracle
from paper_1607_06618_b300 import synth
from tests._util import keys_to_ascii

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1607_06618_b300 import gerbil
    ctx = gerbil.Context(0)
    yield gerbil, ctx
    ctx.close()


def _reads():
    """300 bp reads at every start of a 2 kbp genome, six times over (a k-mer is counted
    6 x (301 - k) times: 270 and more up to k = 256), plus random reads (count 1): both
    one-byte and five-byte counts."""
    gen = synth.genome(2000, 7201)
    tiled, toffs = synth.tiled_reads(gen, 300, 1)
    rnd, roffs = synth.random_small(300, 60, 200, p_n=0.01, seed=7202)
    parts = [(tiled, toffs)] * 6 + [(rnd, roffs)]
    seq = np.concatenate([p[0] for p in parts])
    offs = [np.uint64(0)]
    for s_, o_ in parts:
        offs.extend((o_[1:] + offs[-1]).tolist())
    return seq, np.asarray(offs, dtype=np.uint64)


def _want(keys, counts, k):
    ascii_rows = keys_to_ascii(keys, k)
    return b"".join(oracle.encode_record(r.tobytes().decode(), int(c)) for r, c in zip(ascii_rows, counts))


@pytest.mark.parametrize("k", [8, 31, 32, 33, 65, 99, 127, 200, 256])
def test_records_equal_oracle_encoding(g, k):
    gerbil, ctx = g
    seq, offs = _reads()
    bins = ctx.partition(seq, offs, k, min(9, k - 1), 8)
    res = ctx.count_batch(bins, None, k, 1)
    keys, counts = res.to_host()
    assert counts.max() >= 255 and counts.min() < 255
    want = _want(keys, counts, k)
    host = res.encode_records(k)
    assert host.tobytes() == want
    dev = res.encode_records(k, device=True)
    assert dev.cpu().numpy().tobytes() == want
    # a host buffer with room for every count in its 5-byte form: written without a size pass
    room = np.full(len(counts) * ((k + 3) // 4 + 5), 0xAB, dtype=np.uint8)
    nb = gerbil.gerbil_encode_records(res.handle, k, room.ctypes.data, room.size, 0)
    assert nb == len(want) and room[:nb].tobytes() == want
    with pytest.raises(gerbil.GerbilError):
        gerbil.gerbil_encode_records(res.handle, k + 64 if k + 64 <= 256 else k - 64)
    res.free()
    bins.free()


def test_records_of_a_grouped_result_and_of_an_empty_one(g):
    gerbil, ctx = g
    seq, offs = synth.random_small(20000, 100, 200, p_n=0.005, seed=7203)  # ~2.4 M distinct
    k = 65
    bins = ctx.partition(seq, offs, k, 9, 64)
    ctx.forget_ratio()  # the ratio learned on the repetitive reads above would not fit this input
    res = ctx.count_batch(bins, None, k, 1, gerbil.default_opts(max_table_mib=1))
    assert res.info()[2]["groups"] > 1
    keys, counts = res.to_host()
    assert res.encode_records(k).tobytes() == _want(keys, counts, k)
    res.free()
    res = ctx.count_batch(bins, None, k, 1 << 30)  # no row reaches min_count
    assert len(res) == 0 and res.encode_records(k).size == 0
    res.free()
    bins.free()


@pytest.mark.parametrize("k", [320, 479])
def test_records_of_wide_keys_at_any_output_alignment(g, k):
    """The longest records (k up to 479, counts of five bytes) and device output that starts
    at every offset modulo 16: the writer stages each 32-row chunk in shared memory and copies
    it out in 16-byte stores, with byte stores at the chunk's ends."""
    import torch
    gerbil, ctx = g
    gen = synth.genome(1500, 7204 + k)
    tiled, toffs = synth.tiled_reads(gen, 600, 1)
    rnd, roffs = synth.random_small(60, k, k + 300, p_n=0.0, seed=7205)
    parts = [(tiled, toffs)] * 3 + [(rnd, roffs)]  # up to 3 x 122 = 366 copies at k = 479
    seq = np.concatenate([p[0] for p in parts])
    offs = [np.uint64(0)]
    for s_, o_ in parts:
        offs.extend((o_[1:] + offs[-1]).tolist())
    offs = np.asarray(offs, dtype=np.uint64)
    bins = ctx.partition(seq, offs, k, 11, 4)
    res = ctx.count_batch(bins, None, k, 1)
    keys, counts = res.to_host()
    assert counts.max() >= 255 and counts.min() < 255
    want = _want(keys, counts, k)
    assert res.encode_records(k).tobytes() == want
    buf = torch.full((len(want) + 64,), 0xAB, dtype=torch.uint8, device="cuda")
    for shift in (1, 3, 8, 15):
        buf.fill_(0xAB)
        nb = gerbil.gerbil_encode_records(res.handle, k, buf.data_ptr() + shift, len(want), 1)
        host = buf.cpu().numpy()
        assert nb == len(want)
        assert host[shift:shift + nb].tobytes() == want
        assert (host[:shift] == 0xAB).all() and (host[shift + nb:] == 0xAB).all()
    res.free()
    bins.free()
