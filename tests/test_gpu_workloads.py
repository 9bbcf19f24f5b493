"""The repeat-rich (k=99, log-normal bins) and long-read (k=200, indels) workloads on the GPU:
exact oracle parity at reduced scale (same generators, same structure), closed-form totals at
full size."""
import numpy as np
import pytest

import oracle
from paper_1607_06618_b300 import synth
from tests._util import assert_same_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    from paper_1607_06618_b300 import gerbil
    ctx = gerbil.Context(0)
    yield gerbil, ctx, torch
    ctx.close()


def _count(g, s, o, p, min_count, **opt):
    gerbil, ctx, torch = g
    opts = gerbil.default_opts(**opt)
    bins = ctx.partition(s, o, p["k"], p["m"], p["nbins"], opts, p.get("bin_bounds"))
    info = bins.info()
    res = ctx.count_batch(bins, None, p["k"], min_count, opts)
    keys, counts = res.to_host()
    st = res.info()[2]
    res.free()
    bins.free()
    return (keys, counts), st, info


@pytest.mark.parametrize("name,scale", [("genome100M-repeats-30x-k99", 0.001),
                                        ("genome50M-longreads-20x-k200", 0.004)])
def test_reduced_scale_parity(g, name, scale):
    s, o, p = synth.torch_workload(name, scale=scale, device="cuda")
    seq = s.cpu().numpy()
    offs = o.cpu().numpy().view(np.uint64)
    for mc in (1, p["min_count"]):
        for fused in (0, 1):
            got, st, info = _count(g, s, o, p, mc, fused=fused)
            assert_same_rows(got, oracle.count(seq, offs, p["k"], min_count=mc))
    # the bins as sets of (start, k-mers, bin) rows
    gerbil, ctx, torch = g
    bins = ctx.partition(s, o, p["k"], p["m"], p["nbins"], gerbil.default_opts(), p.get("bin_bounds"))
    ex = bins.export()
    bins.free()
    want = oracle.partition(seq, offs, p["k"], p["m"], p["nbins"], bounds=p.get("bin_bounds"))
    key = lambda d: sorted(zip(d["pos"].tolist(), d["nkmers"].tolist(), d["bin"].tolist()))
    assert key(ex) == key(want)


@pytest.mark.parametrize("name", ["genome100M-repeats-30x-k99", "genome50M-longreads-20x-k200"])
def test_full_size_totals(g, name):
    s, o, p = synth.torch_workload(name, device="cuda")
    seq = s.cpu().numpy()
    offs = o.cpu().numpy().view(np.uint64)
    windows = oracle.windows(seq, offs, p["k"])
    got, st, info = _count(g, s, o, p, 1)
    assert info["n_kmers"] == windows == st["occurrences"]
    assert int(got[1].astype(np.uint64).sum()) == windows
    assert st["distinct"] == got[1].size
