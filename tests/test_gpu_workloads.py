"""The repeat-rich (k=99, log-normal bins) and long-read (k=200, indels) workloads on the GPU:
exact oracle parity at reduced scale (same generators, same structure), and at full size the
rows of a key pass of the oracle plus the closed-form totals; the serving stream's small jobs at
full scale against the oracle, in the mix and alone."""
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
    wk, wc = oracle.count(seq, offs, p["k"], min_count=1)
    for mc in (1, p["min_count"]):
        sel = wc >= mc  # the min_count filter of the oracle's rows (App. A -l: inclusive)
        for fused in (0, 1):
            got, st, info = _count(g, s, o, p, mc, fused=fused)
            assert_same_rows(got, (wk[sel], wc[sel]))
    # the bins as sets of (start, k-mers, bin) rows
    gerbil, ctx, torch = g
    bins = ctx.partition(s, o, p["k"], p["m"], p["nbins"], gerbil.default_opts(), p.get("bin_bounds"))
    ex = bins.export()
    bins.free()
    want = oracle.partition(seq, offs, p["k"], p["m"], p["nbins"], bounds=p.get("bin_bounds"))
    key = lambda d: sorted(zip(d["pos"].tolist(), d["nkmers"].tolist(), d["bin"].tolist()))
    assert key(ex) == key(want)


# ---- full size, in the launch configuration bench.py times ---------------------------------
# npass: the oracle keeps the keys whose FNV-1a hash is 0 mod npass (about 1/npass of them), over
# every read, in spawned processes over read slices (tests/_oracle_pool.py); the GPU rows of the
# same keys are selected on the device.  npass is chosen so that a worker's map stays small.
FULL = [("genome100M-repeats-30x-k99", 256), ("genome50M-longreads-20x-k200", 1024)]


@pytest.mark.parametrize("name,npass", FULL)
def test_full_size_sampled_parity_and_totals(g, name, npass):
    """Every read of the full workload, counted as bench.py counts it (one count_batch over all
    bins, default options): the rows of the pass's keys equal the oracle's at min_count 1 and at
    the workload's min_count, and at min_count 1 the counts add up to the number of windows."""
    from tests._oracle_pool import PassCount
    from tests._util import device_pass_rows
    gerbil, ctx, torch = g
    s, o, p = synth.torch_workload(name, device="cuda")
    k = p["k"]
    seq = s.cpu().numpy()
    offs = o.cpu().numpy().view(np.uint64)
    pool = PassCount([(seq, offs, k, True, npass, 0)])  # runs while the GPU counts
    got = {}
    opts = gerbil.default_opts()
    bins = ctx.partition(s, o, k, p["m"], p["nbins"], opts, p.get("bin_bounds"))
    info = bins.info()
    for mc in (1, p["min_count"]):
        res = ctx.count_batch(bins, None, k, mc, opts)
        st = res.info()[2]
        keys, counts = res.torch_views()
        got[mc] = device_pass_rows(keys, counts, k, npass, 0)
        if mc == 1:
            total = int((counts.to(torch.int64) & 0xFFFFFFFF).sum().item())
            assert st["distinct"] == counts.numel() == st["emitted"]
            occ = st["occurrences"]
        del keys, counts
        res.free()
    bins.free()
    del s, o
    gerbil.gerbil_trim(ctx.handle)  # the next tests need the memory these tables held
    torch.cuda.empty_cache()
    windows = oracle.windows(seq, offs, k)
    assert info["n_kmers"] == windows == occ == total
    wk, wc = pool.result()[0]
    for mc, rows in got.items():
        sel = wc >= mc
        assert_same_rows(rows, (wk[sel], wc[sel]))
    assert len(got[1][1]) > 1000  # the pass is not vacuous


def test_serving_small_jobs_full_scale_equal_oracle_mixed_and_alone(g):
    """The serving stream's jobs on genomes of at most 5 Mbp, at full scale, submitted together
    to one server: each job's rows of the oracle pass's keys (1/8 of the keys, every read) equal
    the oracle's, and each job's whole result in the mix has the digest of the same job run
    alone."""
    from tests._oracle_pool import PassCount
    from tests._util import device_digest, device_pass_rows
    gerbil, ctx, torch = g
    jobs = [j for j in synth.serving_jobs(48) if j["genome"] <= 5e6]
    assert len(jobs) >= 10
    reads = [synth.t_serving_reads(j, "cuda") for j in jobs]
    host = [(s.cpu().numpy(), o.cpu().numpy().view(np.uint64)) for s, o in reads]
    npass = 8
    pool = PassCount([(hs, ho, j["k"], True, npass, 0) for (hs, ho), j in zip(host, jobs)])
    server = gerbil.Server(0, hbm_budget_bytes=int(150e9), slots=4)
    ids = [server.submit(s, o, j["k"], j["m"], j["nbins"], j["min_count"]) for (s, o), j in zip(reads, jobs)]
    mixed, digests = [], []
    for jid, j in zip(ids, jobs):
        res, _ = server.wait(jid)
        keys, counts = res.torch_views()
        mixed.append(device_pass_rows(keys, counts, j["k"], npass, 0))
        digests.append(device_digest(keys, counts, j["k"]))
        del keys, counts
        res.free()
    st = server.stats()
    server.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["max_concurrent"] >= 2
    for (s, o), j, dg in zip(reads, jobs, digests):
        bins = ctx.partition(s, o, j["k"], j["m"], j["nbins"])
        alone = ctx.count_batch(bins, None, j["k"], j["min_count"])
        keys, counts = alone.torch_views()
        assert device_digest(keys, counts, j["k"]) == dg
        del keys, counts
        alone.free()
        bins.free()
    for (hs, ho), j, rows, (wk, wc) in zip(host, jobs, mixed, pool.result()):
        assert_same_rows(rows, (wk, wc))
        assert int(wc.sum()) > 0
