"""Serving: jobs of different k admitted by an HBM budget and run concurrently must give, each,
the same rows as the oracle and as the same job run alone (integers: no tolerance)."""
import numpy as np
import pytest

import oracle
from paper_1607_06618_b300 import synth
from tests._util import assert_same_rows, sort_rows

pytestmark = pytest.mark.gpu

M_FOR_K = {32: 7, 65: 9, 127: 11}


def _job(j):
    import torch
    gen = synth.t_genome(20000 + 7000 * j, 6000 + j, device="cuda")
    k = (32, 65, 127)[j % 3]
    seq, off = synth.t_sampled_reads(gen, 1500 + 300 * j, 150, 0.005, 6100 + j, p_n=0.005)
    return seq, off, k


def test_server_mixed_equals_alone_and_oracle():
    import torch
    from paper_1607_06618_b300 import gerbil
    jobs = [_job(j) for j in range(9)]
    # budget for about two jobs at a time (the estimate assumes every k-mer distinct)
    server = gerbil.Server(0, hbm_budget_bytes=int(0.45e9), slots=3)
    ids = [server.submit(s, o, k, M_FOR_K[k], 16, 1) for s, o, k in jobs]
    mixed = []
    for jid in ids:
        res, times = server.wait(jid)
        mixed.append(res.to_host())
        assert times["latency_ms"] >= times["run_ms"] >= 0
        res.free()
    st = server.stats()
    server.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["max_concurrent"] >= 2  # admitted jobs overlapped
    ctx = gerbil.Context(0)
    for (s, o, k), got in zip(jobs, mixed):
        bins = ctx.partition(s, o, k, M_FOR_K[k], 16)
        alone = ctx.count_batch(bins, None, k, 1)
        ak, ac = alone.to_host()
        alone.free()
        bins.free()
        assert_same_rows(got, (ak, ac))
        seq = s.cpu().numpy()
        offs = o.cpu().numpy().view(np.uint64)
        assert_same_rows(got, oracle.count(seq, offs, k, min_count=1))
    ctx.close()


def test_server_job_larger_than_budget_runs_alone():
    from paper_1607_06618_b300 import gerbil
    s, o, k = _job(4)
    server = gerbil.Server(0, hbm_budget_bytes=1 << 20, slots=2)
    jid = server.submit(s, o, k, M_FOR_K[k], 8, 2)
    res, _ = server.wait(jid)
    got = res.to_host()
    res.free()
    server.close()
    assert_same_rows(got, oracle.count(s.cpu().numpy(), o.cpu().numpy().view(np.uint64), k, min_count=2))


def test_batch_counted_in_groups_under_table_limit():
    """Tables of a batch above the table limit: bins counted in groups, rows joined."""
    from paper_1607_06618_b300 import gerbil
    s, o, k = _job(1)
    ctx = gerbil.Context(0)
    bins = ctx.partition(s, o, k, M_FOR_K[k], 64)
    whole = ctx.count_batch(bins, None, k, 1)
    want = whole.to_host()
    whole_stats = whole.info()[2]
    whole.free()
    opts = gerbil.default_opts(max_table_mib=1)
    grouped = ctx.count_batch(bins, None, k, 1, opts)
    n, W, st = grouped.info()
    assert st["groups"] > 1 and st["bins"] == 64
    assert st["occurrences"] == whole_stats["occurrences"] and st["distinct"] == whole_stats["distinct"]
    assert_same_rows(grouped.to_host(), want)
    keys, cnts = grouped.torch_views()  # joins the groups' rows into one device buffer
    assert_same_rows((keys.cpu().numpy().view(np.uint64), cnts.cpu().numpy().view(np.uint32)), want)
    assert_same_rows(grouped.to_host(), want)
    grouped.free()
    bins.free()
    ctx.close()
    assert_same_rows(want, oracle.count(s.cpu().numpy(), o.cpu().numpy().view(np.uint64), k, min_count=1))
