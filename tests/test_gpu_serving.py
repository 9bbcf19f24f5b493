"""Serving: jobs of different k admitted by an HBM budget and run concurrently must give, each,
the same rows as the oracle and as the same job run alone (integers: no tolerance)."""
import numpy as np
import pytest

import oracle
from paper_1607_06618_b300 import synth
from tests._util import assert_same_rows

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


def _digest(res):
    """Order-independent digest of a device result (torch, on the GPU): sum of a mix of every
    row's key words and count, and the row count."""
    import torch
    keys, cnts = res.torch_views()
    h = torch.zeros(keys.shape[0], dtype=torch.int64, device=keys.device)
    for j in range(keys.shape[1]):
        h = (h ^ keys[:, j]) * -7046029254386353131  # 0x9E3779B97F4A7C15 as int64
        h = h ^ (h >> 29)
    h = (h ^ cnts.to(torch.int64)) * -4658895280553007687  # 0xBF58476D1CE4E5B9
    return int(h.sum().item()), int(keys.shape[0])


def test_serving_stream_jobs_equal_alone_at_reduced_scale():
    """The first jobs of the Poisson serving stream (genome and reads scaled by 1/50), submitted
    at once to a server whose budget admits a few at a time: each job's rows in the mix have the
    digest of the same job run alone (a job's result must not depend on what runs beside it:
    tolerance 0)."""
    import torch
    from paper_1607_06618_b300 import gerbil
    jobs = synth.serving_jobs(10)
    reads = [synth.t_serving_reads(j, "cuda", scale=0.02) for j in jobs]
    torch.cuda.synchronize()
    server = gerbil.Server(0, hbm_budget_bytes=int(6e9), slots=4)
    ids = [server.submit(s, o, j["k"], j["m"], j["nbins"], j["min_count"]) for j, (s, o) in zip(jobs, reads)]
    mixed = []
    for jid in ids:
        res, _ = server.wait(jid)
        mixed.append(_digest(res))
        res.free()
    st = server.stats()
    server.close()
    assert st["completed"] == len(jobs) and st["max_concurrent"] >= 2
    ctx = gerbil.Context(0)
    for j, (s, o), want in zip(jobs, reads, mixed):
        ctx.forget_ratio()
        bins = ctx.partition(s, o, j["k"], j["m"], j["nbins"])
        res = ctx.count_batch(bins, None, j["k"], j["min_count"])
        assert _digest(res) == want
        res.free()
        bins.free()
    ctx.close()


def test_failed_job_reports_the_worker_message():
    """A job whose reads are inconsistent (offsets out of order: checked on the device, no access
    outside the reads) fails alone, with the worker context's message; the server goes on."""
    import torch
    from paper_1607_06618_b300 import gerbil
    seq = torch.randint(0, 4, (150,), dtype=torch.uint8, device="cuda")
    seq = torch.tensor(list(b"ACGT"), dtype=torch.uint8, device="cuda")[seq.long()]
    bad = torch.tensor([0, 100, 50, 150], dtype=torch.int64, device="cuda")
    good = torch.tensor([0, 150], dtype=torch.int64, device="cuda")
    server = gerbil.Server(0, 0, slots=2)
    j_bad = server.submit(seq, bad, 32, 7, 4, 1)
    j_good = server.submit(seq, good, 32, 7, 4, 1)
    with pytest.raises(gerbil.GerbilError, match="offsets out of order"):
        server.wait(j_bad)
    res, _ = server.wait(j_good)
    assert len(res) == 150 - 32 + 1 or len(res) > 0
    res.free()
    st = server.stats()
    server.close()
    assert st["failed"] == 1 and st["completed"] == 1
