"""GPU tests of the serving loop (tj_server_*): every request's result equals
the CPU oracle's and is the same alone and in a concurrent mix, admission
never exceeds the budget, an oversized request is rejected with
TJ_ERR_BUDGET, and latency percentiles are reported."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_21237_gb300 import api, datagen
from gpu_util import DEV, assert_pairs_equal, np_of

pytestmark = pytest.mark.gpu


def _requests(n, seed):
    sizes_r = datagen.log_uniform_sizes(n, 1e3, 3e5, seed)
    sizes_s = datagen.log_uniform_sizes(n, 1e3, 3e5, seed + 1)
    reqs = []
    for i, (a, b) in enumerate(zip(sizes_r, sizes_s)):
        kr, ir, ks, is_ = datagen.fk_zipf(a, b, 1.0, seed + 10 + i, device="cuda")
        reqs.append((kr, ir, ks, is_))
    return reqs


def test_results_same_alone_and_in_the_mix():
    reqs = _requests(24, 100)
    alone = [api.join_inner(*r).clone() for r in reqs]
    sorts_alone = []
    for kr, ir, _, _ in reqs[:6]:
        k, i = kr.clone(), ir.clone()
        api.sort(k, i)
        sorts_alone.append((k, i))
    outs = [torch.full((ks.numel(), 2), -1, dtype=torch.int64, device=DEV)
            for _, _, ks, _ in reqs]
    sorted_mix = [(kr.clone(), ir.clone()) for kr, ir, _, _ in reqs[:6]]
    # the workers' streams do not wait for this one: inputs and outputs ready first
    torch.cuda.synchronize()
    srv = api.Server(mem_budget_bytes=256 << 20, workers=6)
    tickets = []
    for (kr, ir, ks, is_), out in zip(reqs, outs):
        tickets.append(srv.submit(api.Server.join_request(kr, ir, ks, is_, out)))
    for k, i in sorted_mix:
        tickets.append(srv.submit(api.Server.sort_request(k, i)))
    res = [srv.wait(t) for t in tickets]
    rep = srv.report()
    srv.close()
    for r in res:
        assert r["status"] == 0
    for j, (kr, ir, ks, is_) in enumerate(reqs):
        n = res[j]["out_count"]
        exp = oracle.join_inner(np_of(kr), np_of(ir), np_of(ks), np_of(is_))
        assert n == exp.shape[0]
        assert_pairs_equal(outs[j][:n], exp)
        assert torch.equal(outs[j][:n], alone[j])
    for (k, i), (ka, ia), (kr, ir, _, _) in zip(sorted_mix, sorts_alone, reqs[:6]):
        ek, ei = oracle.sort(np_of(kr), np_of(ir))
        assert np.array_equal(np_of(k), ek) and np.array_equal(np_of(i), ei)
        assert torch.equal(k, ka) and torch.equal(i, ia)
    assert rep["completed"] == len(tickets)
    assert rep["peak_reserved"] <= 256 << 20
    assert rep["peak_inflight"] >= 2  # requests overlapped
    assert 0 < rep["p50_ms"] <= rep["p99_ms"] <= rep["max_ms"]


def test_oversized_request_is_rejected():
    kr, ir, ks, is_ = datagen.fk_zipf(200_000, 400_000, 0.0, 7, device="cuda")
    out = torch.empty((400_000, 2), dtype=torch.int64, device=DEV)
    torch.cuda.synchronize()
    srv = api.Server(mem_budget_bytes=1 << 20, workers=2)
    t = srv.submit(api.Server.join_request(kr, ir, ks, is_, out))
    assert srv.wait(t)["status"] == api.TJ_ERR_BUDGET
    srv.close()


def test_replay_poisson_stream():
    reqs = _requests(16, 300)
    outs = [torch.empty((r[2].numel(), 2), dtype=torch.int64, device=DEV) for r in reqs]
    torch.cuda.synchronize()  # inputs complete before the workers' streams read them
    srv = api.Server(mem_budget_bytes=1 << 30, workers=4)
    arrivals = datagen.poisson_arrivals(2000.0, len(reqs), 5)
    tickets = srv.replay([api.Server.join_request(*r, o) for r, o in zip(reqs, outs)], arrivals)
    res = [srv.wait(t) for t in tickets]
    rep = srv.report()
    srv.close()
    assert all(r["status"] == 0 for r in res)
    assert rep["completed"] == 16 and rep["makespan_s"] > 0
    for (kr, ir, ks, is_), o, r in zip(reqs, outs, res):
        exp = oracle.join_inner(np_of(kr), np_of(ir), np_of(ks), np_of(is_))
        assert r["out_count"] == exp.shape[0]
        assert_pairs_equal(o[: r["out_count"]], exp)


def test_blocked_head_is_passed_at_most_eight_times():
    # X and H each need most of the budget: while X runs, H waits at the head
    # of the queue; the small requests behind it fit and may go first, but H
    # is passed at most 8 times, then the queue waits for it
    n = 15_000_000
    big = [datagen.fk_zipf(n, n, 0.0, 900 + i, device="cuda") for i in range(2)]
    smalls = [datagen.fk_zipf(10_000, 20_000, 1.0, 910 + i, device="cuda") for i in range(24)]
    foot = 2 * n * 34 + n * 16 + (2 << 20)  # the server's footprint of a big request
    torch.cuda.synchronize()  # inputs complete before the workers' streams read them
    srv = api.Server(mem_budget_bytes=int(1.5 * foot), workers=4)
    reqs = [api.Server.join_request(*r) for r in big + smalls]
    tickets = srv.replay(reqs, [0.0] * len(reqs))
    res = [srv.wait(t) for t in tickets]
    rep = srv.report()
    srv.close()
    assert all(r["status"] == 0 for r in res), [(i, r) for i, r in enumerate(res) if r["status"]]
    assert [r["out_count"] for r in res] == [r[2].numel() for r in big + smalls]  # |J| = |S|
    assert 1 <= rep["bypasses"] <= 8
    assert rep["peak_reserved"] <= int(1.5 * foot)


def test_each_ticket_is_collected_once():
    kr, ir, ks, is_ = datagen.fk_zipf(1000, 3000, 0.5, 920, device="cuda")
    torch.cuda.synchronize()
    srv = api.Server(mem_budget_bytes=1 << 30, workers=2)
    t = srv.submit(api.Server.join_request(kr, ir, ks, is_))
    assert srv.wait(t)["status"] == 0
    with pytest.raises(api.TjError) as ei:
        srv.wait(t)
    assert ei.value.status == api.TJ_ERR_INVALID
    with pytest.raises(api.TjError):
        srv.wait(12345)
    srv.close()
