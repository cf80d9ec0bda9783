"""Serving loop: every result is the same alone and in the mix (tolerance 0)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

SIZES = list(wl.SERVING_SIZES)


def _collector(reqs, pool, results):
    def collect(rs, addrs, ns):
        base = pool.arena.data_ptr()
        for r, ad, n in zip(rs, addrs, ns):
            L = wl.limbs(int(n))
            off = (int(ad) - base) // 8
            results[int(r)] = pool.arena[off: off + L].clone()
    return collect


@pytest.mark.parametrize("use_graphs", [True, False])
def test_results_identical_alone_and_in_the_mix(use_graphs):
    from paper_2201_10473_gb300 import Context, serve
    ctx = Context(0)
    try:
        # one leaf size over the prepared plans (device-item batches)
        plans = {12323: "T2.K3.K2.K2.K2/6/0/0/1", 17669: "T2.K2.K2.K2.K2.K2/6/0/1/0",
                 24659: "T2.K3.K2.K2.K2.K2/6/0/1/1", 35851: "T4.K2.K2.K2.K2.K2.K2/6/0/1/1",
                 40973: "T2.K3.K3.K2.K2.K2/6/0/1/1", 57637: "T4.K5.K3.K2.K2.K2/6/0/1/1"}
        for n, s in plans.items():
            ctx.set_plan(n, s)
        count = 1500
        sizes = wl.uniform_choice(wl.BASE_SEED + 5, count, SIZES)
        reqs = serve.make_requests(sizes, lambda n, c: wl.dense_pair(wl.BASE_SEED + 5 + n, n, c))
        arrivals = wl.poisson_arrivals(wl.BASE_SEED + 5, count, 2e5)
        # a small budget forces admission to wait for retirements
        srv = serve.Server(ctx, {n: 1 for n in SIZES}, budget_bytes=serve.default_budget(SIZES, 300),
                           max_batch=256, streams=3, use_graphs=use_graphs)
        results = {}
        res = srv.run(reqs, arrivals, collect=_collector(reqs, srv.pool, results))
        ctx.sync_status()
        assert res.completed == count and len(results) == count
        assert res.batches > 3 and res.admission_waits > 0
        # alone: every request as its own single-product call
        for r in range(count):
            n = sizes[r]
            i = int(reqs.index[r])
            alone = ctx.mulmod(reqs.a[n][i], reqs.b[n][i], n)
            assert torch.equal(alone, results[r]), r
        # and the oracle on a sample
        for r in range(0, count, 97):
            n = sizes[r]
            i = int(reqs.index[r])
            a = reqs.a[n][i].cpu().numpy().view(np.uint64)
            b = reqs.b[n][i].cpu().numpy().view(np.uint64)
            assert np.array_equal(results[r].cpu().numpy().view(np.uint64), oracle.mulmod(a, b, n))
    finally:
        ctx.close()


def test_plain_baseline_serves_everything():
    from paper_2201_10473_gb300 import Context, serve
    ctx = Context(0)
    try:
        count = 300
        sizes = wl.uniform_choice(wl.BASE_SEED + 6, count, SIZES)
        reqs = serve.make_requests(sizes, lambda n, c: wl.dense_pair(wl.BASE_SEED + 6 + n, n, c))
        arrivals = wl.poisson_arrivals(wl.BASE_SEED + 6, count, 2e4)
        pool = serve.SlotPool({n: 1 for n in SIZES}, serve.default_budget(SIZES, 60))
        results = {}
        res = serve.serve_plain(ctx, reqs, arrivals, pool, streams=3, collect=_collector(reqs, pool, results))
        assert res.completed == count
        for r in range(0, count, 7):
            n = sizes[r]
            i = int(reqs.index[r])
            assert torch.equal(ctx.mulmod(reqs.a[n][i], reqs.b[n][i], n), results[r])
    finally:
        ctx.close()


@pytest.mark.parametrize("persistent", [True, False])
def test_size_aware_server_identical_alone_and_in_the_mix(persistent):
    """Both launch forms of the size-aware server: persistent CTAs taking the
    item slots from a counter, and one CTA per item slot."""
    from paper_2201_10473_gb300 import Context, autotune, serve
    plans = autotune.best_plans(autotune.packaged_log(), SIZES, 512, allow_split=False)
    assert set(plans) == set(SIZES)
    srv = serve.SizeAwareServer(plans, serve.default_budget(SIZES, 300), max_batch=256, streams_per_size=2,
                                persistent=persistent)
    ctx = Context(0)
    try:
        count = 1500
        sizes = wl.uniform_choice(wl.BASE_SEED + 7, count, SIZES)
        reqs = serve.make_requests(sizes, lambda n, c: wl.dense_pair(wl.BASE_SEED + 7 + n, n, c))
        arrivals = wl.poisson_arrivals(wl.BASE_SEED + 7, count, 2e5)
        results = {}
        res = srv.run(reqs, arrivals, collect=_collector(reqs, srv.pool, results))
        for c in srv.ctx.values():
            c.sync_status()
        assert res.completed == count and len(results) == count
        # the small budget bounds every batch to its size's share of the slots
        cap = max(srv.pool.capacity[n] // 2 for n in SIZES)
        assert res.batches >= count / cap and res.mean_batch <= cap
        for r in range(count):
            n = sizes[r]
            i = int(reqs.index[r])
            assert torch.equal(ctx.mulmod(reqs.a[n][i], reqs.b[n][i], n), results[r]), r
        for r in range(0, count, 101):
            n = sizes[r]
            i = int(reqs.index[r])
            a = reqs.a[n][i].cpu().numpy().view(np.uint64)
            b = reqs.b[n][i].cpu().numpy().view(np.uint64)
            assert np.array_equal(results[r].cpu().numpy().view(np.uint64), oracle.mulmod(a, b, n))
    finally:
        ctx.close()
        srv.close()
