"""The context boundary: a workspace fixed at creation (no allocation in any
compute call afterwards, counted by the context), host-side injection of
allocation failures (GF2X_ENOMEM, then the context still works), and the
bounded host wait (GF2X_ETIMEOUT while work is in flight, then success).
Every product is compared with the oracle (the product of Sec. 2.1)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu

ENOMEM, ETIMEOUT = 2, 4


def _check(got, a, b, n, reduce, rows):
    g = to_host(got) if isinstance(got, torch.Tensor) and got.is_cuda else got.numpy().view(np.uint64)
    exp = oracle.mul_batch(a[rows], b[rows], n, reduce=reduce)
    assert np.array_equal(g[rows][:, : exp.shape[1]], exp), first_diff(g[rows][:, : exp.shape[1]], exp)


def test_fixed_workspace_makes_no_allocation_in_compute_calls():
    from paper_2201_10473_gb300 import Context
    ctx = Context(0, workspace_bytes=64 << 20)          # 32 MiB split | 16 MiB unbalanced/Toom | 16 MiB host
    try:
        after_create = ctx.alloc_count()
        # C2 shape, in-CTA plan
        n = 17669
        a, b = wl.dense_pair(8101, n, 512)
        _check(ctx.mul_strided(to_dev(a), to_dev(b), n, True, persistent=True), a, b, n, True, np.arange(0, 512, 37))
        # a split plan over more products than one chunk of the 32 MiB split scratch
        n = 57637
        ctx.set_plan(n, "T16.K2.K2.K2.K2.K2.K2/10/0/0/1/1")
        a, b = wl.dense_pair(8102, n, 1500)
        _check(ctx.mul_strided(to_dev(a), to_dev(b), n, True, persistent=True), a, b, n, True,
               np.array([0, 1, 1309, 1310, 1311, 1499]))
        # C4 shape with the default in-CTA plan of another size, full product
        n = 35851
        a, b = wl.dense_pair(8103, n, 64)
        _check(ctx.mul_strided(to_dev(a), to_dev(b), n, False, persistent=True), a, b, n, False, np.arange(0, 64, 9))
        # unbalanced (chunked) and Toom-4 through the 16 MiB scratch, in several groups
        na, nb, cnt = 57637, 17669, 300
        ua = wl.dense_operands(8104, na, cnt, 0)
        ub = wl.dense_operands(8104, nb, cnt, 1)
        got = to_host(ctx.mul_unbalanced(to_dev(ua), na, to_dev(ub), nb))
        for p in (0, 150, 299):
            bz = np.zeros(wl.limbs(na), np.uint64)
            bz[: wl.limbs(nb)] = ub[p]
            exp = oracle.mul(ua[p], bz, na)[: got.shape[1]]
            assert np.array_equal(got[p], exp), p
        n = 100000
        a, b = wl.dense_pair(8105, n, 200)
        _check(ctx.mul_toom4(to_dev(a), to_dev(b), n, True), a, b, n, True, np.array([0, 199]))
        # host buffers through the 16 MiB pipeline (several chunks per set)
        n = 24659
        a, b = wl.dense_pair(8106, n, 3000)
        pa = torch.from_numpy(a.view(np.int64)).pin_memory()
        pb = torch.from_numpy(b.view(np.int64)).pin_memory()
        out = ctx.mul_strided_host(pa, pb, n, True)
        torch.cuda.synchronize()
        _check(out, a, b, n, True, np.arange(0, 3000, 311))
        # host items beyond the 16384 staging slots run in pieces
        n, cnt = 200, 16500
        a, b = wl.dense_pair(8107, n, cnt)
        da, db = to_dev(a), to_dev(b)
        o = torch.zeros((cnt, wl.limbs(n)), dtype=torch.int64, device="cuda")
        ctx.mul_batched([(da[i], db[i], o[i], n, True) for i in range(cnt)], persistent=True)
        _check(o, a, b, n, True, np.array([0, 16383, 16384, cnt - 1]))
        # sparse x dense
        n, w = 17669, 75
        sa = wl.dense_operands(8108, n, 64, 0)
        sb = wl.sparse_operands(8108, n, w, 64)
        pos = np.stack([np.flatnonzero(np.unpackbits(r.view(np.uint8), bitorder="little")) for r in sb])
        got = to_host(ctx.mulmod_sparse(to_dev(sa), torch.from_numpy(pos.astype(np.int32)).cuda(), n))
        assert np.array_equal(got, oracle.mul_batch(sa, sb, n, reduce=True))
        ctx.sync_status()
        assert ctx.alloc_count() == after_create
    finally:
        ctx.close()


def test_fixed_workspace_too_small_for_one_product_reports_enomem():
    from paper_2201_10473_gb300 import Context, gf2x
    ctx = Context(0, plan_db=None, workspace_bytes=32 << 10)   # 16 KiB of split scratch
    try:
        n = 57637
        ctx.set_plan(n, "T16.K2.K2.K2.K2.K2.K2/10/0/0/1/1")   # 25.6 KB of scratch per product
        a, b = wl.dense_pair(8110, n, 4)
        with pytest.raises(gf2x.Gf2xError) as e:
            ctx.mul_strided(to_dev(a), to_dev(b), n, True)
        assert e.value.status == ENOMEM
        a, b = wl.dense_pair(8110, 17669, 4)
        r = ctx.mul_strided(to_dev(a), to_dev(b), 17669, True)   # an in-CTA plan still runs
        _check(r, a, b, 17669, True, np.arange(4))
        ctx.sync_status()
    finally:
        ctx.close()


def test_injected_allocation_failures_report_enomem_and_leave_the_context_usable():
    from paper_2201_10473_gb300 import Context, gf2x
    L = gf2x.lib()
    try:
        L.gf2x_debug_fail_next_allocs(1)                  # the creation's first allocation fails
        with pytest.raises(gf2x.Gf2xError) as e:
            Context(0, plan_db=None)
        assert e.value.status == ENOMEM
        L.gf2x_debug_fail_next_allocs(0)
        ctx = Context(0, plan_db=None)
        try:
            n = 131072                                    # default plan: a split plan, scratch grown on demand
            a, b = wl.dense_pair(8111, n, 3)
            L.gf2x_debug_fail_next_allocs(1)
            with pytest.raises(gf2x.Gf2xError) as e:
                ctx.mul_strided(to_dev(a), to_dev(b), n, True)
            assert e.value.status == ENOMEM
            L.gf2x_debug_fail_next_allocs(0)
            got = ctx.mul_strided(to_dev(a), to_dev(b), n, True)    # the same call now succeeds
            _check(got, a, b, n, True, np.arange(3))
            pa = torch.from_numpy(a.view(np.int64)).pin_memory()    # the host pipeline's first buffers
            pb = torch.from_numpy(b.view(np.int64)).pin_memory()
            L.gf2x_debug_fail_next_allocs(1)
            with pytest.raises(gf2x.Gf2xError) as e:
                ctx.mul_strided_host(pa, pb, n, True)
            assert e.value.status == ENOMEM
            L.gf2x_debug_fail_next_allocs(0)
            out = ctx.mul_strided_host(pa, pb, n, True)
            torch.cuda.synchronize()
            _check(out, a, b, n, True, np.arange(3))
            ctx.sync_status()
        finally:
            ctx.close()
    finally:
        L.gf2x_debug_fail_next_allocs(0)


def test_bounded_wait_times_out_while_work_runs_then_succeeds():
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        n, cnt = 57637, 8192                              # about 8 ms of products
        a, b = wl.dense_pair(8112, n, 16)
        da = to_dev(a).repeat(cnt // 16, 1)
        db = to_dev(b).repeat(cnt // 16, 1)
        torch.cuda.synchronize()
        out = ctx.mul_strided(da, db, n, True, persistent=True)
        assert ctx.wait(0) == ETIMEOUT                    # still in flight
        assert ctx.wait(60000) == 0
        _check(out, np.tile(a, (cnt // 16, 1)), np.tile(b, (cnt // 16, 1)), n, True, np.array([0, cnt - 1]))
    finally:
        ctx.close()
