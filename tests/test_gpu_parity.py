"""Parity of the CUDA path with the oracle: bit-exact on every compared limb.

All products go through libgf2x_gb300.so's C ABI (via the ctypes binding);
expected values come only from oracle/ on the same seeded inputs."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu

CONFIG_SIZES = [12323, 17669, 24659, 35851, 40973, 57637]


@pytest.fixture(scope="module")
def ctx():
    from paper_2201_10473_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def check_batch(ctx, a, b, n, reduce, persistent=False):
    out = ctx.mul_strided(to_dev(a), to_dev(b), n, reduce, persistent=persistent)
    torch.cuda.synchronize()
    got = to_host(out)
    exp = oracle.mul_batch(a, b, n, reduce=reduce)
    assert np.array_equal(got, exp), first_diff(got, exp)


# ------------------------------------------------------------ edge sizes

EDGE_N = [1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 500, 1000, 1023, 1024, 1025,
          2047, 2048, 4095, 4097, 9999]


@pytest.mark.parametrize("n", EDGE_N)
@pytest.mark.parametrize("reduce", [False, True])
def test_edge_sizes_default_plan(ctx, n, reduce):
    a, b = wl.dense_pair(1000 + n, n, 5)
    # special operands: zero, all ones, single top bit, X^0
    L = wl.limbs(n)
    a[1] = 0
    b[2] = wl.mask_top(np.full(L, np.uint64(0xFFFFFFFFFFFFFFFF)), n)
    a[3] = 0
    a[3][(n - 1) // 64] = np.uint64(1 << ((n - 1) % 64))
    b[4] = 0
    b[4][0] = np.uint64(1)
    check_batch(ctx, a, b, n, reduce)


@pytest.mark.parametrize("n", CONFIG_SIZES)
@pytest.mark.parametrize("reduce", [False, True])
def test_config_sizes_default_plan(ctx, n, reduce):
    a, b = wl.dense_pair(2000 + n, n, 12)
    check_batch(ctx, a, b, n, reduce)


# ------------------------------------------------------------ plan space

PLANS_17669 = [
    "T2.K3.K2.K2.K2/8", "T2.K2.K2.K2.K2.K2/6", "T1.K3.K2.K2.K2/8", "T4.K3.K2.K2.K2/10", "T8.K3.K2.K2.K2/10",
    "T16.K3.K3.K2.K2/8", "K3.K3.K2.K2.K2/10", "K5.K2.K2.K2.K2/8", "K3.K2.K2.K2.K2.K2/6", "K2.K2.K2.K2.K2.K2/10",
    "T2.K3.K2.K2/16", "T2.K3.K2.K2.K2.K2/4", "T2.K5.K2.K2/12", "T2.K3.K2.K2.K2/8/256/0", "T2.K3.K2.K2.K2/8/0/1",
    "K3.K3.K2.K2.K2/10/0/1", "T2.T2.K3.K2/12", "K2.T1.K3.K2.K2/8", "T3.K3.K2.K2.K2/8", "T5.K2.K2.K2.K2.K2/8",
    "T2.K3.K2.K2.K2/8/0/0/1", "T2.K2.K2.K2.K2.K2/6/0/0/1", "T2.K3.K2.K2.K2.K2/4/0/0/1", "T2.K3.K2.K2.K2/8/0/1/1",
    "K3.K3.K2.K2.K2/10/0/0/1", "T1.K3.K2.K2.K2/8/128/0/1", "T2.K3.K2.K2/16/0/0/0", "K5.K2.K2.K2.K2/8/0/1/1",
]


@pytest.mark.parametrize("spec", PLANS_17669)
def test_plan_space_hqc128(ctx, spec):
    n = 17669
    ctx.set_plan(n, spec)
    try:
        a, b = wl.dense_pair(3000, n, 6)
        check_batch(ctx, a, b, n, True)
        check_batch(ctx, a, b, n, False)
    finally:
        ctx.set_plan(n, None)


PLANS_57637 = ["T16.K5.K2.K2.K2.K2/8/0/1", "K5.K2.K2.K2.K2.K2/12/0/1", "T8.K5.K2.K2.K2/16/0/1",
               "T2.K3.K3.K2.K2.K2/10/0/1", "T16.K5.K3.K2.K2/12/0/1", "T16.K5.K2.K2.K2.K2/8/0/1/1",
               "T16.K5.K2.K2.K2.K2/10/0/1/1", "T4.K5.K3.K2.K2.K2/6/0/1/1"]


@pytest.mark.parametrize("spec", PLANS_57637)
def test_plan_space_hqc256(ctx, spec):
    n = 57637
    ctx.set_plan(n, spec)
    try:
        a, b = wl.dense_pair(3100, n, 3)
        check_batch(ctx, a, b, n, True)
    finally:
        ctx.set_plan(n, None)


@pytest.mark.parametrize("n", [17669, 35851, 57637])
def test_checked_mode_reports_no_violation(ctx, n):
    ctx.set_checked(True)
    try:
        a, b = wl.dense_pair(3200, n, 4)
        check_batch(ctx, a, b, n, True)
        ctx.sync_status()
    finally:
        ctx.set_checked(False)


# ------------------------------------------------------------ entry points

@pytest.mark.parametrize("n", [12323, 17669, 57637])
def test_single_product_entry_points(ctx, n):
    a, b = wl.dense_pair(4000 + n, n, 1)
    da, db = to_dev(a[0]), to_dev(b[0])
    c = to_host(ctx.mul(da, db, n))
    r = to_host(ctx.mulmod(da, db, n))
    assert np.array_equal(c, oracle.mul(a[0], b[0], n))
    assert np.array_equal(r, oracle.mulmod(a[0], b[0], n))


def test_high_input_bits_are_ignored(ctx):
    n = 17669
    a, b = wl.dense_pair(4100, n, 4)
    ga, gb = a.copy(), b.copy()
    ga[:, -1] |= np.uint64(0xFFFFFFFFFFFFFFFF ^ ((1 << (n % 64)) - 1))
    gb[:, -1] |= np.uint64(0xFFFFFFFFFFFFFFFF ^ ((1 << (n % 64)) - 1))
    for reduce in (False, True):
        got = to_host(ctx.mul_strided(to_dev(ga), to_dev(gb), n, reduce))
        assert np.array_equal(got, oracle.mul_batch(a, b, n, reduce=reduce))


def test_persistent_equals_plain(ctx):
    n = 17669
    a, b = wl.dense_pair(4200, n, 700)
    da, db = to_dev(a), to_dev(b)
    p1 = to_host(ctx.mul_strided(da, db, n, True, persistent=False))
    p2 = to_host(ctx.mul_strided(da, db, n, True, persistent=True))
    assert np.array_equal(p1, p2)
    sample = np.arange(0, 700, 37)
    assert np.array_equal(p1[sample], oracle.mul_batch(a[sample], b[sample], n, reduce=True))


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("largest_first", [False, True])
def test_mixed_batch_host_items(ctx, persistent, largest_first):
    sizes = wl.shuffle(77, [17669] * 6 + [35851] * 4 + [57637] * 3 + [12323] * 2 + [1000, 64, 1])
    ops = wl.mixed_operands(5000, sizes)
    items, outs = [], []
    for (a, b), n in zip(ops, sizes):
        o = torch.zeros(wl.limbs(n), dtype=torch.int64, device="cuda")
        items.append((to_dev(a), to_dev(b), o, n, True))
        outs.append(o)
    ctx.mul_batched(items, persistent=persistent, largest_first=largest_first)
    torch.cuda.synchronize()
    for (a, b), n, o in zip(ops, sizes, outs):
        assert np.array_equal(to_host(o), oracle.mulmod(a, b, n)), n


def test_mixed_batch_device_items(ctx):
    from paper_2201_10473_gb300 import Context, pack_items
    c2 = Context(0)
    try:
        sizes_set = [17669, 35851, 57637]
        for n in sizes_set:  # one leaf size over the prepared plans
            c2.set_plan(n, {17669: "T2.K3.K2.K2.K2/8", 35851: "T2.K3.K2.K2.K2.K2/8/0/1",
                            57637: "T16.K5.K2.K2.K2.K2/8/0/1"}[n])
        c2.prepare(sizes_set)
        sizes = wl.shuffle(78, [17669] * 5 + [35851] * 4 + [57637] * 3)
        ops = wl.mixed_operands(5100, sizes)
        keep, rows, outs = [], [], []
        for (a, b), n in zip(ops, sizes):
            da, db = to_dev(a), to_dev(b)
            o = torch.zeros(wl.limbs(n), dtype=torch.int64, device="cuda")
            keep += [da, db]
            outs.append(o)
            rows.append((da.data_ptr(), db.data_ptr(), o.data_ptr(), n, 1))
        items = pack_items(rows).cuda()
        c2.mul_batched_device(items, len(rows), persistent=True)
        c2.sync_status()
        for (a, b), n, o in zip(ops, sizes, outs):
            assert np.array_equal(to_host(o), oracle.mulmod(a, b, n)), n
    finally:
        c2.close()


def test_argument_errors(ctx):
    from paper_2201_10473_gb300 import Gf2xError
    n = 17669
    a, b = wl.dense_pair(4300, n, 2)
    da, db = to_dev(a), to_dev(b)
    with pytest.raises(Gf2xError) as e:      # output overlaps an input
        ctx.mul_strided(da, db, n, True, out=da)
    assert e.value.status == 1
    with pytest.raises(Gf2xError) as e:      # n = 0
        ctx.mulmod(da[0], db[0], 0)
    assert e.value.status == 5
    with pytest.raises(Gf2xError):           # plan that does not cover n
        ctx.set_plan(n, "K2/8")


# ------------------------------------------------------------ closed forms at full size

def binom(m: int, L: int) -> np.ndarray:
    out = np.zeros(L, dtype=np.uint64)
    j = np.arange(m + 1)
    for pos in np.nonzero((j & m) == j)[0]:
        out[pos // 64] |= np.uint64(1 << (int(pos) % 64))
    return out


@pytest.mark.parametrize("n", CONFIG_SIZES)
def test_lucas_products_on_gpu(ctx, n):
    """(1+X)^p (1+X)^q = (1+X)^(p+q) at every workload size, computed on the GPU."""
    L = wl.limbs(n)
    pq = [(n - 1, n - 1), (n // 2, n // 3), (12345 % n, 777)]
    a = np.stack([binom(p, L) for p, _ in pq])
    b = np.stack([binom(q, L) for _, q in pq])
    got = to_host(ctx.mul_strided(to_dev(a), to_dev(b), n, False))
    for i, (p, q) in enumerate(pq):
        assert np.array_equal(got[i], binom(p + q, wl.limbs(2 * n - 1))), (p, q)


@pytest.mark.parametrize("n", [17669, 57637])
def test_sparse_weight_131_through_dense_path(ctx, n):
    a = wl.dense_operands(4400, n, 4, 0)
    b = wl.sparse_operands(4400, n, 131, 4)
    assert all(int(np.unpackbits(row.view(np.uint8)).sum()) == 131 for row in b)
    check_batch(ctx, a, b, n, True)


def _device_item_ctx():
    from paper_2201_10473_gb300 import Context
    c2 = Context(0, plan_db=None)
    plans = {17669: "T2.K3.K2.K2.K2/8", 35851: "T2.K3.K2.K2.K2.K2/8/0/1", 57637: "T16.K5.K2.K2.K2.K2/8/0/1"}
    for n, s in plans.items():
        c2.set_plan(n, s)
    c2.prepare(list(plans))
    return c2


def test_device_items_padding_and_cuda_graph_replay():
    """Empty (n = 0) slots are skipped; a captured persistent launch replays
    correctly, also after the operands change in place."""
    from paper_2201_10473_gb300 import pack_items
    c2 = _device_item_ctx()
    try:
        sizes = wl.shuffle(79, [17669] * 3 + [35851] * 2 + [57637] * 2)
        ops = wl.mixed_operands(5200, sizes)
        dev, rows, outs = [], [], []
        for (a, b), n in zip(ops, sizes):
            da, db = to_dev(a), to_dev(b)
            o = torch.zeros(wl.limbs(n), dtype=torch.int64, device="cuda")
            dev.append((da, db))
            outs.append(o)
            rows.append((da.data_ptr(), db.data_ptr(), o.data_ptr(), n, 1))
            rows.append((0, 0, 0, 0, 0))                      # padding slot
        items = pack_items(rows).cuda()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            c2.mul_batched_device(items, len(rows), persistent=True)   # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            c2.mul_batched_device(items, len(rows), persistent=True)
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        c2.sync_status()
        for (a, b), n, o in zip(ops, sizes, outs):
            assert np.array_equal(to_host(o), oracle.mulmod(a, b, n)), n
        # new operand values, same buffers: replay computes the new products
        ops2 = wl.mixed_operands(5300, sizes)
        for (a, b), (da, db) in zip(ops2, dev):
            da.copy_(to_dev(a))
            db.copy_(to_dev(b))
        g.replay()
        torch.cuda.synchronize()
        for (a, b), n, o in zip(ops2, sizes, outs):
            assert np.array_equal(to_host(o), oracle.mulmod(a, b, n)), n
    finally:
        c2.close()


def test_device_item_without_plan_is_reported():
    from paper_2201_10473_gb300 import Gf2xError, pack_items
    c2 = _device_item_ctx()
    try:
        n = 1000   # not prepared
        a, b = wl.dense_pair(5400, n, 1)
        da, db = to_dev(a[0]), to_dev(b[0])
        o = torch.zeros(wl.limbs(n), dtype=torch.int64, device="cuda")
        items = pack_items([(da.data_ptr(), db.data_ptr(), o.data_ptr(), n, 1)]).cuda()
        c2.mul_batched_device(items, 1)
        with pytest.raises(Gf2xError) as e:
            c2.sync_status()
        assert e.value.status == 7
        c2.sync_status()   # the report is cleared
    finally:
        c2.close()


def test_replayed_graph_refuses_a_plan_changed_under_it():
    """A graph captured for one leaf size, replayed after the size's plan was
    switched to another leaf: the kernel refuses the item and reports it,
    instead of running a plan it was not built for."""
    from paper_2201_10473_gb300 import Gf2xError, pack_items
    from paper_2201_10473_gb300 import Context
    c2 = Context(0, plan_db=None)
    try:
        n = 17669
        c2.set_plan(n, "T2.K3.K2.K2.K2/8")
        c2.prepare([n])
        a, b = wl.dense_pair(5500, n, 2)
        da, db = to_dev(a), to_dev(b)
        o = torch.zeros((2, wl.limbs(n)), dtype=torch.int64, device="cuda")
        items = pack_items([(da[i].data_ptr(), db[i].data_ptr(), o[i].data_ptr(), n, 1) for i in range(2)]).cuda()
        c2.mul_batched_device(items, 2)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            c2.mul_batched_device(items, 2)
        c2.set_plan(n, "T2.K2.K2.K2.K2.K2/6")      # another leaf size, published for device items
        o.zero_()
        g.replay()
        torch.cuda.synchronize()
        with pytest.raises(Gf2xError) as e:
            c2.sync_status()
        assert e.value.status == 7
        assert int(o.abs().sum()) == 0               # nothing was written
    finally:
        c2.close()


# ------------------------------------------------------------ split plans (top level across CTAs)

SPLIT_PLANS = [
    (17669, "T2.K2.K2.K2.K2.K2/6/128/1/0/1"), (17669, "K3.K2.K2.K2.K2.K2/6/0/0/1/1"),
    (57637, "T16.K5.K2.K2.K2.K2/8/0/0/1/1"), (57637, "T16.K2.K2.K2.K2.K2.K2/10/448/1/1/1"),
    (57637, "K5.K2.K2.K2.K2.K2/12/0/1/0/1"), (35851, "T4.K2.K2.K2.K2.K2.K2/6/0/1/1/1"),
    (100000, None), (131072, None), (120001, None),
]


@pytest.mark.parametrize("n,spec", SPLIT_PLANS)
def test_split_plans(ctx, n, spec):
    """The top level evaluated/interpolated by its own kernels through global
    scratch, the children as independent products: bit-exact, batched and single."""
    if spec is not None:
        ctx.set_plan(n, spec)
    try:
        sp = ctx.get_plan(n)
        a, b = wl.dense_pair(7000 + n, n, 5)
        check_batch(ctx, a, b, n, True)
        check_batch(ctx, a, b, n, False)
        check_batch(ctx, a, b, n, True, persistent=True)
        da, db = to_dev(a[0]), to_dev(b[0])
        assert np.array_equal(to_host(ctx.mulmod(da, db, n)), oracle.mulmod(a[0], b[0], n)), sp
        ctx.sync_status()
    finally:
        if spec is not None:
            ctx.set_plan(n, None)


def test_split_plan_in_checked_mode_and_large_batch_chunks(ctx):
    n = 131072
    ctx.set_checked(True)
    try:
        a, b = wl.dense_pair(7100, n, 3)
        check_batch(ctx, a, b, n, True)
        ctx.sync_status()
    finally:
        ctx.set_checked(False)
