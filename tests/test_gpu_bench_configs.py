"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times: the same seeded inputs, the tuned plan database with the
benchmark's batch, every launch form the benchmark reports.  Rows sampled
across each batch (first, last and evenly spaced) are compared bit for bit
with the oracle's product of Sec. 2.1, reduced mod X^n - 1 as in Sec. 1
(full product for the 12323-bit workload).  The whole batch is in addition
compared across launch forms, which must agree everywhere."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu


def _sample(count, k=12):
    return np.unique(np.concatenate([np.linspace(0, count - 1, k).astype(np.int64), [0, count - 1]]))


@pytest.mark.parametrize("key,n,count", [(2, 17669, 4096), (4, 57637, 2048)])
def test_headline_batch_every_launch_form(key, n, count):
    """4096 x 17669 (HQC-128 shape) and 2048 x 57637 (HQC-256 shape), mod X^n - 1:
    one launch of one CTA per product, the persistent grid, and the
    host-buffer entry with its chunked copies."""
    from paper_2201_10473_gb300 import Context
    ctx = Context(0, batch_hint=count)
    try:
        a, b = wl.dense_pair(wl.BASE_SEED + key, n, count)
        da, db = to_dev(a), to_dev(b)
        one = to_host(ctx.mul_strided(da, db, n, True))
        pers = to_host(ctx.mul_strided(da, db, n, True, persistent=True))
        pa = torch.from_numpy(a.view(np.int64)).pin_memory()
        pb = torch.from_numpy(b.view(np.int64)).pin_memory()
        st = torch.cuda.Stream()
        host = ctx.mul_strided_host(pa, pb, n, True, stream=st)
        st.synchronize()
        ctx.sync_status()
        host = host.numpy().view(np.uint64)
        assert np.array_equal(pers, one), first_diff(pers, one)
        assert np.array_equal(host, one), first_diff(host, one)
        s = _sample(count)
        assert np.array_equal(one[s], oracle.mul_batch(a[s], b[s], n, reduce=True))
    finally:
        ctx.close()


def test_large_degree_batch_dense_and_sparse():
    """16384 x 57637 mod X^n - 1: dense operands, the weight-131 variant
    through the dense path, and the same sparse operands by their positions
    through the sparse x dense kernel."""
    from paper_2201_10473_gb300 import Context
    n, count = 57637, 16384
    ctx = Context(0, batch_hint=count)
    try:
        seed = wl.workload(4).seed
        a, b = wl.dense_pair(seed, n, count)
        bs = wl.sparse_operands(seed, n, 131, count)
        rows = [np.flatnonzero(np.unpackbits(r.view(np.uint8), bitorder="little")) for r in bs]
        assert all(len(r) == 131 and r[-1] < n for r in rows)
        pos = np.stack(rows)
        da, db, dbs = to_dev(a), to_dev(b), to_dev(bs)
        dense = to_host(ctx.mul_strided(da, db, n, True))
        sparse_dense = to_host(ctx.mul_strided(da, dbs, n, True))
        by_pos = to_host(ctx.mulmod_sparse(da, torch.from_numpy(pos.astype(np.int32)).cuda(), n))
        ctx.sync_status()
        assert np.array_equal(by_pos, sparse_dense), first_diff(by_pos, sparse_dense)
        s = _sample(count, 8)
        assert np.array_equal(dense[s], oracle.mul_batch(a[s], b[s], n, reduce=True))
        assert np.array_equal(sparse_dense[s], oracle.mul_batch(a[s], bs[s], n, reduce=True))
    finally:
        ctx.close()


def test_small_size_full_products_batched_and_plain():
    """256 x 12323, full products: the batched launch and one launch per
    product with the single-product plan, every row against the oracle."""
    from paper_2201_10473_gb300 import Context, autotune
    n, count = 12323, 256
    ctx = Context(0, batch_hint=count)
    plain = Context(0, plan_db=None)
    try:
        plain.set_plan(n, autotune.single_product_plans([n])[n])
        a, b = wl.dense_pair(wl.BASE_SEED + 1, n, count)
        da, db = to_dev(a), to_dev(b)
        batched = to_host(ctx.mul_strided(da, db, n, False))
        out = torch.zeros((count, (2 * n - 1 + 63) // 64), dtype=torch.int64, device="cuda")
        for p in range(count):
            plain.mul(da[p], db[p], n, out=out[p])
        one_by_one = to_host(out)
        ctx.sync_status()
        plain.sync_status()
        exp = oracle.mul_batch(a, b, n, reduce=False)
        assert np.array_equal(batched, exp), first_diff(batched, exp)
        assert np.array_equal(one_by_one, exp), first_diff(one_by_one, exp)
    finally:
        ctx.close()
        plain.close()
