"""Toom-4 and Toom-5 top levels (gf2x_mul_toom4, gf2x_mul_toom5): every row
equals the product of the regular path (gf2x_mul_strided) bit for bit, and
the oracle's on samples, full and reduced, from one-word operands up to
n = 131072, with garbage above n, padded strides, and batches larger than
one scratch group."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,count", [
    (1, 3), (33, 3), (129, 5), (257, 4), (4096, 9), (17669, 37), (57637, 5), (100000, 3), (131072, 3),
])
@pytest.mark.parametrize("reduce", [False, True])
@pytest.mark.parametrize("k", [4, 5])
def test_matches_regular_path_and_oracle(n, count, reduce, k):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        a, b = wl.dense_pair(9990 + n, n, count)
        a_g = a.copy()
        if n % 64:                                     # bits above n must be ignored
            a_g[:, -1] |= ~np.uint64((1 << (n % 64)) - 1)
        got = getattr(ctx, f"mul_toom{k}")(to_dev(a_g), to_dev(b), n, reduce)
        ref = ctx.mul_strided(to_dev(a), to_dev(b), n, reduce, persistent=True)
        ctx.sync_status()
        assert torch.equal(got, ref)
        host = to_host(got)
        for p in sorted({0, count - 1}):
            exp = oracle.mulmod(a[p], b[p], n) if reduce else oracle.mul(a[p], b[p], n)
            assert np.array_equal(host[p][: len(exp)], exp), p
    finally:
        ctx.close()


@pytest.mark.parametrize("k", [4, 5])
def test_padded_strides(k):
    from paper_2201_10473_gb300 import Context, gf2x
    n, count = 24659, 6
    L = wl.limbs(n)
    ctx = Context(0)
    try:
        a, b = wl.dense_pair(9991, n, count)
        pad = np.full((count, 3), np.uint64(0x3C3C3C3C3C3C3C3C))
        da, db = to_dev(np.concatenate([a, pad], 1)), to_dev(np.concatenate([b, pad], 1))
        out = torch.full((count, L + 2), -1, dtype=torch.int64, device="cuda")
        st = getattr(gf2x.lib(), f"gf2x_mul_toom{k}")(ctx._h, out.data_ptr(), da.data_ptr(), db.data_ptr(), n, count, L + 3, L + 2,
                                       gf2x.REDUCE, None)
        assert st == 0
        torch.cuda.synchronize()
        host = to_host(out)
        for p in range(count):
            assert np.array_equal(host[p, :L], oracle.mulmod(a[p], b[p], n)), p
        assert (host[:, L:] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    finally:
        ctx.close()


@pytest.mark.parametrize("k", [4, 5])
def test_batch_larger_than_one_scratch_group(k):
    """At n = 131072 a product needs 115 KB (Toom-4) or 119 KB (Toom-5) of
    scratch: 2400 products run as two groups of the 256 MiB buffer."""
    from paper_2201_10473_gb300 import Context
    n, count = 131072, 2400
    ctx = Context(0)
    try:
        a, b = wl.dense_pair(9992, n, count)
        got = to_host(getattr(ctx, f"mul_toom{k}")(to_dev(a), to_dev(b), n, True))
        for p in (0, 1000, 2327, 2328, count - 1):
            assert np.array_equal(got[p], oracle.mulmod(a[p], b[p], n)), p
    finally:
        ctx.close()


@pytest.mark.parametrize("n", [129, 17669, 57637, 131072])
@pytest.mark.parametrize("k", [4, 5])
def test_checked_mode_reports_no_violation(n, k):
    """In checked mode the interpolation kernel verifies every division
    (dropped words of x^a, the remainders by x+1 and x^2+x+1) and that each
    coefficient C_k fits its 2m words; correct tables report nothing."""
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        ctx.set_checked(True)
        count = 4
        a, b = wl.dense_pair(9993 + n, n, count)
        a[0] = np.uint64(0xFFFFFFFFFFFFFFFF)            # all-ones row: every word of every part set
        b[0] = np.uint64(0xFFFFFFFFFFFFFFFF)
        if n % 64:
            a[0, -1] &= np.uint64((1 << (n % 64)) - 1)
            b[0, -1] &= np.uint64((1 << (n % 64)) - 1)
        for reduce in (False, True):
            got = to_host(getattr(ctx, f"mul_toom{k}")(to_dev(a), to_dev(b), n, reduce))
            ctx.sync_status()                           # raises on a reported violation
            for p in range(count):
                exp = oracle.mulmod(a[p], b[p], n) if reduce else oracle.mul(a[p], b[p], n)
                assert np.array_equal(got[p][: len(exp)], exp), (p, reduce)
    finally:
        ctx.set_checked(False)
        ctx.close()
