"""Shared-operand batches (GF2X_BATCH_SHARED_A): one a times every row of b.
Every row must equal the oracle's product of a and that row, and the whole
batch must equal the unshared call with a copied into every row (bit-exact),
for in-CTA and split plans, full and reduced products, persistent and
one-CTA-per-product launches, ragged counts and sparse rows of b (the key
operations of Sec. 1: a public key times low-weight vectors)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,count,reduce,persistent,spec", [
    (17669, 3000, True, True, None),
    (17669, 151, False, False, None),
    (24659, 700, True, True, "T4.K3.K2.K2.K2.K2/6/128/0/0/1"),   # split plan, shared a in its evaluation pass
    (57637, 457, True, True, None),
    (100000, 33, True, False, None),                              # beyond one CTA: split plan
    (127, 2049, False, True, None),
    (1, 5, True, True, None),
])
def test_shared_a_matches_oracle_and_unshared_call(n, count, reduce, persistent, spec):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        if spec:
            ctx.set_plan(n, spec)
        a = wl.dense_operands(9500 + n, n, 1, 0)
        b = wl.dense_operands(9500 + n, n, count, 1)
        got = ctx.mul_strided(to_dev(a[0]), to_dev(b), n, reduce, persistent=persistent)
        ref = ctx.mul_strided(to_dev(np.repeat(a, count, axis=0)), to_dev(b), n, reduce, persistent=persistent)
        ctx.sync_status()
        assert torch.equal(got, ref)
        host = got.cpu().numpy().view(np.uint64)
        for p in sorted({0, 1 % count, count // 2, count - 1}):
            exp = oracle.mulmod(a[0], b[p], n) if reduce else oracle.mul(a[0], b[p], n)
            assert np.array_equal(host[p][: len(exp)], exp), p
    finally:
        ctx.close()


def test_shared_public_key_times_sparse_vectors():
    """HQC-128's shape: dense h (n = 17669) times vectors of weight 75."""
    from paper_2201_10473_gb300 import Context
    n, w, count = 17669, 75, 1000
    ctx = Context(0)
    try:
        h = wl.dense_operands(9600, n, 1, 0)[0]
        r = wl.sparse_operands(9600, n, w, count)
        got = ctx.mul_strided(to_dev(h), to_dev(r), n, True, persistent=True).cpu().numpy().view(np.uint64)
        for p in range(0, count, 97):
            assert np.array_equal(got[p], oracle.mulmod(h, r[p], n)), p
    finally:
        ctx.close()


def test_shared_a_may_sit_inside_b_but_not_under_the_results():
    from paper_2201_10473_gb300 import Context, Gf2xError
    n, count = 17669, 64
    L = wl.limbs(n)
    ctx = Context(0)
    try:
        b = to_dev(wl.dense_operands(9700, n, count, 1))
        got = ctx.mul_strided(b[3], b, n, True)    # a is row 3 of b: operands may alias
        row3 = b[3].cpu().numpy().view(np.uint64)
        host = got.cpu().numpy().view(np.uint64)
        for p in (0, 3, count - 1):
            assert np.array_equal(host[p], oracle.mulmod(row3, b[p].cpu().numpy().view(np.uint64), n))
        out = torch.zeros((count, L), dtype=torch.int64, device="cuda")
        with pytest.raises(Gf2xError):
            ctx.mul_strided(out[5], b, n, True, out=out)   # a under the results
    finally:
        ctx.close()
