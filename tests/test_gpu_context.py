"""Context plan control: a rejected plan leaves the current one in force."""
import pytest
import torch

import workloads as wl
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def test_rejected_plan_keeps_the_current_one():
    from paper_2201_10473_gb300 import Context, gf2x
    n = 17669
    ctx = Context(0, plan_db=None)
    try:
        good = "T2.K2.K2.K2.K2.K2/6/128/1/0/0"
        ctx.set_plan(n, good)
        with pytest.raises(gf2x.Gf2xError):
            ctx.set_plan(n, "K2/8")                      # does not cover n
        assert ctx.get_plan(n) == good
        a, b = wl.dense_pair(71, n, 8)
        r = ctx.mul_strided(to_dev(a), to_dev(b), n, True)   # still runs, with the kept plan
        ctx.set_plan(n, "T1.K2.K2.K2.K2.K2/6/0/0/0/0")
        assert torch.equal(r, ctx.mul_strided(to_dev(a), to_dev(b), n, True))
    finally:
        ctx.close()


def test_single_product_plans_from_the_database():
    """batch_hint=1 selects the database's single-product (batch 1) plans --
    split plans, three launches over 15 CTAs -- and they give the oracle's
    product."""
    import numpy as np

    import oracle
    from paper_2201_10473_gb300 import Context, autotune, gf2x
    db = autotune.load_db(gf2x.PACKAGED_PLAN_DB)
    ctx = Context(0, batch_hint=1)
    try:
        for n in (12323, 57637):
            assert ctx.get_plan(n) == db[(n, 1)]["spec"]
            a, b = wl.dense_pair(73 + n, n, 1)
            r = ctx.mulmod(to_dev(a)[0], to_dev(b)[0], n)
            assert np.array_equal(r.cpu().numpy().view(np.uint64), oracle.mulmod(a[0], b[0], n))
    finally:
        ctx.close()
