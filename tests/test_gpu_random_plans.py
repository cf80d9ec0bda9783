"""Seeded random sweep of the plan space: random sizes (1 .. 131072) with
random valid plans (Toom shifts, Karatsuba mixes, leaf sizes, fused leaves,
sequential tops, split tops, CTA sizes), full and reduced products, each
compared limb by limb with the oracle."""
import random

import numpy as np
import pytest

import oracle
import workloads as wl
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu


def _random_cases(count, seed):
    from paper_2201_10473_gb300 import autotune
    rng = random.Random(seed)
    cases = []
    while len(cases) < count:
        n = rng.choice([rng.randint(1, 4096), rng.randint(4097, 40000), rng.randint(40001, 131072)])
        cands = autotune.candidate_specs(n, max_waste=1.6, threads=(0, 128, 256, 512), split_from=1)
        if cands:
            cases.append((n, rng.choice(cands)))
    return cases


@pytest.mark.parametrize("seed", [2201, 10473])
def test_random_plans_against_oracle(seed):
    from paper_2201_10473_gb300 import Context
    failures = []
    ctx = Context(0, plan_db=None)
    try:
        for n, spec in _random_cases(20, seed):
            ctx.set_plan(n, spec)
            a, b = wl.dense_pair(seed + n, n, 3)
            for reduce in (True, False):
                got = to_host(ctx.mul_strided(to_dev(a), to_dev(b), n, reduce, persistent=True))
                exp = oracle.mul_batch(a, b, n, reduce=reduce)
                if not np.array_equal(got, exp):
                    failures.append(f"n={n} spec={spec} reduce={reduce}: {first_diff(got, exp)}")
            ctx.set_plan(n, None)
        ctx.sync_status()
    finally:
        ctx.close()
    assert not failures, "\n".join(failures)
