"""Host logic of the autotuner, the plan database and the cost model's
bookkeeping, checked on CPU: candidate plans are valid and distinct, the
database survives a write and read, plan choices from a timing log follow
their definitions (checked against brute force), and the random-order
baseline of the cost-model gain test equals the exact expectation over
every order."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2201_10473_gb300 import autotune, costmodel, gf2x


def test_batch_bucket_rounds_up_to_a_power_of_two():
    assert [autotune.batch_bucket(b) for b in (0, 1, 2, 3, 4, 5, 511, 512, 513, 4096, 4097)] == \
        [1, 1, 2, 4, 4, 8, 512, 512, 1024, 4096, 8192]


@pytest.mark.parametrize("n", [12323, 17669, 57637])
def test_candidate_specs_are_valid_distinct_and_within_the_padding_bound(n):
    cands = autotune.candidate_specs(n)
    assert len(cands) > 500
    keys = set()
    for spec in cands:
        info = gf2x.plan_info(n, spec)
        assert n <= 32 * info["top_words"] <= 1.30 * n, spec
        s = gf2x.parse_spec(spec)
        key = (spec.split("/")[0], info["leaf_words"], info["threads"], s.seq_top, s.fuse_leaf, s.split_top)
        assert key not in keys, spec
        keys.add(key)
    split = [c for c in cands if c.endswith("/1")]
    assert (len(split) > 0) == (n >= 24000)


def test_every_database_plan_of_the_six_sizes_is_a_candidate():
    """The tuned entries came out of the candidate space the tuner searches."""
    db = autotune.load_db(gf2x.PACKAGED_PLAN_DB)
    sizes = {12323, 17669, 24659, 35851, 40973, 57637}
    cands = {n: set(autotune.candidate_specs(n)) for n in sizes}
    checked = 0
    for (n, bucket), e in db.items():
        if n in sizes and bucket >= 256:
            assert e["spec"] in cands[n], (n, bucket, e["spec"])
            checked += 1
    assert checked >= 24


def test_plan_database_round_trip(tmp_path):
    db = {(17669, 4096): {"spec": "T1.K2.K2.K2.K2.K2/6/128/1/0/0", "ms": 0.51973, "mults_per_s": 7881052.4},
          (57637, 2048): {"spec": "T16.K2.K2.K2.K2.K2.K2/10/128/0/1/1", "ms": 1.7564, "mults_per_s": 1166011.9},
          (12323, 1): {"spec": "K5.K3.K2.K2.K2/4/768/0/0/1", "ms": 0.0216, "mults_per_s": 46227.8}}
    path = str(tmp_path / "db.txt")
    autotune.save_db(path, db, header="test")
    back = autotune.load_db(path)
    assert set(back) == set(db)
    for k, e in db.items():
        assert back[k]["spec"] == e["spec"]
        assert back[k]["ms"] == pytest.approx(e["ms"], abs=5e-5)
        assert back[k]["mults_per_s"] == pytest.approx(e["mults_per_s"], abs=0.05)
    assert autotune.load_db(str(tmp_path / "missing.txt")) == {}


def _rec(n, batch, spec, ms, threads=128):
    return {"n": n, "batch": batch, "spec": spec, "ms": ms, "threads": threads}


def test_best_plans_take_the_fastest_per_product_at_the_nearest_bucket():
    A, B, C = "K2.K2/4/0/0/0/0", "K3.K2/4/0/0/0/0", "T1.K2.K2/4/0/0/0/1"
    recs = [_rec(100, 512, A, 1.00), _rec(100, 512, B, 0.90), _rec(100, 4096, A, 5.0),
            _rec(100, 2048, C, 0.10), _rec(200, 64, A, 2.0)]
    # at 512 only the 512 records count (2048 is two octaves away)
    assert autotune.best_plans(recs, [100, 200, 300], 512) == {100: B, 200: A}
    # at 2048 the split plan is nearest and fastest; without split plans the
    # nearest record left is the one of 4096 (one octave away; 512 is two)
    assert autotune.best_plans(recs, [100], 2048)[100] == C
    assert autotune.best_plans(recs, [100], 2048, allow_split=False)[100] == A


def test_mixed_plan_sets_match_brute_force():
    """One launch needs one (leaf size, CTA threads) pair: every returned set
    uses one pair, and the sets come in the order of the count-weighted sum
    of each size's fastest time per product under that pair."""
    rng = np.random.default_rng(5)
    weights = {17669: 2048, 35851: 1024, 57637: 512}
    recs = []
    for n in weights:
        for S in (4, 6, 8):
            for t in (128, 256):
                for j in range(3):
                    recs.append(_rec(n, 2048, f"K2.K2.K{j + 2}/{S}/{t}/0/0/0", float(rng.uniform(0.5, 2.0)), t))
    recs.append(_rec(17669, 2048, "T1.K2/4/128/0/0/1", 0.01, 128))    # split: never in a mixed set
    recs.append(_rec(35851, 64, "K2.K2.K2/4/128/0/0/0", 0.001, 128))  # batch far from 2048: ignored
    sets = autotune.mixed_plan_sets(recs, weights, 2048, top=10)
    # brute force over the pairs
    scored = []
    for S, t in itertools.product((4, 6, 8), (128, 256)):
        choice, cost = {}, 0.0
        for n, w in weights.items():
            mine = [r for r in recs if r["n"] == n and r["batch"] == 2048 and r["threads"] == t
                    and r["spec"].split("/")[1] == str(S) and not r["spec"].endswith("/1")]
            best = min(mine, key=lambda r: r["ms"])
            choice[n] = best["spec"]
            cost += w * best["ms"] * 1e6 / best["batch"]
        scored.append((cost, choice))
    scored.sort(key=lambda x: x[0])
    assert sets == [c for _, c in scored]
    for s in sets:
        assert len({(v.split("/")[1], v.split("/")[2]) for v in s.values()}) == 1


def test_random_order_expectation_equals_the_average_over_every_order():
    """E[position of the first good plan] over all orders of N candidates with
    G good ones is (N + 1)/(G + 1): checked by enumerating the orders."""
    cases = [{"a": 1.0, "b": 2.0, "c": 3.0},
             {"a": 1.0, "b": 1.04, "c": 1.2, "d": 1.5, "e": 1.01},
             {"a": 2.0, "b": 2.0, "c": 9.0, "d": 9.0, "e": 9.0, "f": 2.09}]
    for times in cases:
        orders = list(itertools.permutations(times))
        mean = Fraction(sum(costmodel.measurements_to_within(list(o), times) for o in orders), len(orders))
        assert math.isclose(costmodel.random_order_expectation(times), float(mean), rel_tol=1e-12), times
    # the first good plan in a given order, and none before it
    times = {"a": 3.0, "b": 1.0, "c": 1.04, "d": 2.0}
    assert costmodel.measurements_to_within(["d", "a", "c", "b"], times) == 3
    assert costmodel.measurements_to_within(["b", "c"], times) == 1


def test_plan_features_are_deterministic_finite_and_distinguish_plans():
    n, batch = 17669, 4096
    specs = autotune.candidate_specs(n)[:200]
    F = np.stack([costmodel.plan_features(n, batch, s) for s in specs])
    assert F.shape == (len(specs), costmodel.IN_DIM) and np.isfinite(F).all()
    assert np.array_equal(F[0], costmodel.plan_features(n, batch, specs[0]))
    # different plans of one size give different descriptors
    assert len({row.tobytes() for row in F}) == len(specs)
    # the batch enters the descriptor and nothing else changes with it
    G = costmodel.plan_features(n, 2 * batch, specs[0])
    assert G[1] != F[0][1] and np.array_equal(np.delete(G, 1), np.delete(F[0], 1))
