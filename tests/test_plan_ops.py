"""The modelled operation count that bench.py's roofline divides by (the
library's gf2x_plan_info.ops_full) against a second derivation in
tests/plan_sim.py, for the benchmark plans and a spread of others, and the
leaf products' useful AND-XOR count against the word products of Table
the Karatsuba-variants complexity table of Sec. 2.1 (clmul64 x 64 x 64 bit products / 32 per 32-bit operation)."""
import pytest

from paper_2201_10473_gb300 import autotune, gf2x
from plan_sim import comb_ops, modelled_ops, parse_levels


def _levels_and_leaf(n, spec):
    info = gf2x.plan_info(n, spec)
    return parse_levels(spec.split("/")[0]), info["leaf_words"], info


def test_comb_loop_count_matches_the_closed_form():
    for S in (4, 6, 8, 10, 12, 16):
        assert comb_ops(S) == 32 * S * S + 83 * S + 3


def test_benchmark_plans_and_others():
    db = autotune.load_db(gf2x.PACKAGED_PLAN_DB)
    specs = {(n, v["spec"]) for (n, _bucket), v in db.items() if not gf2x.parse_spec(v["spec"]).split_top}
    specs |= {(17669, "T2.K2.K2.K2.K2.K2/6/128/1/0/0"), (12323, "T4.K3.K2.K2.K2/6/0/0/1/0"),
              (57637, "T16.K2.K2.K2.K2.K2.K2/10/0/1/1/0"), (24659, "K5.K2.K2.K2.K2/10/0/0/1/0"),
              (1000, "K2.K2/8"), (4096, "K3.K5.K2/8")}
    assert (17669, db[(17669, 2048)]["spec"]) in specs          # the C2 bench plan
    checked = 0
    for n, spec in sorted(specs):
        levels, S, info = _levels_and_leaf(n, spec)
        assert info["ops_full"] == modelled_ops(levels, S, n), (n, spec)
        assert info["ops_leaf"] == info["nleaves"] * comb_ops(S), (n, spec)
        checked += 1
    assert checked >= 8


@pytest.mark.parametrize("n,spec", [(17669, "T2.K2.K2.K2.K2.K2/6/128/1/0/0"), (57637, "T16.K2.K2.K2.K2.K2.K2/10/0/1/1/0"),
                                    (12323, "T4.K3.K2.K2.K2/6/0/0/1/0")])
def test_useful_leaf_operations_are_the_word_products(n, spec):
    _, S, info = _levels_and_leaf(n, spec)
    useful = info["nleaves"] * 32 * S * S                       # one AND-XOR per 32 bit products
    assert useful == info["clmul64"] * 64 * 64 // 32
    assert useful < info["ops_leaf"] < info["ops_full"]
