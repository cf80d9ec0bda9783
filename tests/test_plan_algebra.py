"""CPU checks of the recursion algebra (Karatsuba k-way, word-aligned Toom-3).

The model in plan_sim.py is pinned to the paper (worked example, printed
sizes, M * M^-1 = I, the counts of the Karatsuba-variants complexity table of Sec. 2.1) and then compared with the
oracle on random operands.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from plan_sim import (Counters, clmul, div_by_x_plus_1, parse_levels, plan_mul, sizes)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def to_int(arr) -> int:
    return int.from_bytes(np.ascontiguousarray(arr, dtype=np.uint64).tobytes(), "little")


def poly(exps) -> int:
    v = 0
    for e in exps:
        v |= 1 << e
    return v


def test_worked_example_division_by_x_plus_1():
    g = json.load(open(os.path.join(GOLDEN, "div_x_plus_1_example.json")))
    P = poly(g["P_exponents"])
    inv = poly(g["inverse_exponents"])
    # the printed inverse really is (X+1)^-1 mod X^8
    assert clmul(inv, 0b11) & ((1 << g["d_bits"]) - 1) == 1
    Q = div_by_x_plus_1(P, g["w_bits"], g["d_bits"])
    assert Q == poly(g["Q_exponents"])


def _rat_mul(p, q):
    return clmul(p, q)


def test_toom3_matrix_times_inverse_is_identity():
    """Appendix D: M and M^-1 over F2(x).  With D = x^2 + x the scaled inverse
    D*M^-1 has polynomial entries; M * (D*M^-1) must equal D*I."""
    x = 0b10
    x1 = 0b11
    one = 1
    M = [
        [one, 0, 0, 0, 0],
        [one, one, one, one, one],
        [one, x, clmul(x, x), clmul(clmul(x, x), x), clmul(clmul(x, x), clmul(x, x))],
        [one, x1, clmul(x, x) ^ 1, clmul(clmul(x, x), x) ^ clmul(x, x) ^ x ^ 1, clmul(clmul(x, x), clmul(x, x)) ^ 1],
        [0, 0, 0, 0, one],
    ]
    D = clmul(x, x) ^ x                  # x^2 + x
    x2x1 = clmul(x, x) ^ x ^ 1           # x^2 + x + 1
    # D times each printed entry of M^-1
    DMinv = [
        [D, 0, 0, 0, 0],
        [x2x1, D, x1, x, clmul(D, D)],   # (x2+x+1)/(x2+x), 1, 1/x, 1/(x+1), x2+x
        [0, 1, x, x1, clmul(D, x2x1)],   # 0, 1/(x2+x), 1/(x+1), 1/x, x2+x+1
        [1, 1, 1, 1, 0],                 # 1/(x2+x) four times, 0
        [0, 0, 0, 0, D],
    ]
    for i in range(5):
        for j in range(5):
            acc = 0
            for t in range(5):
                acc ^= _rat_mul(M[i][t], DMinv[t][j])
            assert acc == (D if i == j else 0), (i, j, acc)


def test_paper_sizes_follow_size_rule():
    g = json.load(open(os.path.join(GOLDEN, "paper_plan_sizes.json")))
    for case in g["cases"]:
        levels = [(t[0], int(t[1:])) for t in case["levels"]]
        top = sizes(levels, case["elem_bits"] // 32)[0]
        assert 32 * top == case["bits"], case


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5])
def test_table_compkarat_clmul_counts(r):
    """The Karatsuba-variants complexity table of Sec. 2.1: KaratRec t^lg3, Karat3 6 (t/3)^lg3, Karat5 15 (t/5)^lg3
    64-bit word products, with 64-bit leaves (S = 2 words of 32 bits)."""
    t = 2 ** r
    for top, expect in ((["K2"] * r, 3 ** r), (["K3"] + ["K2"] * r, 6 * 3 ** r), (["K5"] + ["K2"] * r, 15 * 3 ** r)):
        ctr = Counters()
        levels = parse_levels(".".join(top))
        T = sizes(levels, 2)[0]
        A = (1 << (32 * T)) - 1
        plan_mul(A, A, levels, 2, ctr)
        assert ctr.clmul64 == expect
        assert T // 2 == {2: t, 3: 3 * t, 5: 5 * t}[levels[0][1]]


def test_karatrec_xor_count_formula():
    """Sec. 2.1: KaratRec on t = 2^r words costs 8 t^lg3 - 8 t word XORs; a
    2-way level on t words costs t (operand sums) + 2t (R0+R1+R2) + t (middle
    add) = 4t, and the recurrence X(t) = 3 X(t/2) + 4t gives the formula."""
    def xors(t):
        return 0 if t == 1 else 3 * xors(t // 2) + 4 * t
    for r in range(8):
        t = 2 ** r
        assert xors(t) == 8 * 3 ** r - 8 * t


PLANS = [
    ("K2", 2), ("K3", 2), ("K5", 2), ("K2.K2", 4), ("K3.K2", 2),
    ("T1", 3), ("T2", 6), ("T2.K3", 2), ("T1.K2.K2", 2), ("T2.K2", 8),
    ("K5.K2", 2), ("T1.T1", 3), ("K3.T1", 4), ("T4", 10), ("T3.K2", 4),
]


@pytest.mark.parametrize("levels,S", PLANS)
def test_plan_model_matches_oracle_full_size_operands(levels, S):
    lv = parse_levels(levels)
    T = sizes(lv, S)[0]
    n = 32 * T
    a, b = wl.dense_pair(99 + T, n, 2)
    for p in range(2):
        got = plan_mul(to_int(a[p]), to_int(b[p]), lv, S)
        assert got == to_int(oracle.mul(a[p], b[p], n))


@pytest.mark.parametrize("n,levels,S", [(17669, "T2.K3.K2.K2.K2", 8), (12323, "K3.K2.K2.K2.K2", 10),
                                        (2000, "T1.K2.K2", 6), (777, "K5", 6)])
def test_plan_model_on_padded_sizes(n, levels, S):
    lv = parse_levels(levels)
    assert 32 * sizes(lv, S)[0] >= n
    a, b = wl.dense_pair(7, n, 1)
    got = plan_mul(to_int(a[0]), to_int(b[0]), lv, S)
    assert got == to_int(oracle.mul(a[0], b[0], n))
