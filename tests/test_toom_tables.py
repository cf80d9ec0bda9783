"""The Toom-4 / Toom-5 interpolation tables (no GPU).

* The tables compiled into toom.cu are exactly what gen_toom_tables.py
  derives (sympy, Vandermonde system over F2(x)).
* Independently of that script, the tables invert the evaluation: for every
  coefficient k and power i, sum_j P_kj(x) p_j^i / D_k(x) is 1 if i = k and
  0 otherwise, over F2(x).
* A word-level model of the top level built from the compiled tables (the
  child products by the oracle) gives the oracle's full product."""
import os
import re
import sys

import numpy as np
import pytest

import oracle
import workloads as wl

sp = pytest.importorskip("sympy")
CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2201_10473_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_toom_tables as gen  # noqa: E402

X = sp.symbols("x")


def _sets(text):
    """[[n, [e...]], ...] from a C initializer of {n, {e, ...}} pairs."""
    return [(int(n), [int(v) for v in body.split(",")]) for n, body in re.findall(r"\{(\d+), \{([\d, ]+)\}\}", text)]


def compiled_tables(K):
    src = open(os.path.join(CSRC, "toom.cu")).read()
    pow_txt = re.search(rf"kPow{K}\[\d+\]\[\d+\] = \{{(.*?)\n\}};", src, re.S).group(1)
    top_txt = re.search(rf"kTop{K}\[\d+\] = \{{(.*?)\}};", src, re.S).group(1)
    int_txt = re.search(rf"kInterp{K}\[\d+\] = \{{(.*?)\n\}};", src, re.S).group(1)
    flat = [e[:n] for n, e in _sets(pow_txt)]
    pow_rows = [flat[i * K:(i + 1) * K] for i in range(2 * K - 1)]
    top = [e[:n] for n, e in _sets(top_txt + "}")]
    interp = []
    for line in int_txt.strip().splitlines():
        nums = [int(v) for v in re.findall(r"\d+", line)]
        a, b, c = nums[:3]
        nf = 2 * K - 3
        counts = nums[3:3 + nf]
        rest = nums[3 + nf:]
        terms = []
        for cnt in counts:
            take = max(cnt, 1)          # an empty list is printed as {0}
            terms.append(rest[:cnt])
            rest = rest[take:]
        interp.append((a, b, c, terms))
    return pow_rows, top, interp


@pytest.mark.parametrize("K", [4, 5])
def test_compiled_tables_are_the_derived_ones(K):
    assert compiled_tables(K) == tuple(gen.tables(K))


def _poly(exps):
    return sum((X**e for e in exps), sp.Integer(0))


@pytest.mark.parametrize("K", [4, 5])
def test_tables_invert_the_evaluation(K):
    pts = gen.POINTS[K]
    _, _, interp = compiled_tables(K)
    nf = 2 * K - 3
    for k, (a, b, c, terms) in enumerate(interp):
        D = sp.Poly(X**a * (X + 1)**b * (X**2 + X + 1)**c, X, modulus=2)
        for i in range(1, nf + 1):
            num = sp.Poly(sum((_poly(terms[j]) * pts[j]**i for j in range(nf)), sp.Integer(0)), X, modulus=2)
            want = D if i == k + 1 else sp.Poly(0, X, modulus=2)
            assert num == want, (K, k, i)


def _model(a, b, n, K):
    """The top level in 32-bit words: evaluation, child products (oracle),
    interpolation with the compiled tables, recomposition."""
    pow_rows, top, interp = compiled_tables(K)
    L32 = (n + 31) // 32
    m = -(-L32 // K)
    e = m + 2 * (K - 1)
    E = e + (e & 1)
    W = 2 * E + 8 * (K - 2)

    def words(v, cnt):
        return [(v >> (32 * i)) & 0xFFFFFFFF for i in range(cnt)]

    def value(ws):
        return sum(int(w) << (32 * i) for i, w in enumerate(ws))

    ai = sum(int(x) << (64 * i) for i, x in enumerate(a))
    bi = sum(int(x) << (64 * i) for i, x in enumerate(b))
    parts = [[words(v >> (32 * m * i), m) for i in range(K)] for v in (ai, bi)]

    def evaluate(P, sets):
        out = [0] * E
        for i in range(K):
            for s in sets[i]:
                for t in range(m):
                    out[t + s] ^= P[i][t]
        return out

    R = []
    for sets in pow_rows:
        ea, eb = evaluate(parts[0], sets), evaluate(parts[1], sets)
        la = np.array([value(ea[2 * q: 2 * q + 2]) for q in range(E // 2)], np.uint64)
        lb = np.array([value(eb[2 * q: 2 * q + 2]) for q in range(E // 2)], np.uint64)
        r = oracle.mul(la, lb, 32 * E)
        R.append(words(sum(int(x) << (64 * i) for i, x in enumerate(r)), W))
    C0, CT = R[0], R[-1]
    S = []
    for j in range(2 * K - 3):
        s = [R[j + 1][t] ^ C0[t] for t in range(W)]
        for sh in top[j]:
            for t in range(W - sh):
                s[t + sh] ^= CT[t]
        S.append(s)
    total = value(C0) ^ (value(CT) << (32 * m * (2 * K - 2)))
    for k, (a_, b_, c_, terms) in enumerate(interp):
        num = [0] * (W + 8)
        for j, ts in enumerate(terms):
            for sh in ts:
                for t in range(W):
                    num[t + sh] ^= S[j][t]
        assert not any(num[:a_])
        num = num[a_:]
        for _ in range(b_):
            for t in range(1, len(num)):
                num[t] ^= num[t - 1]
        for _ in range(c_):
            num = [num[t] ^ (num[t - 1] if t else 0) for t in range(len(num))]
            for t in range(3, len(num)):
                num[t] ^= num[t - 3]
        total ^= value(num) << (32 * m * (k + 1))
    return total


@pytest.mark.parametrize("K", [4, 5])
@pytest.mark.parametrize("n", [1, 33, 129, 500, 2049])
def test_model_from_compiled_tables_matches_oracle(K, n):
    a, b = wl.dense_pair(77 + n, n, 1)
    full = oracle.mul(a[0], b[0], n)
    assert _model(a[0], b[0], n, K) == sum(int(x) << (64 * i) for i, x in enumerate(full))
