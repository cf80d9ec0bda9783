"""CPU model of the recursion plans the GPU kernel executes (test infrastructure).

Polynomials are Python integers (bit k = coefficient of X^k); sizes are in
32-bit words as on the GPU.  A plan is a top-down list of levels:

  ("K", k)  k-way Karatsuba split, k(k+1)/2 products (Alg. 1, 2, 3);
  ("T", W)  word-aligned Toom-3 with x = X^w, w = 32*W bits, points
            0, 1, x, x+1, infinity (Appendix D), children padded to the
            common size n' + 2W (Sec. 3.2);

ending in a leaf of S words multiplied by a plain carry-less schoolbook.

This model follows the paper's formulas directly: the Karatsuba
reconstruction is the sum of the pair/single terms of Alg. 1-3 written for
any k, and the division by x+1 is the multiplication by
sum_{i<d/w} X^{wi} mod X^d of Sec. 3.2.  It checks every exactness claim on
the way (low w bits zero before /x, zero remainder after /(x+1)) and counts
word products like the Karatsuba-variants complexity table of Sec. 2.1.  It is NOT the oracle: tests compare
it against oracle/ and the GPU path implements the same algebra in CUDA.
"""
from __future__ import annotations

from dataclasses import dataclass


def clmul(x: int, y: int) -> int:
    r = 0
    i = 0
    while y >> i:
        if (y >> i) & 1:
            r ^= x << i
        i += 1
    return r


def mask_words(words: int) -> int:
    return (1 << (32 * words)) - 1


def sizes(levels, S: int) -> list:
    """Operand size (32-bit words) at every depth: sizes[0] is the top, sizes[-1] = S."""
    out = [S]
    for kind, arg in reversed(levels):
        E = out[0]
        if kind == "K":
            out.insert(0, arg * E)
        elif kind == "T":
            nprime = E - 2 * arg
            if nprime < 1:
                raise ValueError("Toom-3 part size would be < 1 word")
            out.insert(0, 3 * nprime)
        else:
            raise ValueError(kind)
    return out


def karatsuba_children(k: int):
    """Operand selections: singles 0..k-1, then pairs (i, j), i < j, in lexicographic order."""
    return [(i,) for i in range(k)] + [(i, j) for i in range(k) for j in range(i + 1, k)]


def div_by_x_plus_1(P: int, w_bits: int, d_bits: int) -> int:
    """Exact quotient P / (X^w + 1): P * sum_{i < d/w} X^{w i} mod X^d (Sec. 3.2)."""
    assert d_bits % w_bits == 0
    inv = 0
    for i in range(d_bits // w_bits):
        inv |= 1 << (w_bits * i)
    Q = clmul(P, inv) & ((1 << d_bits) - 1)
    assert clmul(Q, (1 << w_bits) | 1) == P, "division by x+1 was not exact"
    return Q


@dataclass
class Counters:
    leaves: int = 0
    clmul64: int = 0


def plan_mul(A: int, B: int, levels, S: int, ctr: Counters | None = None) -> int:
    """Product of A and B (each < 2^(32*sizes[0])) following the plan."""
    sz = sizes(levels, S)
    if A >> (32 * sz[0]) or B >> (32 * sz[0]):
        raise ValueError("operand larger than the plan's top size")
    return _rec(A, B, list(levels), sz, 0, ctr)


def _rec(A, B, levels, sz, depth, ctr):
    if depth == len(levels):
        if ctr is not None:
            ctr.leaves += 1
            ctr.clmul64 += (sz[depth] // 2) ** 2 if sz[depth] % 2 == 0 else 0
        return clmul(A, B)
    kind, arg = levels[depth]
    E = sz[depth + 1]
    if kind == "K":
        k = arg
        m = mask_words(E)
        Ap = [(A >> (32 * E * i)) & m for i in range(k)]
        Bp = [(B >> (32 * E * i)) & m for i in range(k)]
        sel = karatsuba_children(k)
        R = {}
        for s in sel:
            a = 0
            b = 0
            for i in s:
                a ^= Ap[i]
                b ^= Bp[i]
            R[s] = _rec(a, b, levels, sz, depth + 1, ctr)
        C = 0
        for p in range(2 * k - 1):
            term = 0
            for i in range(k):                      # singles i with 0 <= p-i < k
                if 0 <= p - i < k:
                    term ^= R[(i,)]
            for i in range(k):                      # pairs i < j with i + j = p
                j = p - i
                if i < j < k:
                    term ^= R[(i, j)]
            C ^= term << (32 * E * p)
        return C
    # Toom-3, word-aligned, x = X^w
    W = arg
    w = 32 * W
    npr = E - 2 * W
    m = mask_words(npr)
    a0, a1, a2 = ((A >> (32 * npr * i)) & m for i in range(3))
    b0, b1, b2 = ((B >> (32 * npr * i)) & m for i in range(3))
    ev = [
        (a0, b0),                                                       # C(0)
        (a0 ^ a1 ^ a2, b0 ^ b1 ^ b2),                                   # C(1)
        (a0 ^ (a1 << w) ^ (a2 << 2 * w), b0 ^ (b1 << w) ^ (b2 << 2 * w)),   # C(x)
        (a0 ^ a1 ^ a2 ^ (a1 << w) ^ (a2 << 2 * w), b0 ^ b1 ^ b2 ^ (b1 << w) ^ (b2 << 2 * w)),  # C(x+1)
        (a2, b2),                                                       # C(inf)
    ]
    for a, b in ev:
        assert a >> (32 * E) == 0 and b >> (32 * E) == 0
    v0, v1, vx, vx1, vinf = (_rec(a, b, levels, sz, depth + 1, ctr) for a, b in ev)
    c0, c4 = v0, vinf
    d = w * (-(-(64 * E) // w))  # a multiple of w above every degree involved
    s = v0 ^ v1 ^ vx ^ vx1  # = c3 x (x+1)
    assert s & ((1 << w) - 1) == 0, "division by x not exact"
    c3 = div_by_x_plus_1(s >> w, w, d)
    u = vx ^ v0             # = x (c1 + c2 x + c3 x^2 + c4 x^3)
    assert u & ((1 << w) - 1) == 0, "division by x not exact"
    u2 = u >> w
    num = u2 ^ (c3 << 2 * w) ^ (c4 << 3 * w) ^ v1 ^ v0 ^ c3 ^ c4   # = c2 (x+1)
    c2 = div_by_x_plus_1(num, w, d)
    c1 = v1 ^ v0 ^ c3 ^ c4 ^ c2
    for c in (c0, c1, c2, c3, c4):
        assert c >> (32 * 2 * npr) == 0, "interpolated coefficient exceeds 2n' words"
    sh = 32 * npr
    return c0 ^ (c1 << sh) ^ (c2 << 2 * sh) ^ (c3 << 3 * sh) ^ (c4 << 4 * sh)


def parse_levels(text: str):
    """'T2.K3.K2' -> [('T', 2), ('K', 3), ('K', 2)]; '' -> []."""
    out = []
    for tok in filter(None, text.split(".")):
        out.append((tok[0], int(tok[1:])))
    return out


# ---------------------------------------------------------------- operation counts
# A second derivation of the library's modelled operation count (the unit of
# bench.py's roofline): the comb leaf counted from its loop nest, the
# Karatsuba and Toom-3 levels counted node by node down the recursion tree
# (the library multiplies per-level counts by the number of parents).  A
# change of either side's model makes tests/test_plan_ops.py fail.

def comb_ops(S: int) -> int:
    """32-bit operations of the S-word comb leaf, counted loop by loop."""
    ops = 3 * (1 + (S - 1) + 1)              # a X^8, a X^16, a X^24: first shift, S-1 funnel shifts, last shift
    for _u in range(8):                      # eight steps of one bit per byte
        ops += (2 * S - 1) + 1               # accumulator shifted left by one: funnel shifts and the low word
        for _i in range(S):                  # every word of b
            ops += 4                         # four byte-sign masks
            ops += 1                         # b word shifted
            ops += (S + 1) * 3 + S           # AND-XORs of a X^24, a X^16, a X^8 (S+1 words) and a (S words)
    return ops


def karatsuba_node_ops(k: int, E: int) -> int:
    pairs = [c for c in karatsuba_children(k) if len(c) == 2]
    ev = sum(2 * E for _ in pairs)           # A and B pair sums, E words each
    nterms = 0
    for p in range(2 * k - 1):
        nterms += sum(1 for i in range(k) if 0 <= p - i < k)
        nterms += sum(1 for i in range(k) if i < p - i < k)
    return ev + nterms * 2 * E - 2 * (k * E)  # every term XORed in, less the first writes of the 2T words


def toom3_node_ops(W: int, E: int) -> int:
    npr = E - 2 * W
    return 2 * (2 * npr + 4 * E) + 36 * npr  # evaluation of A and B; two /x, two /(x+1), recomposition


def modelled_ops(levels, S: int, n: int) -> int:
    """Modelled operations of one full product of size n under the plan."""
    sz = sizes(levels, S)

    def node(depth):
        if depth == len(levels):
            return comb_ops(S)
        kind, arg = levels[depth]
        E = sz[depth + 1]
        if kind == "K":
            return karatsuba_node_ops(arg, E) + len(karatsuba_children(arg)) * node(depth + 1)
        return toom3_node_ops(arg, E) + 5 * node(depth + 1)
    return node(0) + 4 * ((n + 63) // 64)     # the fold and store: two words per output limb, two operations each
