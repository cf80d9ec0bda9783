"""Pins for the oracle: facts fixed by the mathematics, never by the oracle itself.

Each test is chosen so that a plausible slip in oracle/gf2x_oracle.c (a lost
carry between limbs, a wrong shift direction, an off-by-one in the fold, a
missing mask) fails at least one of them.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

CONFIG_SIZES = [12323, 17669, 24659, 35851, 40973, 57637]


def to_int(limbs_arr) -> int:
    return int.from_bytes(np.ascontiguousarray(limbs_arr, dtype=np.uint64).tobytes(), "little")


def from_int(x: int, nlimbs: int) -> np.ndarray:
    return np.frombuffer(x.to_bytes(8 * nlimbs, "little"), dtype=np.uint64).copy()


def clmul_int(x: int, y: int) -> int:
    """Carry-less product of two Python integers (independent brute force)."""
    r = 0
    i = 0
    while y >> i:
        if (y >> i) & 1:
            r ^= x << i
        i += 1
    return r


def binom_poly(m: int, n: int) -> np.ndarray:
    """(1+X)^m as limbs over ceil(max(n, m+1)/64); by Lucas' theorem the
    coefficient of X^j is 1 exactly when (j & m) == j."""
    L = max(oracle.limbs(n), (m + 64) // 64)
    j = np.arange(m + 1)
    bits = (j & m) == j
    out = np.zeros(L, dtype=np.uint64)
    for pos in np.nonzero(bits)[0]:
        out[pos // 64] |= np.uint64(1 << (int(pos) % 64))
    return out


def fold_int(c: int, n: int) -> int:
    mask = (1 << n) - 1
    return (c & mask) ^ (c >> n)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_exhaustive_all_pairs_vs_numpy_clmul(n):
    """Every operand pair for n <= 10 (2^20 pairs at n=10), batch entry point,
    against a vectorised shift-and-XOR of the bit definition."""
    vals = np.arange(1 << n, dtype=np.uint64)
    A = np.repeat(vals, 1 << n)[:, None]
    B = np.tile(vals, 1 << n)[:, None]
    expect = np.zeros(A.shape[0], dtype=np.uint64)
    for j in range(n):
        sel = (B[:, 0] >> np.uint64(j)) & np.uint64(1)
        expect ^= (A[:, 0] << np.uint64(j)) * sel
    got = oracle.mul_batch(A, B, n, reduce=False)
    assert np.array_equal(got[:, 0], expect)
    mask = np.uint64((1 << n) - 1)
    expect_mod = (expect & mask) ^ (expect >> np.uint64(n))
    got_mod = oracle.mul_batch(A, B, n, reduce=True)
    assert np.array_equal(got_mod[:, 0], expect_mod)


@pytest.mark.parametrize("n", [1, 4, 6])
def test_exhaustive_three_formulations_agree(n):
    for x in range(1 << n):
        for y in range(1 << n):
            a = np.array([x], dtype=np.uint64)
            b = np.array([y], dtype=np.uint64)
            c = clmul_int(x, y)
            assert to_int(oracle.mul(a, b, n)) == c
            assert to_int(oracle.mul_bitwise(a, b, n)) == c
            r = fold_int(c, n)
            assert to_int(oracle.mulmod(a, b, n)) == r
            assert to_int(oracle.mulmod_circulant(a, b, n)) == r


@pytest.mark.parametrize("n", [63, 64, 65, 127, 128, 129, 300, 1000, 2048])
def test_random_vs_bigint_and_bitwise(n):
    a, b = wl.dense_pair(77 + n, n, 3)
    for p in range(3):
        c = clmul_int(to_int(a[p]), to_int(b[p]))
        got = oracle.mul(a[p], b[p], n)
        assert to_int(got) == c
        assert np.array_equal(got, oracle.mul_bitwise(a[p], b[p], n))
        assert to_int(oracle.mulmod(a[p], b[p], n)) == fold_int(c, n)


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 511, 1024, 4096])
def test_mulmod_equals_circulant(n):
    a, b = wl.dense_pair(5 + n, n, 2)
    for p in range(2):
        assert np.array_equal(oracle.mulmod(a[p], b[p], n), oracle.mulmod_circulant(a[p], b[p], n))


# --------------------------------------------------------- closed forms (Lucas)

@pytest.mark.parametrize("n", CONFIG_SIZES)
def test_lucas_binomial_products(n):
    """(1+X)^p (1+X)^q = (1+X)^(p+q) in F2[X]; mod X^n-1 it is the fold."""
    for p, q in [(n - 1, n - 1), (n // 3, n - 1 - n // 3), (12345 % n, 777 % n)]:
        a = binom_poly(p, n)[: oracle.limbs(n)]
        b = binom_poly(q, n)[: oracle.limbs(n)]
        expect = binom_poly(p + q, 2 * n - 1)
        got = oracle.mul(a, b, n)
        assert to_int(got) == to_int(expect)
        assert to_int(oracle.mulmod(a, b, n)) == fold_int(to_int(expect), n)


@pytest.mark.parametrize("n", [17669, 57637])
def test_multiply_by_monomial_is_shift_or_rotation(n):
    a = wl.dense_operands(11, n, 1, 0)[0]
    A = to_int(a)
    for k in [0, 1, 31, 63, 64, 65, n // 2, n - 1]:
        xk = from_int(1 << k, oracle.limbs(n))
        assert to_int(oracle.mul(a, xk, n)) == A << k
        rot = ((A << k) | (A >> (n - k))) & ((1 << n) - 1)
        assert to_int(oracle.mulmod(a, xk, n)) == rot


@pytest.mark.parametrize("n", [12323, 35851])
def test_square_is_bit_interleaving(n):
    a = wl.dense_operands(12, n, 1, 0)[0]
    A = to_int(a)
    spread = 0
    for i in range(n):
        if (A >> i) & 1:
            spread |= 1 << (2 * i)
    assert to_int(oracle.mul(a, a, n)) == spread


@pytest.mark.parametrize("n", [17669, 24659])
def test_times_all_ones_mod_is_parity(n):
    a = wl.dense_operands(13, n, 1, 0)[0]
    ones = wl.mask_top(np.full(oracle.limbs(n), np.uint64(0xFFFFFFFFFFFFFFFF)), n)
    par = bin(to_int(a)).count("1") & 1
    expect = ((1 << n) - 1) if par else 0
    assert to_int(oracle.mulmod(a, ones, n)) == expect


@pytest.mark.parametrize("n", [1, 64, 40973])
def test_multiply_by_one_is_identity(n):
    a = wl.dense_operands(14, n, 1, 0)[0]
    one = from_int(1, oracle.limbs(n))
    got = oracle.mul(a, one, n)
    assert to_int(got) == to_int(a)
    assert np.array_equal(oracle.mulmod(a, one, n), a)


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("n", [17669, 35851])
def test_ring_laws_on_random_data(n):
    a, b = wl.dense_pair(21, n, 1)
    c = wl.dense_operands(22, n, 1, 0)
    a, b, c = a[0], b[0], c[0]
    ab = oracle.mul(a, b, n)
    assert np.array_equal(ab, oracle.mul(b, a, n))                              # commutativity
    assert np.array_equal(oracle.mul(a, b ^ c, n), ab ^ oracle.mul(a, c, n))    # distributivity
    pa, pb, pab = (bin(to_int(x)).count("1") & 1 for x in (a, b, ab))
    assert pab == pa * pb                                                        # evaluation at 1
    assert to_int(ab).bit_length() - 1 == (to_int(a).bit_length() - 1) + (to_int(b).bit_length() - 1)
    # associativity in F2[X]/(X^n-1)
    left = oracle.mulmod(oracle.mulmod(a, b, n), c, n)
    right = oracle.mulmod(a, oracle.mulmod(b, c, n), n)
    assert np.array_equal(left, right)


@pytest.mark.parametrize("n", [100, 12323, 57637])
def test_high_input_bits_are_ignored_and_output_pad_is_zero(n):
    a, b = wl.dense_pair(31, n, 1)
    a, b = a[0], b[0]
    ga, gb = a.copy(), b.copy()
    if n % 64:
        ga[-1] |= np.uint64(~((1 << (n % 64)) - 1) & 0xFFFFFFFFFFFFFFFF)
        gb[-1] |= np.uint64(0xFFFFFFFFFFFFFFFF ^ ((1 << (n % 64)) - 1))
    assert np.array_equal(oracle.mul(a, b, n), oracle.mul(ga, gb, n))
    assert np.array_equal(oracle.mulmod(a, b, n), oracle.mulmod(ga, gb, n))
    full = to_int(oracle.mul(ga, gb, n))
    assert full >> (2 * n - 1) == 0
    assert to_int(oracle.mulmod(ga, gb, n)) >> n == 0


def test_batch_matches_single_calls_and_threads():
    n = 17669
    a, b = wl.dense_pair(41, n, 6)
    for reduce in (False, True):
        got = oracle.mul_batch(a, b, n, reduce=reduce, nthreads=3)
        for p in range(6):
            single = oracle.mulmod(a[p], b[p], n) if reduce else oracle.mul(a[p], b[p], n)
            assert np.array_equal(got[p], single)
