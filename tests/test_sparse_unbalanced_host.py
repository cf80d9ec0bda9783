"""Host-side checks of the sparse and unbalanced products (no GPU).

* The shape the library picks for the constant-time sparse kernel, for
  every n it accepts: the result registers hold every result word and the
  funnel's neighbour, the register window holds every word a register
  offset can reach, the shared-memory shifts are the in-place-safe ones
  (>= 256 words), the stages cover all bits of the word offset, and the
  shared memory fits a CTA.
* The two identities the kernels are built on, checked with the oracle on
  small random cases: rot(a, p) is the n-bit window at bit n - p of
  a + X^n a; and a b = sum_i (a_i b) X^(i m) for a's m-bit chunks a_i."""
import numpy as np
import pytest

import oracle
import workloads as wl
from paper_2201_10473_gb300 import build as pbuild
from paper_2201_10473_gb300 import gf2x


@pytest.fixture(scope="module", autouse=True)
def built():
    pbuild.build()


def test_sparse_shape_for_every_n():
    for n in range(1, 65537):
        s = gf2x.sparse_info(n)
        N, qmax = (n + 31) // 32, n >> 5
        T = qmax.bit_length()
        C, R, pre = s["words_per_lane"], s["result_words_per_lane"], s["shared_stages"]
        QH = C - R - 1
        assert 32 * R >= N + 1, n                      # result words and the funnel's neighbour word
        assert QH >= 0 and s["register_stages"] == QH.bit_length(), n
        assert s["lane_stages"] == 5, n
        if pre == 0:
            assert (qmax >> 5) <= QH, n                # every whole-register offset stays in the window
        else:
            assert (1 << (T - pre)) == 32 * (QH + 1), n   # the shared stages leave offsets < 32 (QH + 1)
            assert (1 << (T - pre)) >= 256, n          # in-place shared shifts read 256 words ahead
        assert pre + s["register_stages"] + 5 >= T, n  # the stages cover every bit of the word offset
        assert s["smem_bytes"] <= 227 * 1024, n
    for bad in (0, 65537, 1 << 20):
        with pytest.raises(gf2x.Gf2xError):
            gf2x.sparse_info(bad)


def _bits(x: np.ndarray, nbits: int) -> list:
    return [int(x[i // 64] >> np.uint64(i % 64)) & 1 for i in range(nbits)]


def _from_bits(bits, limbs):
    out = np.zeros(limbs, np.uint64)
    for i, v in enumerate(bits):
        if v:
            out[i // 64] |= np.uint64(1 << (i % 64))
    return out


@pytest.mark.parametrize("n", [1, 5, 31, 32, 33, 64, 65, 200, 1000])
def test_rotation_is_a_window_of_the_doubled_vector(n):
    rng = np.random.default_rng(n)
    a = wl.dense_operands(70 + n, n, 1, 0)[0]
    abits = _bits(a, n)
    doubled = abits + abits                            # a + X^n a, 2n bits
    for p in sorted({0, n - 1, *rng.integers(0, n, size=4).tolist()}):
        s = n - p
        window = doubled[s: s + n]
        xp = _from_bits([1 if i == p else 0 for i in range(n)], wl.limbs(n))
        assert np.array_equal(_from_bits(window, wl.limbs(n)), oracle.mulmod(a, xp, n)), p


@pytest.mark.parametrize("na,nb", [(1000, 130), (577, 64), (300, 299), (129, 1)])
def test_one_sided_split_identity(na, nb):
    a = wl.dense_operands(90 + na, na, 1, 0)[0]
    b = wl.dense_operands(90 + nb, nb, 1, 1)[0]
    n = max(na, nb)
    L = wl.limbs(n)
    pad = lambda x: np.concatenate([x, np.zeros(L - len(x), np.uint64)])   # noqa: E731
    full = oracle.mul(pad(a), pad(b), n)
    m = 64 * wl.limbs(nb)
    k = -(-na // m)
    acc = np.zeros(len(full) + 2 * (m // 64), np.uint64)
    Lm = m // 64
    for i in range(k):
        chunk = np.zeros(Lm, np.uint64)
        part = a[i * Lm: (i + 1) * Lm]
        chunk[: len(part)] = part
        bb = np.zeros(Lm, np.uint64)
        bb[: len(b)] = b
        prod = oracle.mul(chunk, bb, m)
        acc[i * Lm: i * Lm + len(prod)] ^= prod
    assert np.array_equal(acc[: len(full)], full)
    assert not acc[len(full):].any()
