"""Operands of different sizes (gf2x_mul_unbalanced): every result row equals
the oracle's full product of the zero-extended operands, limb for limb, and
the oracle's limbs past ceil((na + nb - 1)/64) are zero (the result is
complete).  Covers the chunked form (b much shorter than a), the padded form
(sizes close), swapped roles, equal sizes, one-limb and one-bit operands,
ragged sizes, batches larger than one scratch group, padded strides and
garbage above the operands' sizes."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _expect(a: np.ndarray, na: int, b: np.ndarray, nb: int) -> np.ndarray:
    n = max(na, nb)
    L = wl.limbs(n)
    pa = np.zeros(L, np.uint64)
    pb = np.zeros(L, np.uint64)
    pa[: wl.limbs(na)] = wl.mask_top(a[: wl.limbs(na)].copy(), na)
    pb[: wl.limbs(nb)] = wl.mask_top(b[: wl.limbs(nb)].copy(), nb)
    full = oracle.mul(pa, pb, n)
    lu = (na + nb - 1 + 63) // 64
    assert not full[lu:].any()
    return full[:lu]


def _rows(seed: int, n: int, count: int, operand: int, width: int = 0, garbage: bool = False) -> np.ndarray:
    x = wl.dense_operands(seed, n, count, operand)
    if garbage and n % 64:   # set the bits above n: the call must ignore them
        x[:, -1] |= ~np.uint64((1 << (n % 64)) - 1)
    if width > x.shape[1]:
        x = np.concatenate([x, np.full((count, width - x.shape[1]), np.uint64(0xA5A5A5A5A5A5A5A5))], axis=1)
    return x


@pytest.mark.parametrize("na,nb,count", [
    (17669, 131, 3),        # chunked: 93 chunks of 192 bits
    (57637, 17669, 5),      # four 17728-bit chunks or one padded product
    (24659, 17669, 7),
    (17669, 57637, 4),      # roles swapped
    (40973, 40973, 3),      # equal sizes
    (1, 100000, 2),         # one-bit operand
    (64, 65, 9),
    (63, 1, 1),
    (131072, 2049, 2),
    (12323, 12289, 33),
])
def test_matches_oracle(na, nb, count):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        a = _rows(9800 + na, na, count, 0, garbage=True)
        b = _rows(9800 + nb, nb, count, 1, garbage=True)
        got = to_host(ctx.mul_unbalanced(to_dev(a), na, to_dev(b), nb))
        ctx.sync_status()
        for p in range(count):
            assert np.array_equal(got[p], _expect(a[p], na, b[p], nb)), p
    finally:
        ctx.close()


def test_equal_sizes_match_the_equal_size_call():
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 300
    ctx = Context(0)
    try:
        a, b = wl.dense_pair(9900, n, count)
        got = ctx.mul_unbalanced(to_dev(a), n, to_dev(b), n)
        ref = ctx.mul_strided(to_dev(a), to_dev(b), n, False, persistent=True)
        assert torch.equal(got, ref)
    finally:
        ctx.close()


def test_padded_strides_and_single_rows():
    from paper_2201_10473_gb300 import Context
    na, nb, count = 35851, 4099, 6
    ctx = Context(0)
    try:
        a = _rows(9901, na, count, 0, width=wl.limbs(na) + 3)
        b = _rows(9902, nb, count, 1, width=wl.limbs(nb) + 5)
        lu = (na + nb - 1 + 63) // 64
        out = torch.full((count, lu + 2), -1, dtype=torch.int64, device="cuda")
        ctx.mul_unbalanced(to_dev(a), na, to_dev(b), nb, out=out)
        host = to_host(out)
        for p in range(count):
            assert np.array_equal(host[p, :lu], _expect(a[p], na, b[p], nb)), p
        assert (host[:, lu:] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()     # limbs between rows untouched
        one = to_host(ctx.mul_unbalanced(to_dev(a[2]), na, to_dev(b[2]), nb))
        assert np.array_equal(one, _expect(a[2], na, b[2], nb))
    finally:
        ctx.close()


def test_batch_larger_than_one_scratch_group():
    """131072 x 131072 needs 64 KiB of scratch per product: 4100 products
    run as two groups of the 256 MiB scratch."""
    from paper_2201_10473_gb300 import Context
    n, count = 131072, 4100
    ctx = Context(0)
    try:
        a, b = wl.dense_pair(9903, n, count)
        got = to_host(ctx.mul_unbalanced(to_dev(a), n, to_dev(b), n - 1))
        for p in (0, 4095, 4096, count - 1):
            assert np.array_equal(got[p], _expect(a[p], n, b[p], n - 1)), p
    finally:
        ctx.close()


def test_calls_on_two_streams_share_the_scratch_safely():
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        cases = [(57637, 1000, 64, s1), (24659, 3000, 64, s2), (57637, 1000, 64, s1), (17669, 700, 64, s2)]
        outs = []
        for k, (na, nb, count, st) in enumerate(cases):
            a = _rows(9910 + k, na, count, 0)
            b = _rows(9910 + k, nb, count, 1)
            with torch.cuda.stream(st):
                da, db = to_dev(a), to_dev(b)
                outs.append((a, b, ctx.mul_unbalanced(da, na, db, nb, stream=st), da, db))
        torch.cuda.synchronize()
        for (na, nb, count, _), (a, b, got, _, _) in zip(cases, outs):
            host = to_host(got)
            for p in (0, count - 1):
                assert np.array_equal(host[p], _expect(a[p], na, b[p], nb))
    finally:
        ctx.close()


def test_rejections():
    from paper_2201_10473_gb300 import Context, gf2x
    ctx = Context(0)
    try:
        # three separate (4, 64)-limb buffers: rows 64 limbs apart, every
        # accepted call stays inside them (a 16 limbs, b 4, result 19 a row)
        bufs = [torch.zeros((4, 64), dtype=torch.int64, device="cuda") for _ in range(3)]
        a, b, out = (t.data_ptr() for t in bufs)

        def call(out, na, nb, sa=64, sb=64, so=64, count=4):
            return gf2x.lib().gf2x_mul_unbalanced(ctx._h, out, a, na, sa, b, nb, sb, count, so, None)
        assert call(out, 1000, 200) == 0
        assert call(out, 1000, 0) == 5 and call(out, 131073, 200) == 5         # GF2X_EUNSUPPORTED
        assert call(out, 1000, 200, sa=10) == 1                                 # stride below ceil(na/64)
        assert call(out, 1000, 200, so=18) == 1                                 # stride below the result size
        assert call(a, 1000, 200) == 1                                          # result over a's rows
        assert call(b + 8, 1000, 200) == 1                                      # result over b's rows
        assert call(out + 4, 1000, 200) == 1                                    # misaligned
        assert call(out, 1000, 200, count=0) == 0
        torch.cuda.synchronize()
    finally:
        ctx.close()
