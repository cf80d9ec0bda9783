"""gf2x_mulmod_shared_tc: one polynomial a times many b_j mod X^n - 1 on the
tensor cores (the circulant product of Sec. 1 as a 0/1 GEMM in block-scaled
fp4 with fp32 counts; the product bit is the count's parity).  Every row
must equal the oracle's product, and the shared-operand comb path
(gf2x_mul_strided with GF2X_BATCH_SHARED_A), bit for bit: ragged tiles
(count not a multiple of 128), sizes below one 480-position unit up to the
largest supported, special operands whose products have closed forms,
garbage above n, padded strides, consecutive calls with different a, and a
fixed workspace that splits the batch into groups."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu


def _expect(a, b, n):
    return oracle.mul_batch(np.repeat(a[None], b.shape[0], 0), b, n, reduce=True)


@pytest.mark.parametrize("n,count", [(1, 3), (3, 2), (33, 5), (63, 1), (65, 129), (129, 130), (481, 7),
                                     (1001, 300), (4099, 128), (12323, 257), (17669, 300), (35851, 131)])
def test_matches_oracle_and_the_comb_path(n, count):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        a = wl.dense_operands(5100 + n, n, 1, 0)[0]
        b = wl.dense_operands(5100 + n, n, count, 1)
        got = ctx.mulmod_shared_tc(to_dev(a), to_dev(b), n)
        comb = ctx.mul_strided(to_dev(a), to_dev(b), n, True, persistent=True)
        ctx.sync_status()
        g = to_host(got)
        exp = _expect(a, b, n)
        assert np.array_equal(g, exp), first_diff(g, exp)
        assert torch.equal(got, comb)
    finally:
        ctx.close()


def test_special_operands_closed_forms():
    """a = 1 gives b; a = X^k rotates b by k; a = 1 + X + ... + X^(n-1) gives
    parity(b) in every bit; a zero row of b gives zero."""
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 140
    L = wl.limbs(n)
    ctx = Context(0)
    try:
        b = wl.dense_operands(5201, n, count, 1)
        b[3] = 0
        def bits(x):
            return np.unpackbits(x.view(np.uint8), bitorder="little")[:n]
        def pack(bitrow):
            out = np.zeros(L * 64, np.uint8)
            out[:n] = bitrow
            return np.packbits(out, bitorder="little").view(np.uint64)
        one = np.zeros(L, np.uint64)
        one[0] = 1
        got = to_host(ctx.mulmod_shared_tc(to_dev(one), to_dev(b), n))
        assert np.array_equal(got, b)
        k = 12345
        xk = np.zeros(L, np.uint64)
        xk[k // 64] = np.uint64(1 << (k % 64))
        got = to_host(ctx.mulmod_shared_tc(to_dev(xk), to_dev(b), n))
        for p in (0, 1, 3, count - 1):
            assert np.array_equal(got[p], pack(np.roll(bits(b[p]), k))), p
        ones = pack(np.ones(n, np.uint8))
        got = to_host(ctx.mulmod_shared_tc(to_dev(ones), to_dev(b), n))
        for p in range(count):
            par = int(bits(b[p]).sum() & 1)
            assert np.array_equal(got[p], ones if par else np.zeros(L, np.uint64)), p
        ctx.sync_status()
    finally:
        ctx.close()


def test_high_bits_ignored_padded_strides_and_consecutive_calls():
    from paper_2201_10473_gb300 import Context, gf2x
    n, count = 12323, 200
    L = wl.limbs(n)
    ctx = Context(0)
    try:
        for call in range(2):                               # a different a each call, scratch reused
            a = wl.dense_operands(5300 + call, n, 1, 0)[0]
            b = wl.dense_operands(5300 + call, n, count, 1)
            ag = a.copy()
            ag[-1] |= ~np.uint64((1 << (n % 64)) - 1)       # garbage above n
            bg = np.concatenate([b, np.full((count, 3), np.uint64(0xA5A5A5A5A5A5A5A5))], 1)
            bg[:, L - 1] |= ~np.uint64((1 << (n % 64)) - 1)
            out = torch.full((count, L + 2), -1, dtype=torch.int64, device="cuda")
            da, db = to_dev(ag), to_dev(bg)
            st = gf2x.lib().gf2x_mulmod_shared_tc(ctx._h, out.data_ptr(), da.data_ptr(), db.data_ptr(), n, count,
                                                  L + 3, L + 2, None)
            assert st == 0
            torch.cuda.synchronize()
            host = to_host(out)
            assert np.array_equal(host[:, :L], _expect(a, b, n))
            assert (host[:, L:] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()    # limbs between rows untouched
        ctx.sync_status()
    finally:
        ctx.close()


def test_full_hqc128_batch_equals_the_comb_path():
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 4096
    ctx = Context(0)
    try:
        a = wl.dense_operands(5400, n, 1, 0)[0]
        b = wl.dense_operands(5400, n, count, 1)
        da, db = to_dev(a), to_dev(b)
        got = ctx.mulmod_shared_tc(da, db, n)
        comb = ctx.mul_strided(da, db, n, True, persistent=True)
        ctx.sync_status()
        assert torch.equal(got, comb)
        rows = np.array([0, 127, 128, 2047, 4095])
        assert np.array_equal(to_host(got)[rows], _expect(a, b[rows], n))
    finally:
        ctx.close()


@pytest.mark.parametrize("n,count", [(57637, 130), (65535, 129)])
def test_largest_sizes(n, count):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        a = wl.dense_operands(5500 + n, n, 1, 0)[0]
        b = wl.dense_operands(5500 + n, n, count, 1)
        got = ctx.mulmod_shared_tc(to_dev(a), to_dev(b), n)
        ctx.sync_status()
        rows = np.array([0, 1, 127, 128, count - 1])
        assert np.array_equal(to_host(got)[rows], _expect(a, b[rows], n))
    finally:
        ctx.close()


def test_fixed_workspace_runs_groups_without_allocating():
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 2000
    ctx = Context(0, workspace_bytes=32 << 20)               # 8 MiB of scratch: groups of a few hundred products
    try:
        before = ctx.alloc_count()
        a = wl.dense_operands(5600, n, 1, 0)[0]
        b = wl.dense_operands(5600, n, count, 1)
        got = ctx.mulmod_shared_tc(to_dev(a), to_dev(b), n)
        ctx.sync_status()
        assert ctx.alloc_count() == before
        rows = np.array([0, 255, 256, 511, 512, 1999])
        assert np.array_equal(to_host(got)[rows], _expect(a, b[rows], n))
    finally:
        ctx.close()


def test_rejected_arguments():
    from paper_2201_10473_gb300 import Context, gf2x
    ctx = Context(0)
    try:
        L = wl.limbs(17670)
        x = torch.zeros((4, L), dtype=torch.int64, device="cuda")
        out = torch.zeros((4, L), dtype=torch.int64, device="cuda")
        f = gf2x.lib().gf2x_mulmod_shared_tc
        assert f(ctx._h, out.data_ptr(), x.data_ptr(), x.data_ptr(), 17670, 4, L, L, None) == 5   # even n
        assert f(ctx._h, out.data_ptr(), x.data_ptr(), x.data_ptr(), 65537, 4, L, L, None) == 5   # too large
        assert f(ctx._h, x.data_ptr(), x.data_ptr(), out.data_ptr(), 17669, 4, L, L, None) == 1   # r overlaps a
        assert f(ctx._h, out.data_ptr(), x.data_ptr(), x.data_ptr(), 17669, 4, L - 1, L, None) == 1  # short stride
    finally:
        ctx.close()


def test_captured_in_a_cuda_graph_and_replayed_with_new_vectors():
    """A server with one fixed key captures the call once and replays it
    with new vectors in the same buffers (the scratch is sized by a first
    call outside the capture)."""
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 300
    ctx = Context(0)
    try:
        a = wl.dense_operands(5700, n, 1, 0)[0]
        da = to_dev(a)
        db = to_dev(wl.dense_operands(5700, n, count, 1))
        out = torch.zeros((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            ctx.mulmod_shared_tc(da, db, n, out=out)        # warm-up: scratch and shapes
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):                # the warm-up's stream: no cross-stream scratch wait
            ctx.mulmod_shared_tc(da, db, n, out=out)
        for rep in range(3):
            b = wl.dense_operands(5701 + rep, n, count, 1)
            db.copy_(to_dev(b))
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            ctx.sync_status()
            rows = np.array([0, 127, 128, count - 1])
            assert np.array_equal(to_host(out)[rows], _expect(a, b[rows], n)), rep
    finally:
        ctx.close()
