"""Constant-time sparse x dense products mod X^n - 1 (gf2x_mulmod_sparse):
every row equals the oracle's product of a and the dense form of the
position list (repeated positions cancel), and the dense path's product of
the same operands, bit for bit.  Covers every kernel shape (2 to 65 result
registers per lane, 0 to 4 shared stages), positions 0 and n - 1, w = 0,
ragged batches, padded strides,
garbage above n, rejections, and launch times independent of the positions."""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _dense(pos: np.ndarray, n: int) -> np.ndarray:
    b = np.zeros(wl.limbs(n), np.uint64)
    for p in pos:
        b[int(p) // 64] ^= np.uint64(1 << (int(p) % 64))
    return b


def _positions(seed: int, n: int, w: int, count: int) -> np.ndarray:
    """Distinct positions per row (HQC's fixed-weight vectors), from the
    seeded sparse operands of the workload module."""
    rows = wl.sparse_operands(seed, n, w, count)
    out = np.zeros((count, w), np.int32)
    for p in range(count):
        bits = np.unpackbits(rows[p].view(np.uint8), bitorder="little")
        out[p] = np.flatnonzero(bits)[:w]
    return out


@pytest.mark.parametrize("n,w,count", [
    (17669, 75, 37),      # HQC-128 shape: 18 result registers per lane, no shared stage
    (35851, 114, 9),      # 36 result registers, six register stages
    (57637, 131, 5),      # 57 result registers, two shared stages
    (65536, 16, 3),       # four shared stages, largest n
    (60000, 50, 3),       # 65 result registers, three shared stages
    (40973, 137, 5),      # 46 result registers, two shared stages (BIKE-5 size)
    (24659, 103, 9),      # 26 result registers (BIKE-3 size)
    (12323, 71, 17),      # 13 result registers (BIKE-1 size)
    (8673, 40, 33),       # 9 result registers
    (4577, 20, 65),       # 5 result registers
    (2017, 9, 5), (2016, 8, 5),   # the two sides of the smallest shape's limit
    (100, 7, 3), (33, 5, 2), (32, 3, 2), (31, 4, 2), (1, 1, 2),
])
def test_matches_oracle_and_dense_path(n, w, count):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        a = wl.dense_operands(9950 + n, n, count, 0)
        pos = _positions(9950 + n, n, w, count)
        pos[0, 0], pos[-1, -1] = 0, n - 1           # the two end positions
        a_g = a.copy()
        if n % 64:                                   # bits above n must be ignored
            a_g[:, -1] |= ~np.uint64((1 << (n % 64)) - 1)
        got = to_host(ctx.mulmod_sparse(to_dev(a_g), torch.from_numpy(pos).cuda(), n))
        dense_b = np.stack([_dense(pos[p], n) for p in range(count)])
        via_dense = to_host(ctx.mul_strided(to_dev(a), to_dev(dense_b), n, True, persistent=True))
        assert np.array_equal(got, via_dense)
        for p in sorted({0, count // 2, count - 1}):
            assert np.array_equal(got[p], oracle.mulmod(a[p], dense_b[p], n)), p
    finally:
        ctx.close()


def test_repeated_positions_cancel_and_empty_lists():
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 4
    ctx = Context(0)
    try:
        a = wl.dense_operands(9960, n, count, 0)
        pos = np.array([[5, 5, 700, 17668]] * count, np.int32)   # 5 twice: cancels
        got = to_host(ctx.mulmod_sparse(to_dev(a), torch.from_numpy(pos).cuda(), n))
        for p in range(count):
            assert np.array_equal(got[p], oracle.mulmod(a[p], _dense([700, 17668], n), n))
        empty = torch.zeros((count, 0), dtype=torch.int32, device="cuda")
        assert not ctx.mulmod_sparse(to_dev(a), empty, n).any()
    finally:
        ctx.close()


def test_padded_strides():
    from paper_2201_10473_gb300 import Context, gf2x
    n, w, count = 57637, 131, 4
    L = wl.limbs(n)
    ctx = Context(0)
    try:
        a = to_dev(np.concatenate([wl.dense_operands(9970, n, count, 0),
                                   np.full((count, 3), np.uint64(0x5A5A5A5A5A5A5A5A))], axis=1))
        pos_np = _positions(9970, n, w, count)
        pos = torch.from_numpy(np.concatenate([pos_np, np.full((count, 5), -7, np.int32)], axis=1)).cuda()
        out = torch.full((count, L + 2), -1, dtype=torch.int64, device="cuda")
        st = gf2x.lib().gf2x_mulmod_sparse(ctx._h, out.data_ptr(), a.data_ptr(), pos.data_ptr(), w, n, count,
                                           L + 3, w + 5, L + 2, None)
        assert st == 0
        torch.cuda.synchronize()
        host, ah = to_host(out), to_host(a)
        for p in range(count):
            assert np.array_equal(host[p, :L], oracle.mulmod(ah[p, :L], _dense(pos_np[p], n), n)), p
        assert (host[:, L:] == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    finally:
        ctx.close()


def test_rejections():
    from paper_2201_10473_gb300 import Context, gf2x
    ctx = Context(0)
    try:
        # separate buffers; every accepted call stays inside them
        a = torch.zeros((4, 64), dtype=torch.int64, device="cuda")
        pos = torch.zeros((4, 16), dtype=torch.int32, device="cuda")
        out = torch.zeros((4, 64), dtype=torch.int64, device="cuda")

        def call(r, n, w=16, sa=64, sp=16, sr=64, count=4, p=None):
            return gf2x.lib().gf2x_mulmod_sparse(ctx._h, r, a.data_ptr(), pos.data_ptr() if p is None else p, w, n,
                                                 count, sa, sp, sr, None)
        assert call(out.data_ptr(), 4000) == 0
        assert call(out.data_ptr(), 0) == 5 and call(out.data_ptr(), 65537) == 5
        assert call(out.data_ptr(), 4000, sa=10) == 1 and call(out.data_ptr(), 4000, sp=15) == 1
        assert call(a.data_ptr(), 4000) == 1                              # result over a
        assert call(pos.data_ptr(), 4000) == 1                            # result over the positions
        assert call(out.data_ptr() + 4, 4000) == 1                        # misaligned result
        assert call(out.data_ptr(), 4000, p=pos.data_ptr() + 2) == 1      # misaligned positions
        assert call(out.data_ptr(), 4000, count=0) == 0
        torch.cuda.synchronize()
    finally:
        ctx.close()


def _median_ms(fn, reps=5, inner=10):
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(inner):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / inner)
    return float(np.median(times))


@pytest.mark.parametrize("n,w", [(17669, 75), (57637, 131)])
def test_launch_time_independent_of_positions(n, w):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0)
    try:
        count = 1216          # 2 x 152 SMs x 4 warps
        a = to_dev(wl.dense_operands(9980, n, count, 0))
        classes = {
            "random": _positions(9980, n, w, count),
            "zeros": np.zeros((count, w), np.int32),
            "last": np.full((count, w), n - 1, np.int32),
            "run": np.tile(np.arange(w, dtype=np.int32), (count, 1)),
        }
        dev = {k: torch.from_numpy(v).cuda() for k, v in classes.items()}
        out = torch.empty((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
        t_end = time.time() + 1.0            # clock ramp-up first
        while time.time() < t_end:
            ctx.mulmod_sparse(a, dev["random"], n, out=out)
            torch.cuda.synchronize()
        rounds = {k: [] for k in dev}
        for _ in range(3):
            for k, p in dev.items():
                rounds[k].append(_median_ms(lambda: ctx.mulmod_sparse(a, p, n, out=out)))
        ms = {k: min(v) for k, v in rounds.items()}
        assert max(ms.values()) / min(ms.values()) < 1.05, ms
    finally:
        ctx.close()
