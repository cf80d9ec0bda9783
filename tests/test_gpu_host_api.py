"""gf2x_mul_strided_host: operands and results in host memory, chunked copies
overlapped with the products.  Its results must equal gf2x_mul_strided's on
the same data (bit-exact) for every chunking (1, 2 and 4 chunks, ragged last
chunk), full and reduced products, split and in-CTA plans, pinned and
pageable buffers, and calls in a row on different streams."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _host(x: np.ndarray, pinned: bool) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(x).view(np.int64))
    return t.pin_memory() if pinned else t.clone()


@pytest.mark.parametrize("n,count,reduce,spec,pinned", [
    (17669, 4096, True, None, True),                                    # four chunks of 1024
    (17669, 2049, True, None, True),                                    # four chunks, ragged last
    (12323, 300, False, None, True),                                    # one chunk, full product
    (24659, 700, True, "T4.K3.K2.K2.K2.K2/6/128/0/0/1", True),          # split plan, two chunks
    (57637, 513, True, None, False),                                    # pageable buffers
    (35851, 1, True, None, True),
])
def test_host_entry_matches_device_entry(n, count, reduce, spec, pinned):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0, plan_db=None)
    try:
        if spec:
            ctx.set_plan(n, spec)
        a, b = wl.dense_pair(9100 + n + count, n, count)
        ref = ctx.mul_strided(to_dev(a), to_dev(b), n, reduce, persistent=True)
        stream = torch.cuda.Stream()
        ha, hb = _host(a, pinned), _host(b, pinned)     # alive until the copies have run
        got = ctx.mul_strided_host(ha, hb, n, reduce, stream=stream)
        stream.synchronize()
        assert torch.equal(got, ref.cpu())
        for p in (0, count // 2, count - 1):
            exp = oracle.mulmod(a[p], b[p], n) if reduce else oracle.mul(a[p], b[p], n)
            assert np.array_equal(got[p].numpy().view(np.uint64)[: len(exp)], exp)
    finally:
        ctx.close()


@pytest.mark.parametrize("ready", [False, True])
def test_calls_in_a_row_on_two_streams_keep_their_own_results(ready):
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 2500
    ctx = Context(0)
    try:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        ins = [wl.dense_pair(9300 + k, n, count) for k in range(5)]
        hosts = [(_host(a, True), _host(b, True)) for a, b in ins]     # alive until the copies have run
        outs = []
        for k, (ha, hb) in enumerate(hosts):     # no synchronization between the calls
            outs.append(ctx.mul_strided_host(ha, hb, n, True, stream=(s1, s1, s2, s1, s2)[k], inputs_ready=ready))
        s1.synchronize()
        s2.synchronize()
        for (a, b), got in zip(ins, outs):
            ref = ctx.mul_strided(to_dev(a), to_dev(b), n, True, persistent=True).cpu()
            assert torch.equal(got, ref)
    finally:
        ctx.close()


def test_rejects_overlap_and_bad_strides():
    from paper_2201_10473_gb300 import Context, gf2x
    ctx = Context(0, plan_db=None)
    try:
        n = 12323
        a = torch.zeros((4, wl.limbs(n)), dtype=torch.int64)
        b = torch.zeros_like(a)
        with pytest.raises(gf2x.Gf2xError):
            ctx.mul_strided_host(a, b, n, True, out=a)                    # result overlaps an operand
        st = gf2x.lib().gf2x_mul_strided_host(ctx._h, torch.zeros_like(a).data_ptr(), a.data_ptr(), b.data_ptr(),
                                              n, 4, 3, wl.limbs(n), gf2x.REDUCE, None)
        assert st == 1                                                     # GF2X_EINVAL: stride < limbs
    finally:
        ctx.close()


@pytest.mark.parametrize("n,count,stride_pad", [(1, 5, 0), (63, 3, 1), (64, 2049, 0), (131072, 3, 2), (100000, 1, 0)])
def test_edge_sizes_and_padded_strides(n, count, stride_pad):
    """Tiny and maximal n, one product, and host rows with padding limbs."""
    from paper_2201_10473_gb300 import Context
    ctx = Context(0, plan_db=None)
    try:
        L = wl.limbs(n)
        a, b = wl.dense_pair(9500 + n, n, count)
        pa = np.zeros((count, L + stride_pad), np.uint64)
        pb = np.zeros_like(pa)
        pa[:, :L], pb[:, :L] = a, b
        pa[:, L:] = np.uint64(0xDEADBEEFDEADBEEF)          # padding limbs are never read as operand words
        ha, hb = _host(pa, True), _host(pb, True)
        out = torch.full((count, L + 1), -1, dtype=torch.int64).pin_memory()
        stream = torch.cuda.Stream()
        ctx.mul_strided_host(ha, hb, n, True, out=out, stream=stream)
        stream.synchronize()
        ref = ctx.mul_strided(to_dev(a), to_dev(b), n, True).cpu()
        assert torch.equal(out[:, :L], ref)
        assert bool((out[:, L] == -1).all())                 # the column past the result is untouched
        for p in (0, count - 1):
            assert np.array_equal(out[p, :L].numpy().view(np.uint64), oracle.mulmod(a[p], b[p], n))
    finally:
        ctx.close()


def test_zero_count_is_a_no_op():
    from paper_2201_10473_gb300 import Context
    ctx = Context(0, plan_db=None)
    try:
        n = 17669
        e = torch.zeros((0, wl.limbs(n)), dtype=torch.int64)
        got = ctx.mul_strided_host(e, e.clone(), n, True)
        assert got.shape == (0, wl.limbs(n))
    finally:
        ctx.close()
