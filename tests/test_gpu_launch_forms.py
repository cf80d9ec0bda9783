"""The two launch forms of gf2x_mul_strided give the same products: one CTA
per product, and the persistent grid whose CTAs take the products in order
from a work counter (Sec. 2.1's product, reduced as in Sec. 1).  Covers
batches that are not a multiple of the grid, a persistent launch captured in
a CUDA graph and replayed with new operands (its counter is a slot of its
own, zeroed by a captured memset), more than 256 persistent launches
alternating between two streams (the counter ring wraps; a slot's next
launch waits for its previous one), and the host-buffer pipeline, whose
chunks run on two compute streams, called back to back."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,count", [(17669, 913), (17669, 1), (4577, 2050), (57637, 457)])
def test_persistent_equals_one_cta_per_product(n, count):
    from paper_2201_10473_gb300 import Context
    ctx = Context(0, batch_hint=max(count, 512))
    try:
        a, b = wl.dense_pair(6100 + n, n, count)
        da, db = to_dev(a), to_dev(b)
        one = to_host(ctx.mul_strided(da, db, n, True, persistent=False))
        pers = to_host(ctx.mul_strided(da, db, n, True, persistent=True))
        ctx.sync_status()
        assert np.array_equal(one, pers), first_diff(pers, one)
        for p in sorted({0, count // 2, count - 1}):
            assert np.array_equal(pers[p], oracle.mulmod(a[p], b[p], n)), p
    finally:
        ctx.close()


def test_persistent_launch_in_a_graph_replayed_with_new_operands():
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 1500
    ctx = Context(0, batch_hint=count)
    try:
        sets = [wl.dense_pair(6200 + k, n, count) for k in range(3)]
        da, db = to_dev(sets[0][0]), to_dev(sets[0][1])
        out = torch.zeros((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            ctx.mul_strided(da, db, n, True, out=out, persistent=True, stream=st)
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            ctx.mul_strided(da, db, n, True, out=out, persistent=True, stream=st)
        for a, b in sets:
            da.copy_(to_dev(a))
            db.copy_(to_dev(b))
            out.zero_()
            torch.cuda.synchronize()
            with torch.cuda.stream(st):
                g.replay()
            st.synchronize()
            got = to_host(out)
            ref = to_host(ctx.mul_strided(da, db, n, True, persistent=False))
            assert np.array_equal(got, ref), first_diff(got, ref)
            assert np.array_equal(got[count - 1], oracle.mulmod(a[count - 1], b[count - 1], n))
        ctx.sync_status()
    finally:
        ctx.close()


def test_counter_ring_wraps_across_two_streams():
    from paper_2201_10473_gb300 import Context
    n, count, launches = 4577, 40, 300
    ctx = Context(0, batch_hint=count)
    try:
        a, b = wl.dense_pair(6300, n, count * launches)
        da, db = to_dev(a), to_dev(b)
        out = torch.zeros((count * launches, wl.limbs(n)), dtype=torch.int64, device="cuda")
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        torch.cuda.synchronize()
        for i in range(launches):
            s = streams[i % 2]
            lo, hi = i * count, (i + 1) * count
            ctx.mul_strided(da[lo:hi], db[lo:hi], n, True, out=out[lo:hi], persistent=True, stream=s)
        torch.cuda.synchronize()
        ctx.sync_status()
        got = to_host(out)
        ref = to_host(ctx.mul_strided(da, db, n, True, persistent=False))
        assert np.array_equal(got, ref), first_diff(got, ref)
        for p in (0, count * launches // 2, count * launches - 1):
            assert np.array_equal(got[p], oracle.mulmod(a[p], b[p], n)), p
    finally:
        ctx.close()


def test_host_pipeline_back_to_back_calls():
    from paper_2201_10473_gb300 import Context
    n, count = 17669, 2600
    ctx = Context(0, batch_hint=count)
    try:
        sets = [wl.dense_pair(6400 + k, n, count) for k in range(3)]
        pins = [(torch.from_numpy(a.view(np.int64)).pin_memory(), torch.from_numpy(b.view(np.int64)).pin_memory())
                for a, b in sets]
        outs = [torch.zeros((count, wl.limbs(n)), dtype=torch.int64).pin_memory() for _ in sets]
        st = torch.cuda.Stream()
        for _ in range(2):
            for (pa, pb), po in zip(pins, outs):
                ctx.mul_strided_host(pa, pb, n, True, out=po, stream=st, inputs_ready=True)
        st.synchronize()
        ctx.sync_status()
        for (a, b), po in zip(sets, outs):
            got = po.numpy().view(np.uint64)
            for p in (0, 1023, 1024, count - 1):
                assert np.array_equal(got[p], oracle.mulmod(a[p], b[p], n)), p
    finally:
        ctx.close()
