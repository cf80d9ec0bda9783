"""Persistent launches whose CTAs take the items in order from a device
counter (GF2X_BATCH_DYNAMIC): every product equals the oracle's (Sec. 2.1 and
the reduction of Sec. 1), for device items of mixed sizes sorted largest
first (with padding slots), replayed from a CUDA graph several times (the
counter is zeroed by a captured memset), and for host items."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _ctx():
    from paper_2201_10473_gb300 import Context
    ctx = Context(0, plan_db=None)
    # one leaf size over the prepared sizes (device items need it)
    for n, spec in ((17669, "T2.K3.K2.K2.K2/8"), (35851, "T2.K3.K2.K2.K2.K2/8/0/1"),
                    (57637, "T16.K5.K2.K2.K2.K2/8/0/1")):
        ctx.set_plan(n, spec)
    ctx.prepare([17669, 35851, 57637])
    return ctx


def test_dynamic_device_items_graph_replay():
    from paper_2201_10473_gb300 import pack_items
    ctx = _ctx()
    try:
        sizes = sorted(wl.shuffle(81, [17669] * 300 + [35851] * 120 + [57637] * 60), reverse=True)
        ops = wl.mixed_operands(5400, sizes)
        rows, outs = [], []
        keep = []
        for i, ((a, b), n) in enumerate(zip(ops, sizes)):
            da, db = to_dev(a), to_dev(b)
            o = torch.zeros(wl.limbs(n), dtype=torch.int64, device="cuda")
            keep.append((da, db))
            outs.append(o)
            rows.append((da.data_ptr(), db.data_ptr(), o.data_ptr(), n, 1))
            if i % 97 == 0:
                rows.append((0, 0, 0, 0, 0))                      # padding slot
        items = pack_items(rows).cuda()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            ctx.mul_batched_device(items, len(rows), persistent=True, dynamic=True)   # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.mul_batched_device(items, len(rows), persistent=True, dynamic=True)
        for rep in range(3):                                    # the captured memset re-zeroes the counter
            for o in outs:
                o.zero_()
            g.replay()
            torch.cuda.synchronize()
            ctx.sync_status()
            for k in range(0, len(sizes), 7 if rep else 1):
                (a, b), n = ops[k], sizes[k]
                assert np.array_equal(to_host(outs[k]), oracle.mulmod(a, b, n)), (rep, k, n)
    finally:
        ctx.close()


def test_dynamic_host_items_match_static():
    ctx = _ctx()
    try:
        sizes = wl.shuffle(82, [17669] * 50 + [35851] * 20 + [1000] * 9)
        ops = wl.mixed_operands(5500, sizes)
        dev = [(to_dev(a), to_dev(b)) for a, b in ops]
        o1 = [torch.zeros(wl.limbs(n), dtype=torch.int64, device="cuda") for n in sizes]
        o2 = [torch.zeros(wl.limbs(n), dtype=torch.int64, device="cuda") for n in sizes]
        ctx.mul_batched([(da, db, o, n, True) for (da, db), o, n in zip(dev, o1, sizes)], persistent=True,
                        largest_first=True, dynamic=True)
        ctx.mul_batched([(da, db, o, n, True) for (da, db), o, n in zip(dev, o2, sizes)], persistent=True)
        torch.cuda.synchronize()
        ctx.sync_status()
        for k, ((a, b), n) in enumerate(zip(ops, sizes)):
            assert torch.equal(o1[k], o2[k]), k
            if k % 5 == 0:
                assert np.array_equal(to_host(o1[k]), oracle.mulmod(a, b, n)), (k, n)
    finally:
        ctx.close()
