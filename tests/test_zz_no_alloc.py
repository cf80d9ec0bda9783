"""gf2x_mul_strided_static: the entry point for callers that cannot allocate
device memory (a framework that owns every device allocation, a service with
a budget fixed at start-up, code that must not let cudaMalloc synchronize the
device).  Call after call it must give exactly what gf2x_mul_strided gives
with the same split plan, and the oracle's products, although its scratch is
one shared file-scope device array.  Collected last (file name) so that a run
stopping at the first failure has already run every other test; it passes
alone in a fresh process too."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import first_diff, to_dev, to_host

pytestmark = pytest.mark.gpu

GF2X_EUNSUPPORTED = 5
STATIC_SCRATCH_BYTES = 4 << 20


def _static_entry():
    from paper_2201_10473_gb300 import gf2x
    fn = gf2x.lib().gf2x_mul_strided_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_size_t,
                   ctypes.c_size_t, ctypes.c_size_t, ctypes.c_uint32, ctypes.POINTER(gf2x.PlanSpec), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("n,spec,count,reduce", [
    (57637, "T16.K2.K2.K2.K2.K2.K2/10/0/0/1/1", 96, True),
    (17669, "T2.K2.K2.K2.K2.K2/6/128/1/0/1", 200, True),
    (12323, "T4.K3.K2.K2.K2/6/0/0/1/1", 100, False),
    (131072, None, 40, True),
])
def test_static_entry_matches_strided_entry_twice(n, spec, count, reduce):
    from paper_2201_10473_gb300 import Context, gf2x
    fn = _static_entry()
    ctx = Context(0, plan_db=None)
    try:
        ps = gf2x.parse_spec(spec) if spec else None
        if spec:
            ctx.set_plan(n, spec)      # the same split plan for the reference call
        L = wl.limbs(n)
        ol = L if reduce else wl.limbs(2 * n - 1)
        stream = torch.cuda.current_stream()
        for call in range(2):                         # two calls in a row share the scratch array
            a, b = wl.dense_pair(8000 + n + call, n, count)
            da, db = to_dev(a), to_dev(b)
            ref = ctx.mul_strided(da, db, n, reduce)  # the existing entry point
            got = torch.full((count, ol), -1, dtype=torch.int64, device="cuda")
            st = fn(got.data_ptr(), da.data_ptr(), db.data_ptr(), n, count, L, ol, 1 if reduce else 0,
                    ctypes.byref(ps) if ps is not None else None, ctypes.c_void_p(stream.cuda_stream))
            assert st == 0, st
            torch.cuda.synchronize()
            assert torch.equal(got, ref), (n, call)   # bit-exact, as every other parity test
            exp = oracle.mul_batch(a, b, n, reduce=reduce)
            g = to_host(got)
            assert np.array_equal(g, exp), (n, call, first_diff(g, exp))
    finally:
        ctx.close()


def test_static_entry_rejects_a_batch_beyond_its_scratch():
    from paper_2201_10473_gb300 import gf2x
    fn = _static_entry()
    n, spec = 57637, "T16.K2.K2.K2.K2.K2.K2/10/0/0/1/1"
    per = gf2x.plan_info(n, spec)["scratch_bytes"]
    count = STATIC_SCRATCH_BYTES // per + 1
    L = wl.limbs(n)
    a = torch.zeros((count, L), dtype=torch.int64, device="cuda")
    b = torch.zeros_like(a)
    out = torch.zeros_like(a)
    ps = gf2x.parse_spec(spec)
    st = fn(out.data_ptr(), a.data_ptr(), b.data_ptr(), n, count, L, L, 1, ctypes.byref(ps),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == GF2X_EUNSUPPORTED
    assert int(out.abs().sum()) == 0                  # nothing was launched
