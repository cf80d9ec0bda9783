"""The two leaf experiments against the oracle (the product of Sec. 2.1),
through their test entry points (paper_2201_10473_gb300/_lib/libgf2x_exp_*.so,
built by build()):

* the tensor-core Toeplitz multiplier (fp8 warp MMA on bit-unpacked
  Toeplitz tiles, counts in fp32, parity = product bit), 512 x 512 bits;
* the bitsliced leaves (32 leaves of 192 x 192 bits per group, Karatsuba and
  diagonal-schoolbook block schedules) and the comb they are measured
  against.

Every result row must equal the oracle's full product bit for bit."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from gpu_util import first_diff

pytestmark = pytest.mark.gpu


def _lib(name):
    from paper_2201_10473_gb300 import build
    build.build()
    return ctypes.CDLL(build.experiment_lib(name))


def _special_rows(x, nwords):
    """Row 0 all ones, row 1 zero, row 2 a single top bit, row 3 a single low bit."""
    x[0] = np.uint64(0xFFFFFFFFFFFFFFFF)
    x[1] = 0
    x[2] = 0
    x[2, nwords // 2 - 1] = np.uint64(1 << 63)
    x[3] = 0
    x[3, 0] = 1
    return x


@pytest.mark.parametrize("kernel", ["gf2x_exp_tc_mul512", "gf2x_exp_comb_mul512"])
def test_tensor_core_toeplitz_512_matches_oracle(kernel):
    lib = _lib("libgf2x_exp_tc.so")
    fn = getattr(lib, kernel)
    fn.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    n, count = 512, 4099                              # several waves of warps and a ragged tail
    a, b = wl.dense_pair(7100, n, count)
    a, b = _special_rows(a.copy(), 16), _special_rows(b.copy(), 16)
    b[0] = np.uint64(0xFFFFFFFFFFFFFFFF)
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    out = torch.full((count, 16), -1, dtype=torch.int64, device="cuda")
    assert fn(da.data_ptr(), db.data_ptr(), out.data_ptr(), count, None) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    exp = oracle.mul_batch(a, b, n, reduce=False)
    assert np.array_equal(got, exp), first_diff(got, exp)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_bitsliced_leaves_match_oracle(mode):
    lib = _lib("libgf2x_exp_bitsliced.so")
    lib.gf2x_exp_bitsliced_group.argtypes = [ctypes.c_int]
    lib.gf2x_exp_bitsliced_group.restype = ctypes.c_int
    fn = lib.gf2x_exp_bitsliced_leaves
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    G = lib.gf2x_exp_bitsliced_group(mode)
    nctas = 2 * 152 + 5
    leaves = nctas * 32 * G
    n = 192
    a, b = wl.dense_pair(7200 + mode, n, leaves)      # 3 limbs = 6 words each
    a, b = _special_rows(a.copy(), 6), _special_rows(b.copy(), 6)
    rows = np.concatenate([a, b], axis=1)             # one leaf: a then b, 12 words
    din = torch.from_numpy(rows.view(np.int64)).cuda()
    dout = torch.full_like(din, -1)
    assert fn(din.data_ptr(), dout.data_ptr(), nctas, mode, None) == 0
    torch.cuda.synchronize()
    got = dout.cpu().numpy().view(np.uint64)
    exp = oracle.mul_batch(a, b, n, reduce=False)     # 6 limbs = the 12-word product
    assert np.array_equal(got, exp), first_diff(got, exp)
