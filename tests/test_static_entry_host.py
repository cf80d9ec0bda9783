"""Argument checks of gf2x_mul_strided_static, on CPU: every refusal the
header lists is returned before the entry touches a device (the addresses
below are never dereferenced), with the header's status codes.  Every call
here is one the entry refuses; the module runs only where no GPU is
visible, so that no call could ever reach a launch."""
import ctypes

import pytest
import torch

from paper_2201_10473_gb300 import gf2x

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="host-only checks with fake device addresses")

OK, EINVAL, EUNSUPPORTED = 0, 1, 5
STATIC_SCRATCH_BYTES = 4 << 20
OUT, A, B = 0x10000000, 0x20000000, 0x30000000     # disjoint, 16-byte aligned, never read


def _entry():
    fn = gf2x.lib().gf2x_mul_strided_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_size_t,
                   ctypes.c_size_t, ctypes.c_size_t, ctypes.c_uint32, ctypes.POINTER(gf2x.PlanSpec), ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _call(out=OUT, a=A, b=B, n=17669, count=2, stride_in=None, stride_out=None, flags=1, spec=None):
    L = gf2x.limbs(n) if n else 1
    s = ctypes.byref(gf2x.parse_spec(spec)) if spec else None
    return _entry()(out, a, b, n, count, L if stride_in is None else stride_in, L if stride_out is None else stride_out,
                    flags, s, None)


def test_sizes_outside_the_range_are_unsupported():
    assert _call(n=0) == EUNSUPPORTED
    assert _call(n=131073) == EUNSUPPORTED


def test_an_empty_batch_is_a_no_op():
    assert _call(out=None, a=None, b=None, count=0) == OK


@pytest.mark.parametrize("kw", [dict(out=None), dict(a=None), dict(b=None), dict(a=A + 4), dict(out=OUT + 12),
                                dict(flags=2), dict(flags=1 | 256)])
def test_bad_pointers_alignment_and_flags_are_invalid(kw):
    assert _call(**kw) == EINVAL


def test_strides_shorter_than_a_row_are_invalid():
    L = gf2x.limbs(17669)
    assert _call(stride_in=L - 1) == EINVAL
    assert _call(stride_out=L - 1) == EINVAL
    assert _call(flags=0, stride_out=L) == EINVAL            # a full product needs ceil((2n-1)/64) limbs


def test_results_overlapping_an_operand_are_invalid():
    L = gf2x.limbs(17669)
    assert _call(out=A + 8 * L) == EINVAL                     # inside a's second row
    assert _call(out=B - 8) == EINVAL                         # ends inside b's first row


def test_a_plan_that_is_not_split_is_invalid():
    assert _call(spec="T1.K2.K2.K2.K2.K2/6/128/1/0/0") == EINVAL


def test_a_batch_beyond_the_static_scratch_is_unsupported():
    spec = "T2.K2.K2.K2.K2.K2/6/128/1/0/1"
    per = gf2x.plan_info(17669, spec)["scratch_bytes"]
    count = STATIC_SCRATCH_BYTES // per + 1
    L = gf2x.limbs(17669)
    assert _call(count=count, spec=spec, out=0x40000000, a=0x80000000, b=0xC0000000) == EUNSUPPORTED
    assert 8 * count * L < 0x40000000                         # the three ranges stay disjoint
    assert _call(count=1 << 31) == EUNSUPPORTED               # more products than one launch takes
