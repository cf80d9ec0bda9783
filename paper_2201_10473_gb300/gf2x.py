"""Python binding of libgf2x_gb300.so (include/gf2x_gb300.h): argument
marshalling only.  Every product is computed by the library's CUDA kernels;
there is no CPU path, and a missing library is an error.

Polynomials are torch tensors of dtype int64 on a CUDA device holding the
little-endian uint64 limbs (bit k of limb i is coefficient 64i + k).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

MAX_N = 131072
MAX_LEVELS = 8
LEVEL_KARATSUBA = 0
LEVEL_TOOM3 = 1
REDUCE = 1
HOST_INPUTS_READY = 1 << 8
BATCH_PERSISTENT = 1
BATCH_ITEMS_ON_DEVICE = 2
BATCH_LARGEST_FIRST = 4
BATCH_SHARED_A = 8
BATCH_DYNAMIC = 16

STATUS = {0: "GF2X_OK", 1: "GF2X_EINVAL", 2: "GF2X_ENOMEM", 3: "GF2X_ECUDA", 4: "GF2X_ETIMEOUT",
          5: "GF2X_EUNSUPPORTED", 6: "GF2X_EBUSY", 7: "GF2X_EDEVICE"}


class Gf2xError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class PlanSpec(ctypes.Structure):
    _fields_ = [("nlev", ctypes.c_uint32), ("kind", ctypes.c_uint32 * MAX_LEVELS),
                ("arg", ctypes.c_uint32 * MAX_LEVELS), ("leaf_words", ctypes.c_uint32),
                ("threads", ctypes.c_uint32), ("seq_top", ctypes.c_uint32), ("fuse_leaf", ctypes.c_uint32),
                ("split_top", ctypes.c_uint32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("top_words", ctypes.c_uint32), ("leaf_words", ctypes.c_uint32),
                ("nleaves", ctypes.c_uint32), ("threads", ctypes.c_uint32), ("smem_bytes", ctypes.c_uint32),
                ("level_words", ctypes.c_uint32 * (MAX_LEVELS + 1)), ("ops_full", ctypes.c_uint64),
                ("ops_leaf", ctypes.c_uint64), ("clmul64", ctypes.c_uint64), ("bytes_in", ctypes.c_uint64),
                ("bytes_out_full", ctypes.c_uint64), ("bytes_out_reduced", ctypes.c_uint64),
                ("scratch_bytes", ctypes.c_uint64)]


class Item(ctypes.Structure):
    _fields_ = [("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("n", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_SZ = ctypes.c_size_t
_I = ctypes.c_int

_SIGNATURES = {
    "gf2x_status_str": ([_I], ctypes.c_char_p),
    "gf2x_version": ([], ctypes.c_char_p),
    "gf2x_default_spec": ([_U32, ctypes.POINTER(PlanSpec)], _I),
    "gf2x_plan_info_get": ([_U32, ctypes.POINTER(PlanSpec), ctypes.POINTER(PlanInfo)], _I),
    "gf2x_spec_parse": ([ctypes.c_char_p, ctypes.POINTER(PlanSpec)], _I),
    "gf2x_ctx_create": ([ctypes.POINTER(_P), _I, _SZ, ctypes.c_char_p], _I),
    "gf2x_ctx_alloc_count": ([_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)], _I),
    "gf2x_debug_fail_next_allocs": ([_U32], _U32),
    "gf2x_ctx_wait": ([_P, _P, _U32], _I),
    "gf2x_copy_rows": ([_P, _P, _SZ, _P], _I),
    "gf2x_ctx_destroy": ([_P], None),
    "gf2x_ctx_set_plan": ([_P, _U32, ctypes.POINTER(PlanSpec)], _I),
    "gf2x_ctx_get_plan": ([_P, _U32, ctypes.POINTER(PlanSpec)], _I),
    "gf2x_ctx_set_checked": ([_P, _I], _I),
    "gf2x_mul": ([_P, _P, _P, _P, _U32, _P], _I),
    "gf2x_mulmod_xn1": ([_P, _P, _P, _P, _U32, _P], _I),
    "gf2x_mul_strided": ([_P, _P, _P, _P, _U32, _SZ, _SZ, _SZ, _U32, _U32, _P], _I),
    "gf2x_mul_strided_host": ([_P, _P, _P, _P, _U32, _SZ, _SZ, _SZ, _U32, _P], _I),
    "gf2x_mul_unbalanced": ([_P, _P, _P, _U32, _SZ, _P, _U32, _SZ, _SZ, _SZ, _P], _I),
    "gf2x_mulmod_sparse": ([_P, _P, _P, _P, _U32, _U32, _SZ, _SZ, _SZ, _SZ, _P], _I),
    "gf2x_sparse_info_get": ([_U32, _P], _I),
    "gf2x_mulmod_shared_tc": ([_P, _P, _P, _P, _U32, _SZ, _SZ, _SZ, _P], _I),
    "gf2x_mul_toom4": ([_P, _P, _P, _P, _U32, _SZ, _SZ, _SZ, _U32, _P], _I),
    "gf2x_mul_toom5": ([_P, _P, _P, _P, _U32, _SZ, _SZ, _SZ, _U32, _P], _I),
    "gf2x_mul_batched": ([_P, _P, _SZ, _U32, _P], _I),
    "gf2x_ctx_prepare": ([_P, ctypes.POINTER(_U32), _SZ, _P], _I),
    "gf2x_ctx_launch_shape": ([_P, _U32, ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32),
                               ctypes.POINTER(_U32)], _I),
    "gf2x_ctx_sync_status": ([_P, _P], _I),
    "gf2x_ctx_last_error": ([_P], ctypes.c_char_p),
    "gf2x_ctx_load_plan_db": ([_P, ctypes.c_char_p, _SZ], _I),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libgf2x_gb300.so is not built ({path}); run paper_2201_10473_gb300.build.build()")
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def limbs(n: int) -> int:
    return (n + 63) // 64


def full_limbs(n: int) -> int:
    return (2 * n - 1 + 63) // 64


# ------------------------------------------------------------------ plans

def parse_spec(text: str) -> PlanSpec:
    s = PlanSpec()
    st = lib().gf2x_spec_parse(text.encode(), ctypes.byref(s))
    if st:
        raise Gf2xError(st, "gf2x_spec_parse", text)
    return s


def spec_text(s: PlanSpec) -> str:
    lv = ".".join(("K" if s.kind[i] == LEVEL_KARATSUBA else "T") + str(s.arg[i]) for i in range(s.nlev))
    return f"{lv}/{s.leaf_words}/{s.threads}/{s.seq_top}/{s.fuse_leaf}/{s.split_top}"


def default_spec(n: int) -> str:
    s = PlanSpec()
    st = lib().gf2x_default_spec(n, ctypes.byref(s))
    if st:
        raise Gf2xError(st, "gf2x_default_spec", str(n))
    return spec_text(s)


def plan_info(n: int, spec: str | None = None) -> dict:
    """Plan facts for size n (default plan when spec is None); host only."""
    s = parse_spec(spec) if spec is not None else parse_spec(default_spec(n))
    info = PlanInfo()
    st = lib().gf2x_plan_info_get(n, ctypes.byref(s), ctypes.byref(info))
    if st:
        raise Gf2xError(st, "gf2x_plan_info_get", f"n={n} spec={spec}")
    d = {f: getattr(info, f) for f, _ in PlanInfo._fields_ if f != "level_words"}
    d["level_words"] = [info.level_words[i] for i in range(s.nlev + 1)]
    d["spec"] = spec_text(s)
    return d


class SparseInfo(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in ("n", "words_per_lane", "result_words_per_lane", "shared_stages",
                                               "register_stages", "lane_stages", "smem_bytes")]


def sparse_info(n: int) -> dict:
    """Kernel shape of the constant-time sparse product for size n; host only."""
    info = SparseInfo()
    st = lib().gf2x_sparse_info_get(n, ctypes.byref(info))
    if st:
        raise Gf2xError(st, "gf2x_sparse_info_get", f"n={n}")
    return {f: getattr(info, f) for f, _ in SparseInfo._fields_}


# ------------------------------------------------------------------ context

def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_operand(t: torch.Tensor, n: int, name: str):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int64 or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA int64 tensor of uint64 limbs")
    if t.shape[-1] < limbs(n) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with at least {limbs(n)} limbs in its last dimension")


PACKAGED_PLAN_DB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", "gb300_plan_db.txt")


class Context:
    """Owns a gf2x_ctx on one device.

    plan_db: a plan database file to install ("packaged" = the GB300-tuned
    database shipped with the package, None = the library's model-based
    default plans); batch_hint selects its batch bucket.
    workspace_bytes: 0 = scratch grows on demand; > 0 = one device arena of
    that size allocated now, and no compute call allocates afterwards."""

    def __init__(self, device: int | None = None, plan_db: str | None = "packaged", batch_hint: int = 2048,
                 workspace_bytes: int = 0):
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = ctypes.c_void_p()
        st = lib().gf2x_ctx_create(ctypes.byref(h), device, workspace_bytes, None)
        if st:
            raise Gf2xError(st, "gf2x_ctx_create")
        self._h = h
        self.plan_db = plan_db
        if plan_db == "packaged":
            plan_db = PACKAGED_PLAN_DB if os.path.exists(PACKAGED_PLAN_DB) else None
        if plan_db:
            self.load_plan_db(plan_db, batch_hint)

    def close(self):
        if getattr(self, "_h", None):
            lib().gf2x_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st, where):
        if st:
            raise Gf2xError(st, where, lib().gf2x_ctx_last_error(self._h).decode())

    # plans
    def set_plan(self, n: int, spec: str | None):
        s = parse_spec(spec) if spec is not None else None
        self._raise(lib().gf2x_ctx_set_plan(self._h, n, ctypes.byref(s) if s is not None else None), "set_plan")

    def get_plan(self, n: int) -> str:
        s = PlanSpec()
        self._raise(lib().gf2x_ctx_get_plan(self._h, n, ctypes.byref(s)), "get_plan")
        return spec_text(s)

    def load_plan_db(self, path: str, batch_hint: int = 4096):
        """Install the tuned plans of a plan database file (see autotune.py)."""
        self._raise(lib().gf2x_ctx_load_plan_db(self._h, path.encode(), batch_hint), "load_plan_db")

    def set_checked(self, on: bool):
        self._raise(lib().gf2x_ctx_set_checked(self._h, 1 if on else 0), "set_checked")

    def prepare(self, sizes, stream=None):
        arr = (ctypes.c_uint32 * len(sizes))(*sizes)
        self._raise(lib().gf2x_ctx_prepare(self._h, arr, len(sizes), _stream_handle(stream)), "prepare")

    def launch_shape(self, n: int) -> dict:
        t, sm, b, c = (ctypes.c_uint32() for _ in range(4))
        self._raise(lib().gf2x_ctx_launch_shape(self._h, n, ctypes.byref(t), ctypes.byref(sm), ctypes.byref(b),
                                                ctypes.byref(c)), "launch_shape")
        return {"threads": t.value, "smem_bytes": sm.value, "blocks_per_sm": b.value, "sm_count": c.value}

    def sync_status(self, stream=None):
        self._raise(lib().gf2x_ctx_sync_status(self._h, _stream_handle(stream)), "sync_status")

    def wait(self, timeout_ms: int, stream=None) -> int:
        """gf2x_ctx_wait: the status code (0, or GF2X_ETIMEOUT = 4 when the
        stream's work is not done within timeout_ms); other errors raise."""
        st = lib().gf2x_ctx_wait(self._h, _stream_handle(stream), timeout_ms)
        if st not in (0, 4):
            self._raise(st, "wait")
        return st

    def copy_rows(self, rows_dev: torch.Tensor, count: int, stream=None):
        """rows_dev: a CUDA int64 tensor of `count` (src, dst, limbs) triples (gf2x_copy_row)."""
        self._raise(lib().gf2x_copy_rows(self._h, rows_dev.data_ptr(), count, _stream_handle(stream)),
                    "gf2x_copy_rows")

    def alloc_count(self) -> tuple[int, int]:
        """(device + pinned allocations, their bytes) made by this context so far."""
        n, b = ctypes.c_uint64(), ctypes.c_uint64()
        self._raise(lib().gf2x_ctx_alloc_count(self._h, ctypes.byref(n), ctypes.byref(b)), "alloc_count")
        return n.value, b.value

    # products
    def mul(self, a: torch.Tensor, b: torch.Tensor, n: int, out: torch.Tensor | None = None, stream=None):
        """Full product a*b (one launch)."""
        _check_operand(a, n, "a")
        _check_operand(b, n, "b")
        if out is None:
            out = torch.empty(full_limbs(n), dtype=torch.int64, device=a.device)
        self._raise(lib().gf2x_mul(self._h, out.data_ptr(), a.data_ptr(), b.data_ptr(), n, _stream_handle(stream)),
                    "gf2x_mul")
        return out

    def mulmod(self, a: torch.Tensor, b: torch.Tensor, n: int, out: torch.Tensor | None = None, stream=None):
        """a*b mod X^n - 1 (one launch)."""
        _check_operand(a, n, "a")
        _check_operand(b, n, "b")
        if out is None:
            out = torch.empty(limbs(n), dtype=torch.int64, device=a.device)
        self._raise(lib().gf2x_mulmod_xn1(self._h, out.data_ptr(), a.data_ptr(), b.data_ptr(), n,
                                          _stream_handle(stream)), "gf2x_mulmod_xn1")
        return out

    def mul_strided(self, a: torch.Tensor, b: torch.Tensor, n: int, reduce: bool, out: torch.Tensor | None = None,
                    persistent: bool = False, stream=None):
        """Row p of the result is the product of rows p of a and b (2-D
        tensors).  A 1-D a is one operand shared by every row of b
        (GF2X_BATCH_SHARED_A)."""
        shared = a.dim() == 1
        if b.dim() != 2 or (not shared and a.shape != b.shape):
            raise ValueError("a and b must be equal-shaped 2-D tensors, or a 1-D a shared by the rows of b")
        _check_operand(a, n, "a")
        _check_operand(b, n, "b")
        count = b.shape[0]
        ol = limbs(n) if reduce else full_limbs(n)
        if out is None:
            out = torch.empty((count, ol), dtype=torch.int64, device=b.device)
        if out.dim() != 2 or out.shape[0] != count or out.shape[1] < ol or not out.is_contiguous():
            raise ValueError("bad output tensor")
        bflags = (BATCH_PERSISTENT if persistent else 0) | (BATCH_SHARED_A if shared else 0)
        self._raise(lib().gf2x_mul_strided(self._h, out.data_ptr(), a.data_ptr(), b.data_ptr(), n, count,
                                           b.shape[1], out.shape[1], REDUCE if reduce else 0,
                                           bflags, _stream_handle(stream)),
                    "gf2x_mul_strided")
        return out

    def mul_unbalanced(self, a: torch.Tensor, na: int, b: torch.Tensor, nb: int, out: torch.Tensor | None = None,
                       stream=None):
        """Full products of operands of different sizes: rows of a (na bits)
        times rows of b (nb bits), each 1-D (one product) or 2-D (one per
        row); result rows of ceil((na + nb - 1)/64) limbs."""
        if a.dim() != b.dim() or a.dim() not in (1, 2) or (a.dim() == 2 and a.shape[0] != b.shape[0]):
            raise ValueError("a and b must both be 1-D, or 2-D with the same number of rows")
        _check_operand(a, na, "a")
        _check_operand(b, nb, "b")
        one = a.dim() == 1
        A, B = (a[None], b[None]) if one else (a, b)
        count, ol = A.shape[0], (na + nb - 1 + 63) // 64
        if out is None:
            out = torch.empty((ol,) if one else (count, ol), dtype=torch.int64, device=a.device)
        O = out[None] if out.dim() == 1 else out
        if O.dim() != 2 or O.shape[0] != count or O.shape[1] < ol or not O.is_contiguous():
            raise ValueError("bad output tensor")
        self._raise(lib().gf2x_mul_unbalanced(self._h, O.data_ptr(), A.data_ptr(), na, A.shape[1], B.data_ptr(), nb,
                                              B.shape[1], count, O.shape[1], _stream_handle(stream)),
                    "gf2x_mul_unbalanced")
        return out

    def mulmod_shared_tc(self, a: torch.Tensor, b: torch.Tensor, n: int, out: torch.Tensor | None = None,
                         stream=None):
        """Row p of the result is a * b[p] mod X^n - 1 for ONE a (1-D), on the
        tensor cores (gf2x_mulmod_shared_tc; n odd, <= 65535)."""
        if a.dim() != 1 or b.dim() != 2:
            raise ValueError("a must be 1-D (one polynomial) and b 2-D (one row per product)")
        _check_operand(a, n, "a")
        _check_operand(b, n, "b")
        count = b.shape[0]
        if out is None:
            out = torch.empty((count, limbs(n)), dtype=torch.int64, device=b.device)
        if out.dim() != 2 or out.shape[0] != count or out.shape[1] < limbs(n) or not out.is_contiguous():
            raise ValueError("bad output tensor")
        self._raise(lib().gf2x_mulmod_shared_tc(self._h, out.data_ptr(), a.data_ptr(), b.data_ptr(), n, count,
                                                b.shape[1], out.shape[1], _stream_handle(stream)),
                    "gf2x_mulmod_shared_tc")
        return out

    def mul_toom4(self, a: torch.Tensor, b: torch.Tensor, n: int, reduce: bool, out: torch.Tensor | None = None,
                  stream=None):
        """mul_strided through a Toom-4 top level (seven child products per row)."""
        return self._toom("gf2x_mul_toom4", a, b, n, reduce, out, stream)

    def mul_toom5(self, a: torch.Tensor, b: torch.Tensor, n: int, reduce: bool, out: torch.Tensor | None = None,
                  stream=None):
        """mul_strided through a Toom-5 top level (nine child products per row)."""
        return self._toom("gf2x_mul_toom5", a, b, n, reduce, out, stream)

    def _toom(self, name, a, b, n, reduce, out, stream):
        if a.dim() != 2 or a.shape != b.shape:
            raise ValueError("a and b must be equal-shaped 2-D tensors")
        _check_operand(a, n, "a")
        _check_operand(b, n, "b")
        count = a.shape[0]
        ol = limbs(n) if reduce else full_limbs(n)
        if out is None:
            out = torch.empty((count, ol), dtype=torch.int64, device=a.device)
        if out.dim() != 2 or out.shape[0] != count or out.shape[1] < ol or not out.is_contiguous():
            raise ValueError("bad output tensor")
        self._raise(getattr(lib(), name)(self._h, out.data_ptr(), a.data_ptr(), b.data_ptr(), n, count, a.shape[1],
                                         out.shape[1], REDUCE if reduce else 0, _stream_handle(stream)), name)
        return out

    def mulmod_sparse(self, a: torch.Tensor, pos: torch.Tensor, n: int, out: torch.Tensor | None = None,
                      stream=None):
        """Constant-time a * b mod X^n - 1 with b = sum_j X^pos[j]: a is a
        (count, >= ceil(n/64)) int64 CUDA tensor of dense rows, pos a
        (count, w) int32 CUDA tensor of positions (< n) of the sparse rows."""
        if a.dim() != 2 or pos.dim() != 2 or pos.shape[0] != a.shape[0]:
            raise ValueError("a and pos must be 2-D with one row per product")
        _check_operand(a, n, "a")
        if pos.dtype != torch.int32 or not pos.is_cuda or not pos.is_contiguous():
            raise TypeError("pos must be a contiguous CUDA int32 tensor")
        count, w = a.shape[0], pos.shape[1]
        if out is None:
            out = torch.empty((count, limbs(n)), dtype=torch.int64, device=a.device)
        if out.dim() != 2 or out.shape[0] != count or out.shape[1] < limbs(n) or not out.is_contiguous():
            raise ValueError("bad output tensor")
        self._raise(lib().gf2x_mulmod_sparse(self._h, out.data_ptr(), a.data_ptr(), pos.data_ptr() if w else None,
                                             w, n, count, a.shape[1], w, out.shape[1], _stream_handle(stream)),
                    "gf2x_mulmod_sparse")
        return out

    def mul_strided_host(self, a: torch.Tensor, b: torch.Tensor, n: int, reduce: bool,
                         out: torch.Tensor | None = None, stream=None, inputs_ready: bool = False):
        """mul_strided with CPU tensors (pinned for overlapped copies): the
        library copies chunks in, multiplies and copies results out on its own
        streams; `stream` waits for the last copy.  Keep a, b and out alive and
        unchanged until `stream` has been synchronized.  inputs_ready: a and b
        are final now and out is unused by earlier work, so nothing of the
        call waits for earlier work on `stream`."""
        if a.dim() != 2 or a.shape != b.shape:
            raise ValueError("a and b must be equal-shaped 2-D tensors")
        for t, name in ((a, "a"), (b, "b")):
            if t.device.type != "cpu" or t.dtype != torch.int64 or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous int64 CPU tensor")
            if t.shape[1] < limbs(n):
                raise ValueError(f"{name} has fewer than ceil(n/64) limbs")
        count = a.shape[0]
        ol = limbs(n) if reduce else full_limbs(n)
        if out is None:
            out = torch.empty((count, ol), dtype=torch.int64, pin_memory=True)
        if out.device.type != "cpu" or out.dim() != 2 or out.shape[0] != count or out.shape[1] < ol \
                or not out.is_contiguous():
            raise ValueError("bad output tensor")
        self._raise(lib().gf2x_mul_strided_host(self._h, out.data_ptr(), a.data_ptr(), b.data_ptr(), n, count,
                                                a.shape[1], out.shape[1],
                                                (REDUCE if reduce else 0) | (HOST_INPUTS_READY if inputs_ready else 0),
                                                _stream_handle(stream)), "gf2x_mul_strided_host")
        return out

    def mul_batched(self, items, persistent: bool = False, largest_first: bool = False, stream=None,
                    dynamic: bool = False):
        """items: list of (a, b, out, n, reduce) with CUDA tensors; one launch per leaf size.
        dynamic (persistent only): CTAs take items in order from a counter."""
        arr = (Item * len(items))()
        for i, (a, b, out, n, reduce) in enumerate(items):
            _check_operand(a, n, "a")
            _check_operand(b, n, "b")
            arr[i] = Item(a.data_ptr(), b.data_ptr(), out.data_ptr(), n, REDUCE if reduce else 0)
        flags = (BATCH_PERSISTENT if persistent else 0) | (BATCH_LARGEST_FIRST if largest_first else 0) | \
            (BATCH_DYNAMIC if dynamic else 0)
        self._raise(lib().gf2x_mul_batched(self._h, ctypes.cast(arr, ctypes.c_void_p), len(items), flags,
                                           _stream_handle(stream)), "gf2x_mul_batched")

    def mul_batched_device(self, items_dev: torch.Tensor, count: int, persistent: bool = True, stream=None,
                           dynamic: bool = False):
        """items_dev: a CUDA tensor holding `count` packed gf2x_item records (see pack_items).
        dynamic (persistent only): CTAs take items in array order from a counter."""
        flags = BATCH_ITEMS_ON_DEVICE | (BATCH_PERSISTENT if persistent else 0) | (BATCH_DYNAMIC if dynamic else 0)
        self._raise(lib().gf2x_mul_batched(self._h, items_dev.data_ptr(), count, flags, _stream_handle(stream)),
                    "gf2x_mul_batched(device)")


def pack_items(rows) -> torch.Tensor:
    """Pack (a_ptr, b_ptr, out_ptr, n, flags) rows into an int64 CPU tensor of
    gf2x_item records (4 int64 words each), ready to copy to the device."""
    t = torch.empty((len(rows), 4), dtype=torch.int64)
    for i, (a, b, o, n, f) in enumerate(rows):
        t[i, 0] = a
        t[i, 1] = b
        t[i, 2] = o
        t[i, 3] = (int(n) & 0xFFFFFFFF) | ((int(f) & 0xFFFFFFFF) << 32)
    return t
