"""The oracle: plain CPU definitions the GPU path is checked against.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (``paper_2201_10473_gb300``) never imports
it, and it imports nothing from the product.

``gf2x_oracle.c`` holds the polynomial arithmetic (plain C, built by
:func:`build`); this module is a ctypes wrapper over numpy ``uint64`` limb
arrays.  ``mlp.py`` holds the fp64 reference of the plan cost-model network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf2x_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_U64P = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP for the batch driver)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            for name in ("oracle_mul", "oracle_mul_bitwise", "oracle_mulmod", "oracle_mulmod_circulant"):
                fn = getattr(lib, name)
                fn.argtypes = [_U64P, _U64P, _U64P, ctypes.c_uint32]
                fn.restype = ctypes.c_int
            lib.oracle_mul_batch.argtypes = [_U64P, _U64P, _U64P, ctypes.c_uint32, ctypes.c_size_t,
                                             ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]
            lib.oracle_mul_batch.restype = ctypes.c_int
            lib.oracle_full_limbs.argtypes = [ctypes.c_uint32]
            lib.oracle_full_limbs.restype = ctypes.c_size_t
            lib.oracle_limbs.argtypes = [ctypes.c_uint32]
            lib.oracle_limbs.restype = ctypes.c_size_t
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def limbs(n: int) -> int:
    """Limbs of a polynomial with n coefficients."""
    return (n + 63) // 64


def full_limbs(n: int) -> int:
    """Limbs of the full product of two n-coefficient polynomials."""
    return (2 * n - 1 + 63) // 64


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(x: np.ndarray):
    return x.ctypes.data_as(_U64P)


def _prep(a, n):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if a.shape[-1] < limbs(n):
        raise ValueError(f"operand has {a.shape[-1]} limbs, need {limbs(n)} for n={n}")
    return a


def _call(name, a, b, n, out_limbs):
    a = _prep(a, n)
    b = _prep(b, n)
    out = np.zeros(out_limbs, dtype=np.uint64)
    st = getattr(_load(), name)(_ptr(out), _ptr(a), _ptr(b), n)
    if st != 0:
        raise RuntimeError(f"{name} failed with status {st}")
    return out


def mul(a, b, n: int) -> np.ndarray:
    """Full product (shift-and-XOR over limbs)."""
    return _call("oracle_mul", a, b, n, full_limbs(n))


def mul_bitwise(a, b, n: int) -> np.ndarray:
    """Full product, coefficient pair by coefficient pair."""
    return _call("oracle_mul_bitwise", a, b, n, full_limbs(n))


def mulmod(a, b, n: int) -> np.ndarray:
    """a*b mod X^n - 1 via the full product and a fold."""
    return _call("oracle_mulmod", a, b, n, limbs(n))


def mulmod_circulant(a, b, n: int) -> np.ndarray:
    """a*b mod X^n - 1 via the circulant matrix formulation."""
    return _call("oracle_mulmod_circulant", a, b, n, limbs(n))


def mul_batch(a: np.ndarray, b: np.ndarray, n: int, reduce: bool, nthreads: int = 0) -> np.ndarray:
    """Row p of the result is the product of rows p of a and b."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    if a.ndim != 2 or a.shape != b.shape:
        raise ValueError("a and b must be equal-shaped 2-D limb arrays")
    count, stride = a.shape
    if stride < limbs(n):
        raise ValueError("too few limbs per row")
    ol = limbs(n) if reduce else full_limbs(n)
    out = np.zeros((count, ol), dtype=np.uint64)
    if count == 0:
        return out
    st = _load().oracle_mul_batch(_ptr(out), _ptr(a), _ptr(b), n, count, stride, ol, int(bool(reduce)), int(nthreads))
    if st != 0:
        raise RuntimeError(f"oracle_mul_batch failed with status {st}")
    return out
