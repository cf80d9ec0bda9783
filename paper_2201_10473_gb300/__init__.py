"""GB300-native constant-time multiplication of dense binary polynomials.

Multiplication in F2[X] and F2[X]/(X^n - 1) for the 10k-60k-bit sizes of
HQC and BIKE (Robert & Veron, "Faster multiplication over F2[X] using AVX512
instruction set and VPCLMULQDQ instruction"), as hand-written CUDA for
sm_103a behind the C ABI of include/gf2x_gb300.h:

  gf2x.py      ctypes binding of libgf2x_gb300.so (marshalling only)
  build.py     nvcc build of the library (in-tree, sm_103a)
  autotune.py  measured plan search and the timing log
  costmodel.py MLP plan cost model trained by the library's CUDA kernels
  serve.py     continuous-batching request loop
"""
from .gf2x import (Context, Gf2xError, default_spec, full_limbs, lib, limbs, pack_items, parse_spec,  # noqa: F401
                   plan_info, sparse_info, spec_text)

__all__ = ["Context", "Gf2xError", "default_spec", "plan_info", "sparse_info", "limbs", "full_limbs", "lib", "parse_spec",
           "spec_text", "pack_items"]
