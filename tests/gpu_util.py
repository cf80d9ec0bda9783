"""Helpers shared by the GPU tests: numpy uint64 limbs <-> CUDA int64 tensors."""
import numpy as np
import torch


def to_dev(x: np.ndarray) -> torch.Tensor:
    x = np.ascontiguousarray(x, dtype=np.uint64)
    return torch.from_numpy(x.view(np.int64)).cuda()


def to_host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def first_diff(got: np.ndarray, expect: np.ndarray) -> str:
    d = np.nonzero(got != expect)
    if len(d[0]) == 0:
        return "equal"
    idx = tuple(int(v[0]) for v in d)
    return f"first differing limb at {idx}: got {int(got[idx]):#018x} expected {int(expect[idx]):#018x} " \
           f"({len(d[0])} limbs differ)"
