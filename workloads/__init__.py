"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module only draws random operands and request streams.  It holds none
of the multiplication arithmetic, so the GPU path and the oracle can both use
it without sharing any of the method.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: output i
of stream `key` is mix64(key + (i+1)*GAMMA).  The stream of operand o
(0 = a, 1 = b) of product p under seed s has key mix64(mix64(s) + (2p+o+1)*GAMMA).

Every limb is a raw 64-bit output, so coefficients are iid Bernoulli(0.5),
and the bits at or above n in the top limb are cleared (dense operands of the
paper's workloads: HQC/BIKE polynomials of 10k-60k bits, Sec. 1 and Sec. 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

#: seed of workload k (1-based) is BASE_SEED + k
BASE_SEED = 22011047300

#: the HQC sizes (Sec. 4) and the BIKE-like sizes used by the serving mix
HQC_SIZES = (17669, 35851, 57637)
SERVING_SIZES = (12323, 17669, 24659, 35851, 40973, 57637)


def mix64(z):
    """SplitMix64 output function on uint64 numpy values (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _py_mix64(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream(key: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of the counter-based SplitMix64 stream `key`."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key & _MASK64) + idx * GAMMA)


def operand_keys(seed: int, products: np.ndarray, operand: int) -> np.ndarray:
    p = np.asarray(products, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = (np.uint64(2) * p + np.uint64(operand + 1)) * GAMMA
        return mix64(mix64(np.uint64(seed & _MASK64)) + ctr)


def limbs(n: int) -> int:
    return (n + 63) // 64


def mask_top(x: np.ndarray, n: int) -> np.ndarray:
    """Clear bits >= n in the last limb of every row (in place) and return x."""
    if n % 64:
        x[..., limbs(n) - 1] &= np.uint64((1 << (n % 64)) - 1)
    return x


def dense_operands(seed: int, n: int, count: int, operand: int, first: int = 0) -> np.ndarray:
    """(count, ceil(n/64)) uint64: operand `operand` of products first..first+count-1."""
    L = limbs(n)
    keys = operand_keys(seed, np.arange(first, first + count), operand)[:, None]
    idx = np.arange(1, L + 1, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        out = mix64(keys + idx * GAMMA)
    return mask_top(np.ascontiguousarray(out), n)


def dense_pair(seed: int, n: int, count: int, first: int = 0):
    return dense_operands(seed, n, count, 0, first), dense_operands(seed, n, count, 1, first)


class _Rng:
    """Sequential uniform integers from one SplitMix64 stream."""

    def __init__(self, key: int):
        self.key = key & _MASK64
        self.ctr = 0

    def next64(self) -> int:
        self.ctr += 1
        return _py_mix64(self.key + self.ctr * 0x9E3779B97F4A7C15)

    def below(self, m: int) -> int:
        """Uniform integer in [0, m) by the multiply-shift map of a 64-bit draw."""
        return (self.next64() * m) >> 64

    def uniform(self) -> float:
        return (self.next64() >> 11) * (1.0 / (1 << 53))


def sparse_operand(seed: int, n: int, weight: int, product: int, operand: int = 1) -> np.ndarray:
    """One operand with exactly `weight` set bits at uniform positions drawn
    without replacement by Floyd's algorithm."""
    rng = _Rng(int(operand_keys(seed, np.array([product]), operand)[0]) ^ 0x5EED5EED)
    chosen = set()
    for j in range(n - weight, n):
        t = rng.below(j + 1)
        chosen.add(j if t in chosen else t)
    out = np.zeros(limbs(n), dtype=np.uint64)
    for pos in chosen:
        out[pos // 64] |= np.uint64(1 << (pos % 64))
    return out


def sparse_operands(seed: int, n: int, weight: int, count: int, first: int = 0) -> np.ndarray:
    return np.stack([sparse_operand(seed, n, weight, first + p) for p in range(count)]) if count else \
        np.zeros((0, limbs(n)), dtype=np.uint64)


def shuffle(seed: int, items: list) -> list:
    """Fisher-Yates shuffle driven by the seed's stream."""
    rng = _Rng(_py_mix64(seed) ^ 0xF15E5)
    out = list(items)
    for i in range(len(out) - 1, 0, -1):
        j = rng.below(i + 1)
        out[i], out[j] = out[j], out[i]
    return out


def poisson_arrivals(seed: int, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = _Rng(_py_mix64(seed) ^ 0xA331)
    t = 0.0
    out = np.empty(count, dtype=np.float64)
    for i in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_per_s
        out[i] = t
    return out


def uniform_choice(seed: int, count: int, choices) -> list:
    rng = _Rng(_py_mix64(seed) ^ 0xC401CE)
    return [choices[rng.below(len(choices))] for _ in range(count)]


@dataclass
class Workload:
    """One of the five measured workloads."""
    key: int
    name: str
    sizes: list = field(default_factory=list)   # n of every product, in launch order
    reduce: bool = True
    description: str = ""

    @property
    def seed(self) -> int:
        return BASE_SEED + self.key


def workload(k: int) -> Workload:
    """The five workloads: k = 1..5."""
    if k == 1:
        return Workload(1, "plain-12323-full", [12323] * 256, False,
                        "256 products at n=12323, full product, one launch per product")
    if k == 2:
        return Workload(2, "hqc128-17669-mulmod", [17669] * 4096, True,
                        "4096 products at n=17669 mod X^n-1")
    if k == 3:
        sizes = [17669] * 2048 + [35851] * 1024 + [57637] * 512
        return Workload(3, "uneven-hqc-mix-mulmod", shuffle(BASE_SEED + 3, sizes), True,
                        "2048@17669 + 1024@35851 + 512@57637, interleaved, mod X^n-1")
    if k == 4:
        return Workload(4, "hqc256-57637-mulmod", [57637] * 16384, True,
                        "16384 products at n=57637 mod X^n-1 (dense; sparse-131 variant)")
    if k == 5:
        return Workload(5, "serving-mix", uniform_choice(BASE_SEED + 5, 200000, SERVING_SIZES), True,
                        "200k requests, sizes uniform over the six serving sizes, mod X^n-1")
    raise ValueError(k)


def mixed_operands(seed: int, sizes, index_base: int = 0):
    """Per-product (a, b) arrays for a list of sizes (product p uses stream p)."""
    out = []
    for p, n in enumerate(sizes):
        a = dense_operands(seed, n, 1, 0, first=index_base + p)[0]
        b = dense_operands(seed, n, 1, 1, first=index_base + p)[0]
        out.append((a, b))
    return out
