"""Constant-time evidence: the same batched launch on four operand classes.

Runs the tuned plan for n (default 17669, 4096 products) on dense random,
all-zero, all-one and sparse (weight 131) operands.  Without --ncu: many
timed launches per class, median times and Welch's t statistic of every class
against dense (dudect-style).  With --ncu: exactly one launch per class, for
an ncu capture of instruction counts, e.g.

  ncu --metrics smsp__inst_executed.sum,gpu__time_duration.sum --clock-control none \\
      -k regex:fused_mul_kernel -c 4 python -m paper_2201_10473_gb300.experiments.ct_operands --ncu
"""
import argparse
import math
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from paper_2201_10473_gb300 import Context  # noqa: E402


def welch_t(x, y):
    x, y = np.asarray(x), np.asarray(y)
    vx, vy = x.var(ddof=1) / len(x), y.var(ddof=1) / len(y)
    return float((x.mean() - y.mean()) / math.sqrt(vx + vy)) if vx + vy > 0 else 0.0


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=17669)
    p.add_argument("--count", type=int, default=4096)
    p.add_argument("--samples", type=int, default=200)
    p.add_argument("--ncu", action="store_true")
    p.add_argument("--launch", choices=("cta", "persistent"), default="cta",
                   help="one CTA per product (the default form) or persistent CTAs taking products from a counter")
    a = p.parse_args()
    persistent = a.launch == "persistent"
    n, count = a.n, a.count
    L = wl.limbs(n)
    ctx = Context(0, batch_hint=count)
    dense_a, dense_b = wl.dense_pair(1, n, count)
    ones = wl.mask_top(np.full((count, L), np.uint64(0xFFFFFFFFFFFFFFFF)), n)
    zeros = np.zeros((count, L), np.uint64)
    classes = {"dense": (dense_a, dense_b), "zero": (zeros, zeros), "ones": (ones, ones),
               "sparse131": (dense_a, wl.sparse_operands(2, n, 131, count))}
    dev = {k: (torch.from_numpy(x.view(np.int64)).cuda(), torch.from_numpy(y.view(np.int64)).cuda())
           for k, (x, y) in classes.items()}
    out = torch.empty((count, L), dtype=torch.int64, device="cuda")
    if a.ncu:
        for k, (x, y) in dev.items():
            ctx.mul_strided(x, y, n, True, out=out, persistent=persistent)
            torch.cuda.synchronize()
            print(f"launched class {k}", flush=True)
        return
    times = {k: [] for k in dev}
    for _ in range(3):
        for x, y in dev.values():
            ctx.mul_strided(x, y, n, True, out=out, persistent=persistent)
    torch.cuda.synchronize()
    order = list(dev)
    for s in range(a.samples):
        for k in order[s % len(order):] + order[: s % len(order)]:   # rotate the class order
            x, y = dev[k]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.mul_strided(x, y, n, True, out=out, persistent=persistent)
            e1.record()
            torch.cuda.synchronize()
            times[k].append(e0.elapsed_time(e1))
    print(f"n={n} count={count} plan={ctx.get_plan(n)} launch={a.launch} samples={a.samples}")
    for k, t in times.items():
        print(f"{k:10s} median {np.median(t):.4f} ms  mean {np.mean(t):.4f}  sd {np.std(t):.4f}  "
              f"Welch t vs dense {welch_t(t, times['dense']):+.2f}")


if __name__ == "__main__":
    main()
