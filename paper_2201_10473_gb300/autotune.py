"""Measured plan search for the fused multiplication kernel.

The autotuner enumerates recursion plans for a size n (optional Toom-3 top
level with several word shifts, non-increasing Karatsuba split sequences,
every compiled leaf size, fused or shared-memory last level, breadth-first or
sequential top, several CTA sizes), measures each on the GPU with CUDA events
in the launch form it will be used in (one batched launch: a persistent grid,
or one CTA per product with --launch cta), and
keeps the fastest.  Every measurement is appended to a JSONL timing log,
which also trains the learned cost model (costmodel.py).

Plans differ only in how the product is computed, never in its value: before
a candidate is timed, its outputs on a probe batch are compared with those of
the context's current plan, and a mismatch is an error.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import time
from dataclasses import dataclass

from . import gf2x

TOOM_SHIFTS = (0, 1, 2, 4, 8, 16)
THREAD_CHOICES = (0, 128, 192, 256, 320, 384, 448, 512, 640, 768)


def _kseqs(max_depth: int = 7):
    out = [()]
    def rec(cur, maxk, depth):
        if depth == 0:
            return
        for k in (5, 3, 2):
            if k <= maxk:
                nxt = cur + (k,)
                out.append(nxt)
                rec(nxt, k, depth - 1)
    rec((), 5, max_depth)
    return out


def candidate_specs(n: int, max_waste: float = 1.30, threads=THREAD_CHOICES, limit: int | None = None,
                    split_from: int = 24000):
    """Valid plan specs for size n whose padded size is at most max_waste * n
    (split-top plans too, for n >= split_from)."""
    seen = set()
    out = []
    for W in TOOM_SHIFTS:
        for ks in _kseqs():
            levels = ([f"T{W}"] if W else []) + [f"K{k}" for k in ks]
            if not levels:
                continue
            base = ".".join(levels)
            for S in (4, 6, 8, 10, 12, 16):
                for seq, fuse, split in itertools.product((0, 1), (0, 1), (0, 1) if n >= split_from else (0,)):
                        spec0 = f"{base}/{S}/0/{seq}/{fuse}/{split}"
                        try:
                            info = gf2x.plan_info(n, spec0)
                        except gf2x.Gf2xError:
                            continue
                        if 32 * info["top_words"] > max_waste * n:
                            continue
                        maxT = 768 if S <= 6 else 512
                        for t in threads:
                            if t and (t > maxT or t < 64):
                                continue
                            spec = f"{base}/{S}/{t}/{seq}/{fuse}/{split}"
                            if t:
                                try:
                                    gf2x.plan_info(n, spec)
                                except gf2x.Gf2xError:
                                    continue
                            key = (base, S, t or info["threads"], seq, fuse, split)
                            if key in seen:
                                continue
                            seen.add(key)
                            out.append(spec)
                            if limit and len(out) >= limit:
                                return out
    return out


@dataclass
class Measurement:
    n: int
    batch: int
    spec: str
    ms: float
    mults_per_s: float
    threads: int
    smem_bytes: int
    blocks_per_sm: int


class Autotuner:
    """Times plan specs for one context; appends every timing to `log_path`."""

    def __init__(self, ctx: gf2x.Context, log_path: str | None = None, reps: int = 5, warmup: int = 2,
                 persistent: bool = True):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.log_path = log_path
        self.persistent = persistent   # the launch form timed (False: one CTA per product)
        self.reps = reps
        self.warmup = warmup
        self._inputs = {}
        self.failures = []   # (n, batch, spec, message) of candidates that could not be measured

    def renew_context(self):
        """Replace the context by a fresh one on the same device (same plan database)."""
        old = self.ctx
        self.ctx = gf2x.Context(old.device, plan_db=getattr(old, "plan_db", "packaged"))
        old.close()

    def _operands(self, n: int, batch: int):
        key = (n, batch)
        if key not in self._inputs:
            torch = self.torch
            g = torch.Generator(device="cuda")
            g.manual_seed(n * 1000003 + batch)
            L = gf2x.limbs(n)
            a = torch.randint(-2**62, 2**62, (batch, L), dtype=torch.int64, device="cuda", generator=g)
            b = torch.randint(-2**62, 2**62, (batch, L), dtype=torch.int64, device="cuda", generator=g)
            out = torch.empty((batch, L), dtype=torch.int64, device="cuda")
            ref = torch.empty((min(batch, 64), L), dtype=torch.int64, device="cuda")
            chk = torch.empty_like(ref)
            self._inputs[key] = (a, b, out, ref, chk)
        return self._inputs[key]

    def measure(self, n: int, spec: str, batch: int, persistent: bool | None = None, verify: bool = True) -> Measurement:
        torch = self.torch
        persistent = self.persistent if persistent is None else persistent
        a, b, out, ref, chk = self._operands(n, batch)
        m = ref.shape[0]
        prev = self.ctx.get_plan(n)
        if verify:
            self.ctx.mul_strided(a[:m], b[:m], n, True, out=ref)
        self.ctx.set_plan(n, spec)
        try:
            if verify:
                self.ctx.mul_strided(a[:m], b[:m], n, True, out=chk)
                if not torch.equal(ref, chk):
                    raise RuntimeError(f"plan {spec} disagrees with plan {prev} at n={n}")
            for _ in range(self.warmup):
                self.ctx.mul_strided(a, b, n, True, out=out, persistent=persistent)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(self.reps):
                self.ctx.mul_strided(a, b, n, True, out=out, persistent=persistent)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / self.reps
            shape = self.ctx.launch_shape(n)
        finally:
            self.ctx.set_plan(n, prev)
        meas = Measurement(n, batch, spec, ms, batch / (ms * 1e-3), shape["threads"], shape["smem_bytes"],
                           shape["blocks_per_sm"])
        self._log(meas)
        return meas

    def _log(self, m: Measurement):
        if not self.log_path:
            return
        info = gf2x.plan_info(m.n, m.spec)
        rec = dict(m.__dict__)
        rec.update(ts=time.time(), ops_full=info["ops_full"], top_words=info["top_words"],
                   nleaves=info["nleaves"], launch="persistent" if self.persistent else "cta")
        os.makedirs(os.path.dirname(os.path.abspath(self.log_path)), exist_ok=True)
        with open(self.log_path, "a") as f:
            f.write(json.dumps(rec) + "\n")

    def search(self, n: int, batch: int, specs=None, budget_s: float | None = None) -> list:
        """Measure every candidate (or `specs`); returns measurements sorted fastest first."""
        specs = specs if specs is not None else candidate_specs(n)
        res = []
        t0 = time.time()
        for s in specs:
            if budget_s is not None and time.time() - t0 > budget_s:
                break
            try:
                res.append(self.measure(n, s, batch))
            except gf2x.Gf2xError as e:
                if "plan table full" in str(e):   # a context holds 8192 plans: go on in a fresh one
                    self.renew_context()
                    try:
                        res.append(self.measure(n, s, batch))
                        continue
                    except gf2x.Gf2xError as e2:
                        e = e2
                self.failures.append((n, batch, s, str(e)))
                continue
        res.sort(key=lambda m: m.ms)
        return res


def guided_search(tuner: "Autotuner", n: int, batch: int, model=None, k: int = 10) -> list:
    """Measure only the k candidates the cost model ranks fastest; without a
    model, fall back to exhaustive measured search."""
    cands = candidate_specs(n)
    if model is None:
        return tuner.search(n, batch, cands)
    return tuner.search(n, batch, model.rank(n, batch, cands)[:k])


def best_plans(records: list, sizes, batch: int, allow_split: bool = True) -> dict:
    """Fastest measured plan of every size at the batch bucket nearest `batch`."""
    out = {}
    for n in sizes:
        recs = [r for r in records if r["n"] == n
                and (allow_split or r["spec"].split("/")[5:6] != ["1"])]
        if not recs:
            continue
        near = min(abs(math.log2(r["batch"]) - math.log2(batch)) for r in recs)
        recs = [r for r in recs if abs(math.log2(r["batch"]) - math.log2(batch)) == near]
        out[n] = min(recs, key=lambda r: r["ms"] / r["batch"])["spec"]
    return out


def mixed_plan_sets(records: list, weights: dict, batch: int, top: int = 3) -> list:
    """Candidate plan sets for ONE launch over several sizes, from a timing log.

    A mixed launch needs one leaf size (one kernel) and runs every CTA with
    the largest thread count and shared memory of its plans, so the sets are
    formed per (leaf size, CTA threads): for each size the fastest measured
    plan with that pair, ranked by the count-weighted sum of their times per
    product.  The caller measures the first few as real mixed launches."""
    best = {}   # (n, S, threads) -> (ns per product, spec)
    for r in records:
        if r["n"] not in weights or abs(math.log2(r["batch"]) - math.log2(batch)) > 1.0:
            continue
        fields = r["spec"].split("/")
        if len(fields) > 5 and fields[5] == "1":
            continue    # split plans run through strided launches only
        S = int(r["spec"].split("/")[1])
        key = (r["n"], S, r["threads"])
        ns = r["ms"] * 1e6 / r["batch"]
        if key not in best or ns < best[key][0]:
            best[key] = (ns, r["spec"])
    pairs = {(S, t) for (_, S, t) in best}
    scored = []
    for S, t in pairs:
        if all((n, S, t) in best for n in weights):
            cost = sum(w * best[(n, S, t)][0] for n, w in weights.items())
            scored.append((cost, {n: best[(n, S, t)][1] for n in weights}))
    scored.sort(key=lambda x: x[0])
    return [plans for _, plans in scored[:top]]


def model_mixed_plan_sets(model, weights: dict, batch: int, top: int = 3, cands: dict | None = None) -> list:
    """Candidate plan sets for ONE launch over several sizes, proposed by the
    learned cost model (costmodel.CostModel) instead of measurements: every
    in-CTA candidate of every size is scored by the network, and for each
    (leaf size, CTA threads) pair the set takes each size's best-scored plan;
    sets are ranked by the count-weighted predicted time.  Only the first
    `top` are then measured as real launches."""
    best = {}   # (n, S, threads) -> (predicted ns per product, spec)
    for n in weights:
        specs = [c for c in (cands[n] if cands else candidate_specs(n)) if c.split("/")[5:6] != ["1"]]
        pred = model.predict(n, batch, specs)
        for spec, y in zip(specs, pred):
            info = gf2x.plan_info(n, spec)
            key = (n, info["leaf_words"], info["threads"])
            ns = 2.0 ** float(y)
            if key not in best or ns < best[key][0]:
                best[key] = (ns, spec)
    pairs = {(S, t) for (_, S, t) in best}
    scored = []
    for S, t in pairs:
        if all((n, S, t) in best for n in weights):
            cost = sum(w * best[(n, S, t)][0] for n, w in weights.items())
            scored.append((cost, {n: best[(n, S, t)][1] for n in weights}))
    scored.sort(key=lambda x: x[0])
    return [plans for _, plans in scored[:top]]


PACKAGED_TIMING_LOG = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", "gb300_timing_log.jsonl.gz")
# exhaustive search of one product per launch (batch 1): the single-product plans
PACKAGED_SINGLE_LOG = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans",
                                   "gb300_timing_log_batch1.jsonl.gz")


# top plans of the exhaustive log re-measured in the one-CTA-per-product
# launch form (--launch cta), batches 2048, 4096 and 8192 of the six serving sizes
# and an exhaustive search (split plans included) of 12323 at batch 256
PACKAGED_CTA_LOG = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", "gb300_timing_log_cta.jsonl.gz")


def packaged_cta_log() -> list:
    import gzip
    with gzip.open(PACKAGED_CTA_LOG, "rt") as f:
        return [json.loads(line) for line in f if line.strip()]


def single_product_plans(sizes, one_launch: bool = True) -> dict:
    """Fastest plan for one product per launch of every size, from the batch-1
    timing log; one_launch excludes split plans (three launches)."""
    import gzip
    with gzip.open(PACKAGED_SINGLE_LOG, "rt") as f:
        recs = [json.loads(line) for line in f if line.strip()]
    return best_plans(recs, sizes, 1, allow_split=not one_launch)


def packaged_log() -> list:
    """The GB300 timing log shipped with the package (exhaustive search over six sizes)."""
    import gzip
    with gzip.open(PACKAGED_TIMING_LOG, "rt") as f:
        return [json.loads(line) for line in f if line.strip()]


# ------------------------------------------------------------------ plan database
# Text file read by the C library (gf2x_ctx_load_plan_db): one line
# "n batch_bucket spec ms mults_per_s" per tuned (size, batch bucket).

def batch_bucket(batch: int) -> int:
    """Power-of-two bucket of a batch size (plans are stored per bucket)."""
    return 1 << max(0, int(math.ceil(math.log2(max(1, batch)))))


def load_db(path: str) -> dict:
    """{(n, bucket): {"spec", "ms", "mults_per_s"}}"""
    db = {}
    try:
        with open(path) as f:
            for line in f:
                line = line.split("#", 1)[0].split()
                if len(line) >= 3:
                    rec = {"spec": line[2]}
                    if len(line) >= 5:
                        rec.update(ms=float(line[3]), mults_per_s=float(line[4]))
                    db[(int(line[0]), int(line[1]))] = rec
    except OSError:
        pass
    return db


def save_db(path: str, db: dict, header: str = ""):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write("# gf2x_gb300 plan database: n batch_bucket spec ms_per_launch mults_per_s\n")
        if header:
            f.write(f"# {header}\n")
        for (n, bucket), rec in sorted(db.items()):
            f.write(f"{n} {bucket} {rec['spec']} {rec.get('ms', 0):.4f} {rec.get('mults_per_s', 0):.1f}\n")
    os.replace(tmp, path)


def record_best(db: dict, n: int, batch: int, m: Measurement):
    db[(n, batch_bucket(batch))] = {"spec": m.spec, "ms": m.ms, "mults_per_s": m.mults_per_s}


def read_log(path: str) -> list:
    out = []
    try:
        with open(path) as f:
            for line in f:
                line = line.strip()
                if line:
                    out.append(json.loads(line))
    except OSError:
        pass
    return out


def main(argv=None):
    """python -m paper_2201_10473_gb300.autotune --sizes 17669,35851 --batches 2048 --log L --db D"""
    import argparse
    import random

    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--sizes", default="12323,17669,24659,35851,40973,57637")
    p.add_argument("--batches", default="2048", help="first batch: exhaustive search; others: --sample candidates")
    p.add_argument("--sample", type=int, default=200, help="candidates re-measured at the other batch sizes")
    p.add_argument("--log", required=True)
    p.add_argument("--db", required=True)
    p.add_argument("--budget", type=float, default=None, help="seconds per (size, batch) search")
    p.add_argument("--limit", type=int, default=None)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--from-log", default=None, help="re-measure only the best --top plans of this timing log "
                                                     "('packaged' = the shipped GB300 log)")
    p.add_argument("--top", type=int, default=60)
    p.add_argument("--split-from", type=int, default=24000, help="also try split-top plans from this size on")
    p.add_argument("--launch", choices=["persistent", "cta"], default="persistent",
                   help="launch form timed: a persistent grid (products from a counter) or one CTA per product")
    p.add_argument("--guided", type=int, default=0,
                   help="measure only the K candidates a cost model (trained on the packaged log) ranks first")
    a = p.parse_args(argv)
    model = None
    if a.guided:
        from . import costmodel
        model = costmodel.CostModel(seed=a.seed)
        model.fit(costmodel.training_records(packaged_log()))
    prior = None
    if a.from_log:
        prior = packaged_log() if a.from_log == "packaged" else read_log(a.from_log)
    db = load_db(a.db)
    rng = random.Random(a.seed)
    sizes = [int(x) for x in a.sizes.split(",") if x]
    batches = [int(x) for x in a.batches.split(",") if x]
    for n in sizes:
        ctx = gf2x.Context()          # a fresh plan table per size
        tuner = Autotuner(ctx, a.log, persistent=a.launch == "persistent")
        cands = candidate_specs(n, limit=a.limit, split_from=a.split_from)
        if prior is not None:
            ranked = sorted((r for r in prior if r["n"] == n and r["batch"] == batches[0]), key=lambda r: r["ms"])
            cands = list(dict.fromkeys(r["spec"] for r in ranked))[: a.top] or cands
        if model is not None:
            cands = model.rank(n, batches[0], cands)[: a.guided]
        t0 = time.time()
        res = tuner.search(n, batches[0], cands, a.budget)
        if not res:
            print(f"n={n}: no candidate could be measured", flush=True)
            tuner.ctx.close()
            continue
        record_best(db, n, batches[0], res[0])
        print(f"n={n} batch={batches[0]} measured={len(res)} best={res[0].spec} {res[0].mults_per_s:.4g}/s "
              f"default={gf2x.default_spec(n)} ({time.time() - t0:.0f}s)", flush=True)
        for bsz in batches[1:]:
            sub = [m.spec for m in res[:20]] + rng.sample(cands, min(a.sample, len(cands)))
            r2 = tuner.search(n, bsz, list(dict.fromkeys(sub)), a.budget)
            if not r2:
                print(f"n={n} batch={bsz}: no candidate could be measured", flush=True)
                continue
            record_best(db, n, bsz, r2[0])
            print(f"n={n} batch={bsz} measured={len(r2)} best={r2[0].spec} {r2[0].mults_per_s:.4g}/s", flush=True)
        if tuner.failures:
            print(f"n={n}: {len(tuner.failures)} candidates failed, first: {tuner.failures[0]}", flush=True)
        save_db(a.db, db, header="tuned on " + torch_device_name())
        tuner.ctx.close()


def torch_device_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


if __name__ == "__main__":
    main()
