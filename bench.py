"""Benchmark of the hot path: batched constant-time F2[X] products mod X^n - 1.

Default workload: 4096 products of dense Bernoulli(0.5) polynomials with
n = 17669 coefficients (HQC-128 size), reduced mod X^n - 1, in ONE batched
launch per step (one CTA per product: the block scheduler spreads the
products of a partial last round over the SMs); the persistent form of the
same launch (a grid of resident CTAs taking products from a counter) and
the plain form (one launch per product) are measured beside it.  One JSON
line on stdout (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload hqc128|hqc192|hqc256|c1] [--no-plain]

--impl reference times the oracle (oracle/, plain C on the host cores) on a
bounded sample of the same workload: the only reference this method has.
Multi-GPU (torchrun): every rank multiplies its own 4096 products (weak
scaling, no collective on the data path); time = max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Integer ALU pipe: 64 lanes/clk/SM for LOP3/SHF (32-bit logical ops and
# shifts), 152 SMs, 2070 MHz maximum SM clock: 152 * 64 * 2.07e9 = 20.1 Tops/s.
ALU_LANES_PER_SM = 64
SMS = 152
SM_MAX_MHZ = 2070.0

WORKLOADS = {
    "hqc128": dict(name="hqc128-17669-mulmod", n=17669, batch=4096, reduce=True, key=2),
    "hqc192": dict(name="hqc192-35851-mulmod", n=35851, batch=2048, reduce=True, key=3),
    "hqc256": dict(name="hqc256-57637-mulmod", n=57637, batch=2048, reduce=True, key=4),
    "c1": dict(name="plain-12323-full", n=12323, batch=256, reduce=False, key=1),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="hqc128")
    p.add_argument("--no-plain", action="store_true", help="skip the plain one-launch-per-product measurement")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle cpu_baseline sample")
    p.add_argument("--no-extras", action="store_true", help="skip the other workloads (C1, C3, C4, the three HQC sizes, shared key, unbalanced, sparse, Toom-4, C5)")
    p.add_argument("--serving-requests", type=int, default=200000)
    p.add_argument("--plan", default=None, help="plan spec for the main workload (default: the tuned database)")
    p.add_argument("--only-extra", default=None, choices=sorted(EXTRAS),
                   help="run one of the other workloads alone and print its JSON (for profiling runs)")
    return p.parse_args()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- distributed

def dist_setup():
    from paper_2201_10473_gb300 import shard
    return shard.world_info()


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- oracle legs

def oracle_rate(w: dict, seconds: float, first_product: int = 0) -> dict:
    """The oracle as it stands, on all host cores, over a bounded sample:
    chunks of the workload's products until about `seconds` have passed."""
    import oracle
    n, reduce = w["n"], w["reduce"]
    cores = cpu_cores()
    seed = wl.BASE_SEED + w["key"]
    chunk = min(w["batch"], 4 * cores)
    a, b = wl.dense_pair(seed, n, chunk, first=first_product)
    oracle.mul_batch(a[:cores], b[:cores], n, reduce=reduce, nthreads=cores)      # warm-up
    done = 0
    t0 = time.perf_counter()
    while True:
        oracle.mul_batch(a, b, n, reduce=reduce, nthreads=cores)
        done += chunk
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    # the same oracle on one thread, for the per-core rate
    done1 = 0
    t1 = time.perf_counter()
    while True:
        oracle.mul_batch(a[:1], b[:1], n, reduce=reduce, nthreads=1)
        done1 += 1
        dt1 = time.perf_counter() - t1
        if dt1 >= min(2.0, seconds / 4):
            break
    return {"value": done / dt, "unit": "mults/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} products ({chunk} distinct of the workload, n={n}, seed {seed}) in {dt:.1f} s, "
                      f"oracle_mul_batch on {cores} threads",
            "single_thread_value": done1 / dt1}


def run_reference(args, w):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    # each step: a bounded sample so the whole run stays within minutes
    import oracle
    n, reduce = w["n"], w["reduce"]
    cores = cpu_cores()
    seed = wl.BASE_SEED + w["key"]
    a1, b1 = wl.dense_pair(seed, n, 1)
    t0 = time.perf_counter()
    oracle.mul_batch(a1, b1, n, reduce=reduce, nthreads=1)
    one = max(time.perf_counter() - t0, 1e-4)
    per_step = int(max(cores, min(w["batch"], (120.0 / max(K + W, 1)) * cores / one)))
    a, b = wl.dense_pair(seed, n, per_step)
    for _ in range(W):
        oracle.mul_batch(a, b, n, reduce=reduce, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(K):
        oracle.mul_batch(a, b, n, reduce=reduce, nthreads=cores)
    dt = time.perf_counter() - t0
    value = K * per_step / dt
    line = {"metric": metric_name(), "value": value, "unit": "mults/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": dt / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "impl": "reference",
            "config": config_of(w, None, None),
            "cpu_baseline": {"value": value, "unit": "mults/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} products per step of the workload (n={n}), oracle_mul_batch"},
            "e2e": {"value": value, "unit": "mults/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def metric_name() -> str:
    return "GF(2)[X] mults/sec + ns/mult at n=17669/35851/57637, batched vs plain, bit-exact"


def config_of(w, spec, shape):
    c = {"workload": w["name"], "n": w["n"], "batch_per_gpu": w["batch"], "reduce_mod_xn1": w["reduce"],
         "operands": "dense iid Bernoulli(0.5), SplitMix64 seeded",
         "l2": "8 rotating input sets larger than the 129 MB L2 (no flush)"}
    if spec:
        c["plan"] = spec
    if shape:
        c["launch"] = dict(shape, form="one batched launch, one CTA per product")
    return c


# ---------------------------------------------------------------- our arm

def launches_per_step(info: dict, batch: int) -> int:
    """Kernel launches of one batched call: 1, or 3 per scratch chunk for a
    split plan (evaluation, children, interpolation)."""
    per = info.get("scratch_bytes", 0)
    if not per:
        return 1
    chunk = max(1, min(batch, (256 << 20) // per))
    return 3 * (-(-batch // chunk))


def kernel_source_hash() -> str:
    """Hash of the fused kernel's source: traffic counters apply only to this version."""
    import hashlib
    h = hashlib.sha256()
    for f in ("fused.cuh", "plan.h"):
        with open(os.path.join(ROOT, "paper_2201_10473_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_tc_traffic(n: int, count: int):
    """DRAM bytes of one tensor-core GEMM launch from the committed ncu summary
    (profiles/traffic.txt: "tc-shared-<n>-<count> tc <tc_source_hash> bytes"),
    or None if the kernel changed since the counters were taken."""
    import hashlib
    with open(os.path.join(ROOT, "paper_2201_10473_gb300", "csrc", "tc_circulant.cu"), "rb") as fh:
        h = hashlib.sha256(fh.read()).hexdigest()[:16]
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split("#", 1)[0].split()
                if len(parts) == 4 and parts[0] == f"tc-shared-{n}-{count}" and parts[1] == "tc" and parts[2] == h:
                    return float(parts[3])
    except OSError:
        pass
    return None


def measured_traffic(workload: str, spec: str):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.txt:
    "workload plan kernel_source_hash dram_bytes_per_launch"), or None if the
    kernel or the plan changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split("#", 1)[0].split()
                if len(parts) == 4 and parts[0] == workload and parts[1] == spec and parts[2] == kernel_source_hash():
                    return float(parts[3])
    except OSError:
        pass
    return None



def run_ours(args, w):
    import torch
    import torch.distributed as dist

    from paper_2201_10473_gb300 import Context, plan_info

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n, batch, reduce = w["n"], w["batch"], w["reduce"]
    seed = wl.BASE_SEED + w["key"]
    ctx = Context(local, batch_hint=batch)
    if args.plan:
        ctx.set_plan(n, args.plan)
    spec = ctx.get_plan(n)
    info = plan_info(n, spec)
    shape = ctx.launch_shape(n)

    # input sets: rank r multiplies products r*batch .. (r+1)*batch-1 of the seeded
    # stream (weak scaling); rotate R copies so the inputs touched between two
    # uses exceed L2
    from paper_2201_10473_gb300 import shard
    mine = shard.shard_range(rank, world, batch)
    in_bytes = 2 * batch * wl.limbs(n) * 8
    R = max(2, int(np.ceil(160e6 / in_bytes)))
    host_a, host_b = wl.dense_pair(seed, n, batch, first=mine.start)
    sets = []
    for r in range(R):
        # every set is the same products (identical results); rotating copies defeat L2 reuse
        sets.append((torch.from_numpy(host_a.view(np.int64)).cuda(), torch.from_numpy(host_b.view(np.int64)).cuda()))
    ol = wl.limbs(n) if reduce else (2 * n - 1 + 63) // 64
    out = torch.empty((batch, ol), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def step(i, persistent=False):
        a, b = sets[i % R]
        ctx.mul_strided(a, b, n, reduce, out=out, persistent=persistent, stream=stream)

    # parity spot check of this run's launch configuration before timing
    import_oracle_ok = True
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if rank == 0:
        try:
            import oracle
            sample = np.arange(0, batch, max(1, batch // 16))
            got = out.cpu().numpy().view(np.uint64)[sample]
            exp = oracle.mul_batch(host_a[sample], host_b[sample], n, reduce=reduce)
            if not np.array_equal(got, exp):
                raise SystemExit("bench: GPU results differ from the oracle")
        except ImportError:
            import_oracle_ok = False

    # the spot check left the GPU idle: untimed steps for ~0.2 s bring the
    # clocks back up before the timed region
    t_ramp = time.perf_counter()
    i_ramp = 0
    while time.perf_counter() - t_ramp < 0.2:
        for _ in range(8):
            step(i_ramp)
            i_ramp += 1
        torch.cuda.synchronize()

    # ---- timed region: K steps; per-launch events on the launching stream
    # around every EV_EVERY-th step (a sample of the launch durations: event
    # records between every pair of launches would add their own gaps)
    K = args.steps
    EV_EVERY = 8 if K >= 64 else 1
    evs = {i: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for i in range(0, K, EV_EVERY)}
    clocks = ClockSampler(local)
    clocks.start()
    # untimed steps while the sampler starts, so that the GPU does not idle
    # (and drop its clock) just before the timed region
    t_busy = time.perf_counter()
    while time.perf_counter() - t_busy < 0.3:
        for _ in range(8):
            step(i_ramp)
            i_ramp += 1
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(K):
        ev = evs.get(i)
        if ev:
            ev[0].record(stream)
        step(args.warmup + i)
        if ev:
            ev[1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    clk = clocks.stop()
    launch_ms = [e0.elapsed_time(e1) for e0, e1 in evs.values()]
    total_ms = shard.max_over_ranks(total_ms, device="cuda")
    value = shard.whole_job_rate(batch * K, world, total_ms * 1e-3)

    # ---- end to end through the public API with host buffers
    pin_a = torch.from_numpy(host_a.view(np.int64)).pin_memory()
    pin_b = torch.from_numpy(host_b.view(np.int64)).pin_memory()
    pin_out = torch.empty((batch, ol), dtype=torch.int64).pin_memory()

    def e2e_step():
        # the public host-buffer call: chunked copies in and out overlapped with the products
        ctx.mul_strided_host(pin_a, pin_b, n, reduce, out=pin_out, stream=stream, inputs_ready=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    K2 = max(3, K // 2)
    for _ in range(K2):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = shard.max_over_ranks(e2e_ms, device="cuda")
    got_e2e = pin_out.numpy().view(np.uint64)
    e2e_value = shard.whole_job_rate(batch * K2, world, e2e_ms * 1e-3)
    # the host-buffer results of the last timed call, sampled rows against the oracle
    e2e_ok = None
    if rank == 0 and import_oracle_ok:
        import oracle
        rows = np.unique(np.concatenate([np.arange(0, batch, max(1, batch // 16)), [batch - 1]]))
        e2e_ok = bool(np.array_equal(got_e2e[rows], oracle.mul_batch(host_a[rows], host_b[rows], n, reduce=reduce)))
        if not e2e_ok:
            raise SystemExit("bench: host-buffer (e2e) results differ from the oracle")

    # ---- the persistent form of the batched launch (a grid of resident CTAs
    # taking the products in order from a counter), same inputs and plan
    Kp = max(3, min(K, 400))
    for i in range(3):
        step(i, persistent=True)
    torch.cuda.synchronize()
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for i in range(Kp):
        step(i, persistent=True)
    q1.record(stream)
    torch.cuda.synchronize()
    pers_ms = shard.max_over_ranks(q0.elapsed_time(q1), device="cuda")
    persistent_form = {"mults_per_s": shard.whole_job_rate(batch * Kp, world, pers_ms * 1e-3), "steps": Kp,
                       "grid": int(shape["blocks_per_sm"]) * int(shape["sm_count"]),
                       "order": "CTAs take the products in order from a counter"}
    if rank == 0 and import_oracle_ok:
        import oracle
        sample = np.arange(0, batch, max(1, batch // 16))
        if not np.array_equal(out.cpu().numpy().view(np.uint64)[sample],
                              oracle.mul_batch(host_a[sample], host_b[sample], n, reduce=reduce)):
            raise SystemExit("bench: persistent-launch results differ from the oracle")

    # ---- consecutive steps on two streams without a join between them: the
    # next batch's CTAs start on the SMs that the previous batch's last wave
    # leaves idle (what the host-buffer pipeline does across its chunks and
    # calls); same inputs, plan and launch, each stream its own result buffer
    Ko = max(4, min(K, 400))
    out2 = torch.empty_like(out)
    two = [torch.cuda.Stream(device=local), torch.cuda.Stream(device=local)]

    def overlapped(k):
        a, b = sets[k % R]
        st = two[k % 2]
        ctx.mul_strided(a, b, n, reduce, out=out if k % 2 == 0 else out2, stream=st)

    torch.cuda.synchronize()
    o0 = torch.cuda.Event(enable_timing=True)
    o1 = torch.cuda.Event(enable_timing=True)
    o0.record(stream)
    for st in two:
        st.wait_stream(stream)
    for k in range(Ko):
        overlapped(k)
    for st in two:
        stream.wait_stream(st)
    o1.record(stream)
    torch.cuda.synchronize()
    ov_ms = shard.max_over_ranks(o0.elapsed_time(o1), device="cuda")
    overlapped_form = {"mults_per_s": shard.whole_job_rate(batch * Ko, world, ov_ms * 1e-3), "steps": Ko,
                       "form": "consecutive batches alternate between two streams, one launch of one CTA per "
                               "product each, no join between batches"}
    if rank == 0 and import_oracle_ok:
        import oracle
        sample = np.arange(0, batch, max(1, batch // 16))
        for o in (out, out2):
            if not np.array_equal(o.cpu().numpy().view(np.uint64)[sample],
                                  oracle.mul_batch(host_a[sample], host_b[sample], n, reduce=reduce)):
                raise SystemExit("bench: overlapped-step results differ from the oracle")

    # ---- plain form: one launch of one CTA per product, with the plan tuned
    # for a single product per launch
    plain = None
    if not args.no_plain:
        from paper_2201_10473_gb300 import autotune
        a, b = sets[0]
        outs1 = out
        cp = Context(local, plan_db=None)
        single = autotune.single_product_plans([n]).get(n)
        if single:
            cp.set_plan(n, single)
        for _ in range(2):
            for p in range(batch):
                (cp.mulmod if reduce else cp.mul)(a[p], b[p], n, out=outs1[p], stream=stream)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for p in range(batch):
            (cp.mulmod if reduce else cp.mul)(a[p], b[p], n, out=outs1[p], stream=stream)
        p1.record(stream)
        torch.cuda.synchronize()
        plain_ms = p0.elapsed_time(p1)
        plain = {"value": batch / (plain_ms * 1e-3), "unit": "mults/s", "launches": batch,
                 "plan": cp.get_plan(n),
                 "note": "one launch of one CTA per product, the plan tuned for one product per launch"}
        cp.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the fused kernel (the only kernel of the step)
    mean_launch_ms = float(np.mean(launch_ms))
    ops_per_launch = info["ops_full"] * batch
    achieved = ops_per_launch / (mean_launch_ms * 1e-3) / 1e12
    peak = SMS * ALU_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    traffic = measured_traffic(w["name"], spec)
    observed = clk.get("sm_mhz")
    # the leaf products' useful AND-XORs alone (one 32-bit AND-XOR per 32 bit
    # products: the word products of the plan x 64 x 64 / 32), without the
    # comb's shifts and masks or the evaluation / interpolation passes
    useful = info["nleaves"] * 32 * info["leaf_words"] ** 2
    useful_achieved = useful * batch / (mean_launch_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": traffic,
            "ops_per_product": info["ops_full"], "products_per_launch": batch,
            "useful_leaf_ops_per_product": useful, "useful_leaf_achieved": useful_achieved,
            "frac_useful_leaf_ops": useful_achieved / peak,
            "clmul64_per_product": info["clmul64"],
            # plan-independent context: the schoolbook's n^2 bit products as 32-bit AND-XORs per second
            # (what the recursion saves shows up as a rate above the peak)
            "schoolbook_equivalent_tops": (n * n / 32) * batch / (mean_launch_ms * 1e-3) / 1e12,
            "peak_note": "152 SMs x 64 ALU lanes/clk x 2070 MHz (unit counts and max clock)",
            "launch_time": f"mean of {len(launch_ms)} launches timed by CUDA events in the timed region "
                           f"(every {EV_EVERY}th step)",
            "frac_at_observed_clock": (achieved / (SMS * ALU_LANES_PER_SM * observed * 1e6 / 1e12)) if observed else None,
            "hbm_gbs": (info["bytes_in"] + (info["bytes_out_reduced"] if reduce else info["bytes_out_full"])) * batch
            / (mean_launch_ms * 1e-3) / 1e9}

    cpu = None
    if world == 1:
        cpu = oracle_rate(w, args.cpu_seconds)
    extras = None
    if world == 1 and not args.no_extras:
        extras = run_extras(args, local)

    line = {
        "metric": metric_name(),
        "value": value,
        "unit": "mults/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": total_ms / K,
        "ns_per_mult": 1e9 / value,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": config_of(w, spec, shape),
        "e2e": {"value": e2e_value, "unit": "mults/s", "h2d_bytes_per_step": int(pin_a.numel() * 8 * 2),
                "d2h_bytes_per_step": int(pin_out.numel() * 8), "steps": K2},
        "gpu_launches": K * launches_per_step(info, batch),
        "roofline": roof,
        "cpu_baseline": cpu,
        "persistent_launch": persistent_form,
        "overlapped_steps": overlapped_form,
        "plain": plain,
        "batched_over_plain": (value / world / plain["value"]) if plain else None,
        "clocks": clk,
        "parity_checked": import_oracle_ok,
        "e2e_sample_checked_against_oracle": e2e_ok,
        "workloads": extras,
        "paper_context": {"note": "the paper's own CPU figures (unreduced product, one core), context only",
                          "hw": "Intel Core i7-1165G7 (Tiger Lake) 2.8 GHz, Turbo off, one thread",
                          "hqc128_17669_avx512_cycles": 14872, "hqc128_17669_avx512_mults_per_s": 2.8e9 / 14872,
                          "hqc256_57637_avx512_cycles": 110568},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- the other workloads

def _time_calls(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint64).view(np.int64)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint64)


def run_c1(device):
    """256 full products at n=12323, one plain launch per product, all checked."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context
    from paper_2201_10473_gb300 import autotune
    n, count = 12323, 256
    ctx = Context(device, batch_hint=count)
    cp = Context(device, plan_db=None)            # the plan tuned for one product per launch
    single = autotune.single_product_plans([n]).get(n)
    if single:
        cp.set_plan(n, single)
    a, b = wl.dense_pair(wl.BASE_SEED + 1, n, count)
    da, db = _dev(a), _dev(b)
    out = torch.empty((count, (2 * n - 1 + 63) // 64), dtype=torch.int64, device="cuda")

    def plain():
        for p in range(count):
            cp.mul(da[p], db[p], n, out=out[p])
    ms = _time_calls(plain, 3, 1)
    ok = bool(np.array_equal(_host(out), oracle.mul_batch(a, b, n, reduce=False)))
    out.zero_()
    ms_b = _time_calls(lambda: ctx.mul_strided(da, db, n, False, out=out), 10, 3)
    ok &= bool(np.array_equal(_host(out), oracle.mul_batch(a, b, n, reduce=False)))
    plain_plan = cp.get_plan(n)
    ctx.close()
    cp.close()
    return {"workload": "plain-12323-full", "n": n, "products": count, "plan": ctx_plan_text(n, count),
            "plain_plan": plain_plan,
            "plain_mults_per_s": count / (ms * 1e-3), "batched_mults_per_s": count / (ms_b * 1e-3),
            "all_checked_against_oracle": ok}


def ctx_plan_text(n, batch):
    from paper_2201_10473_gb300 import Context
    c = Context(batch_hint=batch)
    t = c.get_plan(n)
    c.close()
    return t


def run_c3(device):
    """2048@17669 + 1024@35851 + 512@57637 interleaved, ONE persistent launch
    over device items replayed from a CUDA graph, vs plain and per-size launches."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context, autotune, pack_items, serve
    wk = wl.workload(3)
    sizes = np.array(wk.sizes)
    weights = {n: int((sizes == n).sum()) for n in np.unique(sizes)}
    reqs = serve.make_requests(sizes, lambda n, c: wl.dense_pair(wk.seed + n, n, c))
    outs = {n: torch.zeros((cnt, wl.limbs(n)), dtype=torch.int64, device="cuda") for n, cnt in weights.items()}
    pa, pb = reqs.ptrs(np.arange(len(sizes)))
    po = np.array([outs[int(n)].data_ptr() + int(i) * 8 * wl.limbs(int(n)) for n, i in zip(sizes, reqs.index)])
    items = pack_items(list(zip(pa, pb, po, sizes, [1] * len(sizes)))).cuda()
    # the same items largest first: a persistent CTA takes items i, i + grid, ...,
    # so a sorted list hands every CTA one item of each size band in turn
    by_size = np.argsort(-sizes, kind="stable")
    items_lf = items[torch.from_numpy(by_size).cuda()].contiguous()
    log = autotune.packaged_log()

    def time_mixed(plans):
        """One graph-replayed launch over the device items: persistent as
        interleaved (static stride), largest first (static stride), largest
        first with CTAs taking items from a counter (dynamic); and one CTA
        per item, largest first."""
        ctx = Context(device, plan_db=None)
        for n, sp in plans.items():
            ctx.set_plan(int(n), sp)
        ctx.prepare(sorted(int(n) for n in weights))
        stream = torch.cuda.Stream()
        res = []
        for its, pers, dyn in ((items, True, False), (items_lf, True, False), (items_lf, True, True),
                               (items_lf, False, False)):
            with torch.cuda.stream(stream):
                ctx.mul_batched_device(its, len(sizes), persistent=pers, dynamic=dyn)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                ctx.mul_batched_device(its, len(sizes), persistent=pers, dynamic=dyn)
            res.append(_time_calls(g.replay, 10, 3))
        ctx.sync_status()
        ctx.close()
        return res

    # plan sets: (i) from the exhaustive measured log, (ii) proposed by the
    # learned cost model trained on that log; the measured best of (i)
    # judges the regret of (ii)
    from paper_2201_10473_gb300 import costmodel
    measured_sets = autotune.mixed_plan_sets(log, weights, 2048, top=3)
    model = costmodel.CostModel(seed=0)
    model.fit(costmodel.training_records(log), steps=3000, seed=0)
    model_top = 10   # as many as the per-size guided search measures
    model_sets = autotune.model_mixed_plan_sets(model, weights, 2048, top=model_top)
    timed = []
    for origin, sets in (("log", measured_sets), ("model", model_sets)):
        for plans in sets:
            t = time_mixed(plans)
            timed.append((min(t), origin, plans, t))
    best_log = min((x for x in timed if x[1] == "log"), key=lambda x: x[0])
    best_model = min((x for x in timed if x[1] == "model"), key=lambda x: x[0])
    _, _, plans, (ms, ms_lf, ms_dyn, ms_cta) = min(timed, key=lambda x: x[0])
    model_regret = best_model[0] / best_log[0] - 1.0
    best = (ms, plans, min(ms_lf, ms_dyn))
    ms, plans, ms_lf = best
    dyn_best = ms_dyn <= ms_lf
    # recompute with the best set and check a sample against the oracle
    ctx = Context(device, plan_db=None)
    for n, sp in plans.items():
        ctx.set_plan(int(n), sp)
    ctx.prepare(sorted(int(n) for n in weights))
    for o in outs.values():
        o.zero_()
    ctx.mul_batched_device(items_lf, len(sizes), persistent=True, dynamic=dyn_best)
    torch.cuda.synchronize()
    ok = True
    for r in range(0, len(sizes), 149):
        n, i = int(sizes[r]), int(reqs.index[r])
        got = _host(outs[n][i])
        ok &= bool(np.array_equal(got, oracle.mulmod(_host(reqs.a[n][i]), _host(reqs.b[n][i]), n)))
    # plain: one launch of one CTA per product, the single-product plans
    cp = Context(device, plan_db=None)
    for n, sp in autotune.single_product_plans([int(x) for x in weights]).items():
        cp.set_plan(int(n), sp)

    def plain():
        for r in range(len(sizes)):
            n, i = int(sizes[r]), int(reqs.index[r])
            cp.mulmod(reqs.a[n][i], reqs.b[n][i], n, out=outs[n][i])
    ms_plain = _time_calls(plain, 1, 1)
    cp.close()
    ctx.close()
    # per-size launches with each size's own tuned plan, one after the other
    # (one CTA per product)
    ctx2 = Context(device, batch_hint=2048)

    def grouped():
        for n in weights:
            ctx2.mul_strided(reqs.a[int(n)], reqs.b[int(n)], int(n), True, out=outs[int(n)])
    ms_grouped = _time_calls(grouped, 10, 3)
    ctx2.close()
    # ONE graph launch: the per-size tuned kernels (split plans included) on
    # forked streams, largest n first, so that the sizes overlap on the GPU;
    # one context per size keeps the split scratch of each on its own
    # stream.  One CTA per product lets the block scheduler interleave the
    # three kernels' CTAs; persistent grids each fill the GPU, so the later
    # kernels mostly run in the first one's tail.
    sizes_n = sorted((int(n) for n in weights), reverse=True)

    def forked_graph(persistent):
        ctxs = {n: Context(device, batch_hint=2048) for n in sizes_n}
        branch = {n: torch.cuda.Stream() for n in sizes_n}
        root = torch.cuda.Stream()
        for n in sizes_n:                         # warm-up on the streams the graph will use
            with torch.cuda.stream(branch[n]):
                ctxs[n].mul_strided(reqs.a[n], reqs.b[n], n, True, out=outs[n], persistent=persistent)
        torch.cuda.synchronize()
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2, stream=root):
            fork = torch.cuda.Event()
            fork.record(root)
            for n in sizes_n:
                branch[n].wait_event(fork)
                with torch.cuda.stream(branch[n]):
                    ctxs[n].mul_strided(reqs.a[n], reqs.b[n], n, True, out=outs[n], persistent=persistent)
            for n in sizes_n:
                root.wait_stream(branch[n])
        for o in outs.values():
            o.zero_()
        ms_g = min(_time_calls(g2.replay, 10, 3) for _ in range(2))
        ok_g = True
        for r in range(0, len(sizes), 149):
            n, i = int(sizes[r]), int(reqs.index[r])
            ok_g &= bool(np.array_equal(_host(outs[n][i]), oracle.mulmod(_host(reqs.a[n][i]), _host(reqs.b[n][i]), n)))
        for c in ctxs.values():
            c.close()
        return ms_g, ok_g
    ms_graph_p, ok_graph_p = forked_graph(True)
    ms_graph, ok_graph = forked_graph(False)
    total = len(sizes)
    return {"workload": wk.name, "products": total, "plans": {str(k): v for k, v in plans.items()},
            "one_launch_graph_mults_per_s": total / (ms * 1e-3),
            "one_launch_graph_largest_first_mults_per_s": total / (ms_lf * 1e-3),
            "one_launch_graph_one_cta_per_item_mults_per_s": total / (ms_cta * 1e-3),
            "one_launch_schedule": "largest first, items from a counter" if dyn_best else "largest first, static stride",
            "plan_sets_timed": [{"origin": o, "plans": {str(k): v for k, v in p.items()},
                                 "interleaved_ms": t[0], "largest_first_ms": t[1], "largest_first_dynamic_ms": t[2],
                                 "one_cta_per_item_ms": t[3]}
                                for _, o, p, t in timed],
            "model_proposed_best_mults_per_s": total / (best_model[0] * 1e-3),
            "log_best_mults_per_s": total / (best_log[0] * 1e-3),
            "model_regret_vs_measured_log": model_regret,
            "model_sets_measured": model_top,
            "plain_mults_per_s": total / (ms_plain * 1e-3),
            "per_size_launches_mults_per_s": total / (ms_grouped * 1e-3),
            "one_graph_concurrent_per_size_kernels_mults_per_s": total / (ms_graph * 1e-3),
            "one_graph_form": "forked streams, largest n first, one CTA per product",
            "one_graph_persistent_kernels_mults_per_s": total / (ms_graph_p * 1e-3),
            "graph_plans": {str(n): ctx_plan_text(n, 2048) for n in sizes_n},
            "sample_checked_against_oracle": ok and ok_graph and ok_graph_p}


def run_c4(device):
    """16384 products at n=57637: dense, and sparse (weight 131) x dense through
    the same path and through the sparse x dense kernel (positions)."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context
    n, count = 57637, 16384
    ctx = Context(device, batch_hint=count)
    wk = wl.workload(4)
    a, b = wl.dense_pair(wk.seed, n, count)
    bs = wl.sparse_operands(wk.seed, n, 131, count)
    da, db, dbs = _dev(a), _dev(b), _dev(bs)
    out = torch.empty((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
    ms_dense = _time_calls(lambda: ctx.mul_strided(da, db, n, True, out=out), 5, 2)
    sample = np.arange(0, count, 2048)
    ok = bool(np.array_equal(_host(out)[sample], oracle.mul_batch(a[sample], b[sample], n, reduce=True)))
    ms_sparse = _time_calls(lambda: ctx.mul_strided(da, dbs, n, True, out=out), 5, 2)
    ok &= bool(np.array_equal(_host(out)[sample], oracle.mul_batch(a[sample], bs[sample], n, reduce=True)))
    # the same sparse operands given by their 131 positions, through the
    # constant-time sparse x dense kernel
    pos = np.stack([np.flatnonzero(np.unpackbits(r.view(np.uint8), bitorder="little"))[:131] for r in bs])
    dpos = torch.from_numpy(pos.astype(np.int32)).cuda()
    out.zero_()
    ms_kernel = _time_calls(lambda: ctx.mulmod_sparse(da, dpos, n, out=out), 5, 2)
    ok &= bool(np.array_equal(_host(out)[sample], oracle.mul_batch(a[sample], bs[sample], n, reduce=True)))
    plan = ctx.get_plan(n)
    ctx.close()
    return {"workload": wk.name, "products": count, "plan": plan,
            "dense_mults_per_s": count / (ms_dense * 1e-3), "sparse131_mults_per_s": count / (ms_sparse * 1e-3),
            "sparse_over_dense_time": ms_sparse / ms_dense,
            "sparse131_positions_kernel_mults_per_s": count / (ms_kernel * 1e-3),
            "note": "dense path: the sparse operand goes through the dense constant-time path (same work, same "
                    "time); positions kernel: gf2x_mulmod_sparse on the same operands",
            "launch": "one CTA per product",
            "sample_checked_against_oracle": ok}


def run_hqc_sizes(device):
    """The three HQC sizes of the metric (17669, 35851, 57637 mod X^n - 1):
    the batched launch (tuned plan, one CTA per product; 4096, 2048 and 2048
    products, rotating copies of the inputs that together exceed L2) against
    one plain launch per product with the single-product plan (256
    launches)."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context, autotune
    res = {"workload": "hqc-sizes-mulmod"}
    for key, n, count in ((2, 17669, 4096), (3, 35851, 2048), (4, 57637, 2048)):
        ctx = Context(device, batch_hint=count)
        cp = Context(device, plan_db=None)
        single = autotune.single_product_plans([n]).get(n)
        if single:
            cp.set_plan(n, single)
        a, b = wl.dense_pair(wl.BASE_SEED + key, n, count)
        R = max(2, int(np.ceil(160e6 / (2 * a.nbytes))))
        sets = [(_dev(a), _dev(b)) for _ in range(R)]
        out = torch.empty((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
        it = [0]

        def batched():
            da, db = sets[it[0] % R]
            it[0] += 1
            ctx.mul_strided(da, db, n, True, out=out)
        ms_b = _time_calls(batched, 20, 3)
        s = np.arange(0, count, count // 8)
        ok = bool(np.array_equal(_host(out)[s], oracle.mul_batch(a[s], b[s], n, reduce=True)))
        m = 256
        da, db = sets[0]

        def plain():
            for p in range(m):
                cp.mulmod(da[p], db[p], n, out=out[p])
        out.zero_()
        ms_p = _time_calls(plain, 2, 1)
        ok &= bool(np.array_equal(_host(out)[:m:37], oracle.mul_batch(a[:m:37], b[:m:37], n, reduce=True)))
        res[f"n{n}"] = {"products": count, "plan": ctx.get_plan(n), "mults_per_s": count / (ms_b * 1e-3),
                        "ns_per_mult": ms_b * 1e6 / count, "plain_plan": cp.get_plan(n),
                        "plain_mults_per_s": m / (ms_p * 1e-3), "batched_over_plain": (count / ms_b) / (m / ms_p),
                        "sample_checked_against_oracle": ok}
        ctx.close()
        cp.close()
    return res


def run_shared(device):
    """One public key h times many vectors at n = 17669 (reduced mod X^n - 1),
    shared-operand launch against the unshared launch with h copied into every
    row (one CTA per product) and the tensor-core circulant GEMM; 4096
    products per launch, 8 rotating input sets (> L2)."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context
    n, count, R = 17669, 4096, 8
    ctx = Context(device, batch_hint=count)
    h = wl.dense_operands(wl.BASE_SEED + 8, n, 1, 0)
    vecs = [wl.dense_operands(wl.BASE_SEED + 8, n, count, 1, first=r * count) for r in range(R)]
    dh, dhs = _dev(h[0]), _dev(np.repeat(h, count, axis=0))
    dv = [_dev(v) for v in vecs]
    out = torch.empty((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
    it = [0]

    def call(a_of):
        r = it[0] % R
        it[0] += 1
        ctx.mul_strided(a_of(r), dv[r], n, True, out=out)
    def call_tc():
        r = it[0] % R
        it[0] += 1
        ctx.mulmod_shared_tc(dh, dv[r], n, out=out)
    rates = {}
    ms_tc = []
    for rep in range(3):        # interleaved: shared, unshared, tensor cores, shared, ...
        for name, a_of in (("shared", lambda r: dh), ("unshared", lambda r: dhs)):
            it[0] = 0
            ms = _time_calls(lambda: call(a_of), 40, 3)
            rates.setdefault(name, []).append(count / (ms * 1e-3))
        it[0] = 0
        ms_tc.append(_time_calls(call_tc, 40, 3))
    # the HQC encapsulation shape: the shared key times secret vectors of
    # weight 75, on the tensor cores and through the constant-time sparse
    # kernel (positions; the key repeated in every row)
    sp_rows = wl.sparse_operands(wl.BASE_SEED + 12, n, 75, count)
    sp_pos = np.stack([np.flatnonzero(np.unpackbits(r.view(np.uint8), bitorder="little"))[:75] for r in sp_rows])
    dsp, dpos = _dev(sp_rows), torch.from_numpy(sp_pos.astype(np.int32)).cuda()
    ms_tc_sparse = _time_calls(lambda: ctx.mulmod_shared_tc(dh, dsp, n, out=out), 40, 3)
    ms_sparse_kernel = _time_calls(lambda: ctx.mulmod_sparse(dhs, dpos, n, out=out), 40, 3)
    ok_sp = bool(np.array_equal(_host(out)[::512], np.stack([oracle.mulmod(h[0], sp_rows[p], n)
                                                             for p in range(0, count, 512)])))
    sample = np.arange(0, count, 512)
    exp = np.stack([oracle.mulmod(h[0], vecs[0][p], n) for p in sample])
    it[0] = 0
    call(lambda r: dh)
    ok = bool(np.array_equal(_host(out)[sample], exp))
    it[0] = 0
    out.zero_()
    call_tc()
    ok_tc = bool(np.array_equal(_host(out)[sample], exp))
    ctx.sync_status()
    plan = ctx.get_plan(n)
    ctx.close()
    shared, unshared = max(rates["shared"]), max(rates["unshared"])
    ms = min(ms_tc)
    # roofline of the tensor-core call: the n^2 multiply-adds of each product
    # (2 n^2 flops), over the whole call (its GEMM kernel is ~91% of it in the
    # ncu launch list), against the fp4 dense peak taken as the measured bf16
    # burst x the nominal fp4/bf16 ratio (13.5 / 2.25 = 6)
    flops = 2.0 * n * n * count
    peak = None
    try:
        with open(PEAKS_FILE) as f:
            peak = json.load(f)["bf16_tflops"] * 6.0
    except (OSError, KeyError, ValueError):
        peak = 1900.0 * 6.0
    achieved = flops / (ms * 1e-3) / 1e12
    return {"workload": "shared-key-17669-mulmod", "products": count, "plan": plan,
            "shared_mults_per_s": shared, "unshared_mults_per_s": unshared, "shared_over_unshared": shared / unshared,
            "tensor_core_mults_per_s": count / (ms * 1e-3), "tensor_over_shared_comb": count / (ms * 1e-3) / shared,
            "hqc_encaps_shape_weight75": {"tensor_core_mults_per_s": count / (ms_tc_sparse * 1e-3),
                                          "sparse_kernel_mults_per_s": count / (ms_sparse_kernel * 1e-3),
                                          "sample_checked_against_oracle": ok_sp},
            "tensor_core_roofline": {"bound": "tensor", "dtype": "fp4 e2m1 (0/1), fp32 counts", "achieved": achieved,
                                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                                     "peak_note": "MEASURED_PEAKS bf16_tflops x 6 (nominal fp4/bf16); whole call timed",
                                     "traffic": measured_tc_traffic(n, count)},
            "note": "one a for every product: GF2X_BATCH_SHARED_A on the comb path (ALU-bound: sharing saves memory "
                    "reads, not time), and gf2x_mulmod_shared_tc, the circulant GEMM on the tensor cores",
            "sample_checked_against_oracle": ok and ok_tc}


def run_unbalanced(device):
    """2048 full products of a 57637-bit a and a 17669-bit b through the
    unbalanced entry (four 17728-bit chunk products and an overlap-add, as
    the op model picks), against the equal-size 57637 product of the
    zero-extended b (one CTA per product); 4 rotating input sets (> L2)."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context
    na, nb, count, R = 57637, 17669, 2048, 4
    ctx = Context(device, batch_hint=count)
    la, lb, lu = wl.limbs(na), wl.limbs(nb), (na + nb - 1 + 63) // 64
    sets = []
    for r in range(R):
        a = wl.dense_operands(wl.BASE_SEED + 9, na, count, 0, first=r * count)
        b = wl.dense_operands(wl.BASE_SEED + 9, nb, count, 1, first=r * count)
        bz = np.zeros((count, la), np.uint64)
        bz[:, :lb] = b
        sets.append((a, b, _dev(a), _dev(b), _dev(bz)))
    out = torch.empty((count, lu), dtype=torch.int64, device="cuda")
    full = torch.empty((count, (2 * na - 1 + 63) // 64), dtype=torch.int64, device="cuda")
    it = [0]

    def unbalanced():
        _, _, da, db, _ = sets[it[0] % R]
        it[0] += 1
        ctx.mul_unbalanced(da, na, db, nb, out=out)

    def padded():
        _, _, da, _, dbz = sets[it[0] % R]
        it[0] += 1
        ctx.mul_strided(da, dbz, na, False, out=full)
    rates = {}
    for rep in range(2):
        for name, fn in (("unbalanced", unbalanced), ("padded", padded)):
            it[0] = 0
            ms = _time_calls(fn, 8, 3)
            rates.setdefault(name, []).append(count / (ms * 1e-3))
    it[0] = 0
    unbalanced()
    a, b = sets[0][0], sets[0][1]
    got = _host(out)
    ok = True
    for p in range(0, count, 512):
        bz = np.zeros(la, np.uint64)
        bz[:lb] = b[p]
        ok &= bool(np.array_equal(got[p], oracle.mul(a[p], bz, na)[:lu]))
    ctx.close()
    u, pz = max(rates["unbalanced"]), max(rates["padded"])
    return {"workload": "unbalanced-57637x17669-full", "products": count,
            "unbalanced_mults_per_s": u, "padded_equal_size_mults_per_s": pz, "speedup": u / pz,
            "sample_checked_against_oracle": ok}


def run_sparse(device):
    """Constant-time sparse x dense products mod X^n - 1 (HQC shapes: n =
    17669 with weight 75, n = 57637 with weight 131) against the dense path
    on the same operands (the sparse operand expanded to n bits; one CTA per
    product)."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context
    res = {}
    for n, w, count in ((17669, 75, 4096), (57637, 131, 2048)):
        ctx = Context(device, batch_hint=count)
        rows = wl.sparse_operands(wl.BASE_SEED + 10, n, w, count)
        pos = np.stack([np.flatnonzero(np.unpackbits(r.view(np.uint8), bitorder="little"))[:w] for r in rows])
        R = 16 if n < 40000 else 10     # rotating a sets: more than the 129 MB L2 in all
        da = [_dev(wl.dense_operands(wl.BASE_SEED + 10, n, count, 0, first=r * count)) for r in range(R)]
        dpos, dden = torch.from_numpy(pos.astype(np.int32)).cuda(), _dev(rows)
        out = torch.empty((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
        it = [0]

        def sparse():
            ctx.mulmod_sparse(da[it[0] % R], dpos, n, out=out)
            it[0] += 1

        def dense():
            ctx.mul_strided(da[it[0] % R], dden, n, True, out=out)
            it[0] += 1
        rates = {}
        for rep in range(2):
            for name, fn in (("sparse", sparse), ("dense", dense)):
                it[0] = 0
                ms = _time_calls(fn, 10, 3)
                rates.setdefault(name, []).append(count / (ms * 1e-3))
        it[0] = 0
        sparse()
        a0 = _host(da[0])
        got = _host(out)
        ok = all(np.array_equal(got[p], oracle.mulmod(a0[p], rows[p], n)) for p in range(0, count, 512))
        ctx.close()
        sp, de = max(rates["sparse"]), max(rates["dense"])
        res[f"n{n}_w{w}"] = {"products": count, "sparse_mults_per_s": sp, "dense_path_mults_per_s": de,
                             "sparse_over_dense": sp / de, "sample_checked_against_oracle": ok}
    res["workload"] = "hqc-sparse-times-dense-mulmod"
    return res


def run_toom4(device):
    """Toom-4 and Toom-5 top levels against the regular path (the tuned or
    default plan, one CTA per product) at 57637, 100000 and 131072 bits, 512 products mod X^n - 1
    each."""
    import torch

    import oracle
    from paper_2201_10473_gb300 import Context
    res = {"workload": "toom4-toom5-top-level-mulmod"}
    for n in (57637, 100000, 131072):
        count = 512
        ctx = Context(device, batch_hint=count)
        a, b = wl.dense_pair(wl.BASE_SEED + 11, n, count)
        da, db = _dev(a), _dev(b)
        out = torch.empty((count, wl.limbs(n)), dtype=torch.int64, device="cuda")
        rates = {}
        for rep in range(2):
            for name, fn in (("toom4", lambda: ctx.mul_toom4(da, db, n, True, out=out)),
                             ("toom5", lambda: ctx.mul_toom5(da, db, n, True, out=out)),
                             ("regular", lambda: ctx.mul_strided(da, db, n, True, out=out))):
                ms = _time_calls(fn, 5, 2)
                rates.setdefault(name, []).append(count / (ms * 1e-3))
        ok = True
        for fn in (ctx.mul_toom4, ctx.mul_toom5):
            fn(da, db, n, True, out=out)
            got = _host(out)
            ok &= all(np.array_equal(got[p], oracle.mulmod(a[p], b[p], n)) for p in (0, count - 1))
        plan = ctx.get_plan(n)
        ctx.close()
        t4, t5, rg = max(rates["toom4"]), max(rates["toom5"]), max(rates["regular"])
        res[f"n{n}"] = {"products": count, "toom4_mults_per_s": t4, "toom5_mults_per_s": t5,
                        "regular_mults_per_s": rg, "toom4_over_regular": t4 / rg, "toom5_over_regular": t5 / rg,
                        "regular_plan": plan, "sample_checked_against_oracle": ok}
    return res


def run_c5(device, requests):
    """Serving: Poisson arrivals, HBM-budget admission, continuous batching."""
    import torch  # noqa: F401

    from paper_2201_10473_gb300 import Context, autotune, serve
    wk = wl.workload(5)
    sizes = np.array(wk.sizes[:requests])
    distinct = 4096
    sub = {}

    def operands(n, c):
        if n not in sub:
            sub[n] = wl.dense_pair(wk.seed + n, n, min(c, distinct))
        a, b = sub[n]
        reps = -(-c // a.shape[0])
        return np.tile(a, (reps, 1))[:c], np.tile(b, (reps, 1))[:c]
    reqs = serve.make_requests(sizes, operands)
    weights = {int(n): 1 for n in wl.SERVING_SIZES}
    plans = autotune.mixed_plan_sets(autotune.packaged_log(), weights, 2048, top=1)[0]
    ctx = Context(device, plan_db=None)
    for n, sp in plans.items():
        ctx.set_plan(n, sp)
    budget = 64 << 20
    srv = serve.Server(ctx, weights, budget, max_batch=2048, streams=3, use_graphs=True)
    closed = srv.run(reqs, np.zeros(len(sizes)))
    cap = closed.completed / closed.wall_s
    out = {"workload": wk.name, "requests": len(sizes), "budget_bytes": budget,
           "budget_covers": "request slots (both operands, copied in on admission, and the result) and the "
                            "servers' item and copy lists; device-item launches use no other scratch",
           "plans": {str(k): v for k, v in plans.items()},
           "closed_loop": closed.summary(), "loads": {}}
    for f in (0.5, 0.8, 0.95, 1.2):
        arr = wl.poisson_arrivals(wk.seed + int(f * 100), len(sizes), f * cap)
        r = srv.run(reqs, arr)
        out["loads"][str(f)] = dict(r.summary(), offered_per_s=f * cap)
    # size-aware server: one queue, tuned plan and stream pair per size, so
    # that sizes overlap on the GPU, each with its own plan's shape
    sa_plans = autotune.best_plans(autotune.packaged_log(), list(weights), 512, allow_split=False)
    sa = serve.SizeAwareServer(sa_plans, budget, max_batch=2048, streams_per_size=2, device=device)
    sa_closed = sa.run(reqs, np.zeros(len(sizes)))
    sa_cap = sa_closed.completed / sa_closed.wall_s
    out["size_aware"] = {"plans": {str(k): v for k, v in sa_plans.items()}, "closed_loop": sa_closed.summary(),
                         "loads": {}}
    for f in (0.5, 0.8, 0.95, 1.2):
        arr = wl.poisson_arrivals(wk.seed + 200 + int(f * 100), len(sizes), f * sa_cap)
        r = sa.run(reqs, arr)
        out["size_aware"]["loads"][str(f)] = dict(r.summary(), offered_per_s=f * sa_cap)
    for c in sa.ctx.values():
        c.sync_status()
    sa.close()
    # the same server with a 1 GiB output budget: batches are bounded by max_batch, not by slots
    big = serve.SizeAwareServer(sa_plans, 1 << 30, max_batch=2048, streams_per_size=2, device=device)
    big_closed = big.run(reqs, np.zeros(len(sizes)))
    big_cap = big_closed.completed / big_closed.wall_s
    arr = wl.poisson_arrivals(wk.seed + 395, len(sizes), 0.95 * big_cap)
    r = big.run(reqs, arr)
    out["size_aware_1GiB"] = {"closed_loop": big_closed.summary(),
                              "load_0.95": dict(r.summary(), offered_per_s=0.95 * big_cap)}
    for c in big.ctx.values():
        c.sync_status()
    big.close()
    # a tight budget (4 MiB of output slots): admission has to wait for retirements
    tight = serve.Server(ctx, weights, 4 << 20, max_batch=2048, streams=3, use_graphs=True)
    arr = wl.poisson_arrivals(wk.seed + 95, len(sizes), 0.95 * cap)
    r = tight.run(reqs, arr)
    out["tight_budget_4MiB_load_0.95"] = dict(r.summary(), offered_per_s=0.95 * cap,
                                            slots=sum(tight.pool.capacity.values()))
    ctx.sync_status()
    # plain per-request launches (one launch each, holding a request slot), every request
    m = len(sizes)
    sub_reqs = serve.RequestSet(reqs.sizes[:m], reqs.index[:m], reqs.a, reqs.b)
    pool = serve.SlotPool(weights, budget)
    # (the single-product plans, tuned for one launch at a time, serve three
    # concurrent streams of launches more slowly than these plans: 22.5 k/s)
    pc = serve.serve_plain(ctx, sub_reqs, np.zeros(m), pool, streams=3)
    pcap = pc.completed / pc.wall_s
    arr = wl.poisson_arrivals(wk.seed + 7, m, 0.8 * pcap)
    pl = serve.serve_plain(ctx, sub_reqs, arr, pool, streams=3)
    out["plain"] = {"requests": m, "closed_loop": pc.summary(), "load_0.8": dict(pl.summary(), offered_per_s=0.8 * pcap)}
    ctx.close()
    return out


EXTRAS = ("c1", "c3", "c4", "hqc_sizes", "shared_key", "unbalanced", "sparse_ct", "toom4", "c5")


def run_extras(args, device, only=None):
    res = {}
    for name, fn in (("c1", lambda: run_c1(device)), ("c3", lambda: run_c3(device)), ("c4", lambda: run_c4(device)),
                     ("hqc_sizes", lambda: run_hqc_sizes(device)),
                     ("shared_key", lambda: run_shared(device)), ("unbalanced", lambda: run_unbalanced(device)),
                     ("sparse_ct", lambda: run_sparse(device)), ("toom4", lambda: run_toom4(device)),
                     ("c5", lambda: run_c5(device, args.serving_requests))):
        if only and name != only:
            continue
        t0 = time.time()
        try:
            res[name] = fn()
        except Exception as e:  # report, keep the main line
            res[name] = {"error": f"{type(e).__name__}: {e}"}
        res[name]["seconds"] = round(time.time() - t0, 1)
    return res


def main():
    args = parse()
    w = WORKLOADS[args.workload]
    if args.only_extra:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_extras(args, 0, only=args.only_extra)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
