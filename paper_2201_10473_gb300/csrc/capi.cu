// capi.cu -- the C ABI of include/gf2x_gb300.h: contexts, plan tables,
// argument checks and kernel launches.  Compute happens only in the CUDA
// kernels; there is no host fallback.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gf2x_gb300.h"
#include "launchers.h"
#include "plan.h"
#include "plan_host.h"

using namespace gf2x;

namespace {

constexpr uint32_t kPlanCapacity = 8192;  // distinct (n, spec) plans per context
constexpr int kRing = 4;                  // item staging buffers

struct PlanEntry {
    uint32_t slot;
    gf2x_plan_spec spec;
};

constexpr uint64_t kWorkspaceCap = 256ull << 20;  // split plans run in chunks of at most this much scratch
constexpr size_t kFixedStagingItems = 16384;      // item staging per ring buffer in a fixed-workspace context
// Work counters of dynamic launches: a ring for launches made outside a
// stream capture (a slot is reused only after the event recorded behind its
// last launch), and slots that a captured launch keeps for the graph's
// lifetime (never reused; when they run out, a captured persistent launch
// uses the static order instead).
constexpr uint32_t kCounters = 256;
constexpr uint32_t kGraphCounters = 1024;

// Allocation failures injected on the host (tests of the GF2X_ENOMEM paths):
// the next g_fail_allocs allocations of any context fail without a CUDA call.
std::atomic<uint32_t> g_fail_allocs{0};

struct Staging {
    DevItem *host = nullptr;   // pinned
    DevItem *dev = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    bool pending = false;
};

// Device buffers, streams and events of gf2x_mul_strided_host: two sets
// (chunk parity) of a, b and out; in/done/out mark each set's last operand
// copy, product and result copy (across calls: a set is reused only after
// its previous product and result copy, whichever call made them).  The
// products of the two sets run on two streams of their own, so that one
// chunk's launch fills the SMs that the other's last wave leaves idle.
struct HostPipe {
    uint64_t *buf = nullptr;
    size_t bytes = 0;
    cudaStream_t h2d = nullptr, d2h = nullptr, comp[2] = {};
    cudaEvent_t entry = nullptr, in[2] = {}, done[2] = {}, out[2] = {};
    bool ready = false;
};

}  // namespace

struct gf2x_ctx {
    int device = 0;
    int sm_count = 0;
    int checked = 0;
    GPlan *plans_host = nullptr;   // pinned mirror, slots never change once written
    GPlan *plans_dev = nullptr;
    uint32_t nplans = 0;
    std::unordered_map<uint32_t, PlanEntry> by_n;        // current plan per n
    std::unordered_map<uint32_t, PlanEntry> by_n_checked;
    Staging ring[kRing];
    int ring_next = 0;
    uint32_t *err_dev = nullptr;
    uint32_t *plan_of_n_host = nullptr;  // pinned, GF2X_MAX_N + 1 entries
    uint32_t *plan_of_n_dev = nullptr;
    std::string last_error;
    std::vector<DevItem> scratch_items;
    std::vector<uint32_t> scratch_S;
    std::unordered_map<std::string, uint32_t> slot_of;  // (n, spec, checked) -> plan slot, for reuse
    std::unordered_map<uint64_t, int> occupancy;        // (leaf, threads, smem) -> resident CTAs per SM
    std::vector<uint32_t> device_set;                   // sizes of device-item batches (last gf2x_ctx_prepare)
    std::unordered_map<uint32_t, uint32_t> child_of;    // split plan slot -> its children's plan slot
    uint32_t *ws = nullptr;                             // split-plan scratch
    size_t ws_bytes = 0;
    cudaEvent_t ws_done = nullptr;                      // recorded after the last split launch
    cudaStream_t ws_stream = nullptr;
    bool ws_used = false;
    HostPipe hp;                                        // gf2x_mul_strided_host
    uint64_t *ub = nullptr;                             // gf2x_mul_unbalanced: padded operands and products
    size_t ub_bytes = 0;
    cudaEvent_t ub_done = nullptr;                      // recorded after the last use of ub
    cudaStream_t ub_stream = nullptr;
    bool ub_used = false;
    uint32_t *counters = nullptr;                       // work counters of dynamic launches (a ring)
    uint32_t counter_next = 0;
    cudaEvent_t counter_ev[kCounters] = {};               // recorded behind the last launch on each ring slot
    bool counter_used[kCounters] = {};
    uint32_t graph_counter_next = 0;                      // next never-reused slot for captured launches
    bool fixed = false;                                 // workspace fixed at creation: compute calls allocate nothing
    void *arena = nullptr;                              // the fixed workspace (split | unbalanced/Toom | host pipeline)
    uint64_t allocs = 0;                                // device and pinned allocations made by the context
    uint64_t alloc_bytes = 0;
};

// Every device or pinned allocation of a context goes through these two
// (counted; failures injectable by gf2x_debug_fail_next_allocs).
static bool injected_failure()
{
    uint32_t v = g_fail_allocs.load();
    while (v > 0 && !g_fail_allocs.compare_exchange_weak(v, v - 1)) {
    }
    return v > 0;
}

static cudaError_t ctx_malloc(gf2x_ctx *ctx, void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure())
        return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        ctx->allocs++;
        ctx->alloc_bytes += bytes;
    } else {
        *p = nullptr;
    }
    return e;
}

static cudaError_t ctx_malloc_host(gf2x_ctx *ctx, void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure())
        return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) {
        ctx->allocs++;
        ctx->alloc_bytes += bytes;
    } else {
        *p = nullptr;
    }
    return e;
}

static std::string plan_key(uint32_t n, const gf2x_plan_spec &spec, int checked)
{
    std::string k(reinterpret_cast<const char *>(&spec), sizeof(spec));
    k.append(reinterpret_cast<const char *>(&n), sizeof(n));
    k.push_back(checked ? 'c' : 'u');
    return k;
}

static gf2x_status fail(gf2x_ctx *ctx, gf2x_status st, const std::string &msg)
{
    if (ctx)
        ctx->last_error = msg;
    return st;
}

static gf2x_status cuda_fail(gf2x_ctx *ctx, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(ctx, GF2X_ECUDA, m);
}

extern "C" const char *gf2x_status_str(gf2x_status s)
{
    switch (s) {
    case GF2X_OK: return "ok";
    case GF2X_EINVAL: return "invalid argument";
    case GF2X_ENOMEM: return "out of memory";
    case GF2X_ECUDA: return "CUDA error";
    case GF2X_ETIMEOUT: return "timeout";
    case GF2X_EUNSUPPORTED: return "unsupported size or plan";
    case GF2X_EBUSY: return "busy";
    case GF2X_EDEVICE: return "device invariant violated";
    default: return "unknown status";
    }
}

extern "C" const char *gf2x_version(void) { return "gf2x_gb300 1.0 sm_103a"; }

extern "C" gf2x_status gf2x_default_spec(uint32_t n, gf2x_plan_spec *spec) { return default_spec(n, spec); }

extern "C" gf2x_status gf2x_plan_info_get(uint32_t n, const gf2x_plan_spec *spec, gf2x_plan_info *info)
{
    if (!spec || !info)
        return GF2X_EINVAL;
    return build_plan(n, spec, nullptr, info);
}

extern "C" gf2x_status gf2x_spec_parse(const char *text, gf2x_plan_spec *spec) { return parse_spec(text, spec); }

extern "C" gf2x_status gf2x_ctx_create(gf2x_ctx **out, int device, size_t workspace_bytes, const char *plan_db_path)
{
    if (!out)
        return GF2X_EINVAL;
    *out = nullptr;
    gf2x_ctx *ctx = new (std::nothrow) gf2x_ctx();
    if (!ctx)
        return GF2X_ENOMEM;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return GF2X_ECUDA;
    }
    ctx->device = device;
    bool oom = false;   // an allocation (not another CUDA call) failed
    auto alloc = [&](void **p, size_t bytes, bool host) {
        if (e != cudaSuccess)
            return;
        e = host ? ctx_malloc_host(ctx, p, bytes) : ctx_malloc(ctx, p, bytes);
        oom = e == cudaErrorMemoryAllocation;
    };
    e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    alloc((void **)&ctx->plans_host, sizeof(GPlan) * kPlanCapacity, true);
    alloc((void **)&ctx->plans_dev, sizeof(GPlan) * kPlanCapacity, false);
    alloc((void **)&ctx->err_dev, sizeof(uint32_t), false);
    if (e == cudaSuccess)
        e = cudaMemset(ctx->err_dev, 0, sizeof(uint32_t));
    alloc((void **)&ctx->plan_of_n_host, sizeof(uint32_t) * (GF2X_MAX_N + 1), true);
    alloc((void **)&ctx->plan_of_n_dev, sizeof(uint32_t) * (GF2X_MAX_N + 1), false);
    alloc((void **)&ctx->counters, sizeof(uint32_t) * (kCounters + kGraphCounters), false);
    for (auto &ev : ctx->counter_ev)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        memset(ctx->plan_of_n_host, 0xff, sizeof(uint32_t) * (GF2X_MAX_N + 1));
        e = cudaMemset(ctx->plan_of_n_dev, 0xff, sizeof(uint32_t) * (GF2X_MAX_N + 1));
    }
    if (workspace_bytes > 0 && e == cudaSuccess) {
        // one arena: half for split-plan scratch, a quarter for the
        // unbalanced / Toom scratch, a quarter for the host-buffer pipeline
        // (they may be live at the same time: a host-buffer or Toom call runs
        // split plans inside it)
        const size_t W = workspace_bytes & ~(size_t)1023;
        alloc(&ctx->arena, W, false);
        if (e == cudaSuccess) {
            uint8_t *base = static_cast<uint8_t *>(ctx->arena);
            ctx->ws = reinterpret_cast<uint32_t *>(base);
            ctx->ws_bytes = W / 2;
            ctx->ub = reinterpret_cast<uint64_t *>(base + W / 2);
            ctx->ub_bytes = W / 4;
            ctx->hp.buf = reinterpret_cast<uint64_t *>(base + W / 2 + W / 4);
            ctx->hp.bytes = W / 4;
            ctx->fixed = true;
        }
        for (auto &r : ctx->ring) {
            alloc((void **)&r.host, kFixedStagingItems * sizeof(DevItem), true);
            alloc((void **)&r.dev, kFixedStagingItems * sizeof(DevItem), false);
            if (e == cudaSuccess)
                r.cap = kFixedStagingItems;
        }
        ctx->scratch_items.reserve(kFixedStagingItems);
        ctx->scratch_S.reserve(kFixedStagingItems);
    }
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    for (uint32_t S : kLeafSizes)
        if (e == cudaSuccess)
            e = preparer_for(S)(nullptr, 0, 0);
    if (e == cudaSuccess)
        e = prepare_split();
    if (e == cudaSuccess)
        e = prepare_tc();
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ctx->ws_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ctx->ub_done, cudaEventDisableTiming);
    for (auto &r : ctx->ring)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
    if (e == cudaSuccess) {   // streams and events of the host-buffer pipeline
        HostPipe &hp = ctx->hp;
        for (cudaStream_t *st : {&hp.h2d, &hp.d2h, &hp.comp[0], &hp.comp[1]})
            if (e == cudaSuccess)
                e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
        cudaEvent_t *evs[] = {&hp.entry, &hp.in[0], &hp.in[1], &hp.done[0], &hp.done[1], &hp.out[0], &hp.out[1]};
        for (cudaEvent_t *ev : evs)
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        hp.ready = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        gf2x_ctx_destroy(ctx);
        return oom ? GF2X_ENOMEM : GF2X_ECUDA;
    }
    if (plan_db_path) {
        gf2x_status st = gf2x_ctx_load_plan_db(ctx, plan_db_path, 4096);
        if (st != GF2X_OK) {
            gf2x_ctx_destroy(ctx);
            return st;
        }
    }
    *out = ctx;
    return GF2X_OK;
}

extern "C" gf2x_status gf2x_ctx_alloc_count(gf2x_ctx *ctx, uint64_t *allocations, uint64_t *bytes)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (allocations)
        *allocations = ctx->allocs;
    if (bytes)
        *bytes = ctx->alloc_bytes;
    return GF2X_OK;
}

extern "C" uint32_t gf2x_debug_fail_next_allocs(uint32_t count)
{
    return g_fail_allocs.exchange(count);
}

extern "C" void gf2x_ctx_destroy(gf2x_ctx *ctx)
{
    if (!ctx)
        return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &r : ctx->ring) {
        if (r.host)
            cudaFreeHost(r.host);
        if (r.dev)
            cudaFree(r.dev);
        if (r.done)
            cudaEventDestroy(r.done);
    }
    if (ctx->plans_host)
        cudaFreeHost(ctx->plans_host);
    if (ctx->plans_dev)
        cudaFree(ctx->plans_dev);
    if (ctx->err_dev)
        cudaFree(ctx->err_dev);
    if (ctx->plan_of_n_host)
        cudaFreeHost(ctx->plan_of_n_host);
    if (ctx->plan_of_n_dev)
        cudaFree(ctx->plan_of_n_dev);
    if (ctx->counters)
        cudaFree(ctx->counters);
    for (cudaEvent_t ev : ctx->counter_ev)
        if (ev)
            cudaEventDestroy(ev);
    if (ctx->arena) {   // ws, ub and hp.buf live in it
        cudaFree(ctx->arena);
    } else {
        if (ctx->ws)
            cudaFree(ctx->ws);
        if (ctx->ub)
            cudaFree(ctx->ub);
        if (ctx->hp.buf)
            cudaFree(ctx->hp.buf);
    }
    if (ctx->ws_done)
        cudaEventDestroy(ctx->ws_done);
    if (ctx->ub_done)
        cudaEventDestroy(ctx->ub_done);
    HostPipe &hp = ctx->hp;
    for (cudaStream_t st : {hp.h2d, hp.d2h, hp.comp[0], hp.comp[1]})
        if (st)
            cudaStreamDestroy(st);
    for (cudaEvent_t ev : {hp.entry, hp.in[0], hp.in[1], hp.done[0], hp.done[1], hp.out[0], hp.out[1]})
        if (ev)
            cudaEventDestroy(ev);
    delete ctx;
}

// Build the plan for (n, spec), store it in a new slot and enqueue its upload.
static gf2x_status install_plan(gf2x_ctx *ctx, uint32_t n, const gf2x_plan_spec &spec, int checked,
                                cudaStream_t stream, uint32_t *slot)
{
    const std::string key = plan_key(n, spec, checked);
    auto found = ctx->slot_of.find(key);
    if (found != ctx->slot_of.end()) {  // slots never change once written: reuse
        *slot = found->second;
        return GF2X_OK;
    }
    const uint32_t need = spec.split_top ? 2u : 1u;
    if (ctx->nplans + need > kPlanCapacity)
        return fail(ctx, GF2X_EUNSUPPORTED, "plan table full");
    GPlan P, C;
    gf2x_status st = build_plan(n, &spec, &P, nullptr, &C);
    if (st != GF2X_OK)
        return fail(ctx, st, "plan does not fit this size");
    P.checked = checked ? 1u : 0u;
    C.checked = checked ? 1u : 0u;
    const uint32_t s = ctx->nplans;
    ctx->nplans += need;
    ctx->plans_host[s] = P;
    if (spec.split_top) {
        ctx->plans_host[s + 1] = C;
        ctx->child_of[s] = s + 1;
    }
    cudaError_t e = cudaMemcpyAsync(ctx->plans_dev + s, ctx->plans_host + s, need * sizeof(GPlan),
                                    cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "plan upload");
    ctx->slot_of[key] = s;
    *slot = s;
    return GF2X_OK;
}

// Make `slot` the plan device-resident item batches use for n.
static gf2x_status publish_plan(gf2x_ctx *ctx, uint32_t n, uint32_t slot, cudaStream_t stream)
{
    ctx->plan_of_n_host[n] = slot;
    cudaError_t e = cudaMemcpyAsync(ctx->plan_of_n_dev + n, ctx->plan_of_n_host + n, sizeof(uint32_t),
                                    cudaMemcpyHostToDevice, stream);
    return e == cudaSuccess ? GF2X_OK : cuda_fail(ctx, e, "plan index upload");
}

static gf2x_status plan_for(gf2x_ctx *ctx, uint32_t n, cudaStream_t stream, uint32_t *slot)
{
    if (n < 1 || n > GF2X_MAX_N)
        return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 131072]");
    auto &map = ctx->checked ? ctx->by_n_checked : ctx->by_n;
    auto it = map.find(n);
    if (it != map.end()) {
        *slot = it->second.slot;
        return GF2X_OK;
    }
    // the spec currently chosen for n (set by gf2x_ctx_set_plan or the default)
    gf2x_plan_spec spec;
    auto other = (ctx->checked ? ctx->by_n : ctx->by_n_checked).find(n);
    if (other != (ctx->checked ? ctx->by_n : ctx->by_n_checked).end()) {
        spec = other->second.spec;
    } else {
        gf2x_status st = default_spec(n, &spec);
        if (st != GF2X_OK)
            return fail(ctx, st, "no plan fits this size");
    }
    uint32_t s;
    gf2x_status st = install_plan(ctx, n, spec, ctx->checked, stream, &s);
    if (st != GF2X_OK)
        return st;
    map[n] = PlanEntry{s, spec};
    *slot = s;
    return GF2X_OK;
}

static bool in_device_set(const gf2x_ctx *ctx, uint32_t n)
{
    return std::find(ctx->device_set.begin(), ctx->device_set.end(), n) != ctx->device_set.end();
}

extern "C" gf2x_status gf2x_ctx_set_plan(gf2x_ctx *ctx, uint32_t n, const gf2x_plan_spec *spec)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (n < 1 || n > GF2X_MAX_N)
        return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 131072]");
    cudaSetDevice(ctx->device);
    if (!spec) {
        ctx->by_n.erase(n);
        ctx->by_n_checked.erase(n);
        if (in_device_set(ctx, n)) {
            uint32_t slot;
            gf2x_status st = plan_for(ctx, n, nullptr, &slot);
            if (st != GF2X_OK)
                return st;
            st = publish_plan(ctx, n, slot, nullptr);
            if (st != GF2X_OK)
                return st;
            cudaStreamSynchronize(nullptr);
        }
        return GF2X_OK;
    }
    // the current plan stays in force unless the new one is valid and installed
    gf2x_plan_info info;
    gf2x_status st = build_plan(n, spec, nullptr, &info);
    if (st != GF2X_OK)
        return fail(ctx, st, "plan rejected for this size");
    uint32_t s;
    st = install_plan(ctx, n, *spec, ctx->checked, nullptr, &s);
    if (st != GF2X_OK)
        return st;
    ctx->by_n.erase(n);
    ctx->by_n_checked.erase(n);
    (ctx->checked ? ctx->by_n_checked : ctx->by_n)[n] = PlanEntry{s, *spec};
    if (in_device_set(ctx, n)) {
        st = publish_plan(ctx, n, s, nullptr);
        if (st != GF2X_OK)
            return st;
    }
    cudaError_t e = cudaStreamSynchronize(nullptr);
    return e == cudaSuccess ? GF2X_OK : cuda_fail(ctx, e, "plan upload");
}

extern "C" gf2x_status gf2x_ctx_get_plan(gf2x_ctx *ctx, uint32_t n, gf2x_plan_spec *spec)
{
    if (!ctx || !spec)
        return GF2X_EINVAL;
    auto &map = ctx->checked ? ctx->by_n_checked : ctx->by_n;
    auto it = map.find(n);
    if (it != map.end()) {
        *spec = it->second.spec;
        return GF2X_OK;
    }
    auto &o = ctx->checked ? ctx->by_n : ctx->by_n_checked;
    auto it2 = o.find(n);
    if (it2 != o.end()) {
        *spec = it2->second.spec;
        return GF2X_OK;
    }
    return default_spec(n, spec);
}

extern "C" gf2x_status gf2x_ctx_set_checked(gf2x_ctx *ctx, int on)
{
    if (!ctx)
        return GF2X_EINVAL;
    ctx->checked = on ? 1 : 0;
    // device-item batches follow the mode: republish the prepared sizes' plans
    for (uint32_t n : ctx->device_set) {
        uint32_t slot;
        gf2x_status st = plan_for(ctx, n, nullptr, &slot);
        if (st != GF2X_OK)
            return st;
        st = publish_plan(ctx, n, slot, nullptr);
        if (st != GF2X_OK)
            return st;
    }
    cudaStreamSynchronize(nullptr);
    return GF2X_OK;
}

static bool ranges_overlap(const void *p, size_t pbytes, const void *q, size_t qbytes)
{
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + qbytes && b < a + pbytes;
}

static gf2x_status check_operands(gf2x_ctx *ctx, const uint64_t *out, const uint64_t *a, const uint64_t *b,
                                  uint32_t n, uint32_t flags, size_t count, size_t stride_in, size_t stride_out,
                                  bool shared_a = false)
{
    if (!out || !a || !b)
        return fail(ctx, GF2X_EINVAL, "null operand or result pointer");
    if (((uintptr_t)out | (uintptr_t)a | (uintptr_t)b) & 7u)
        return fail(ctx, GF2X_EINVAL, "operands and results must be 8-byte aligned");
    if (flags & ~GF2X_REDUCE)
        return fail(ctx, GF2X_EINVAL, "unknown flag");
    const size_t L = (n + 63) / 64;
    const size_t Lo = (flags & GF2X_REDUCE) ? L : (size_t)((2ull * n - 1 + 63) / 64);
    if (count > 1 && (stride_in < L || stride_out < Lo))
        return fail(ctx, GF2X_EINVAL, "stride smaller than the operand or result size");
    const size_t in_bytes = 8 * ((count - 1) * stride_in + L);
    const size_t out_bytes = 8 * ((count - 1) * stride_out + Lo);
    if (ranges_overlap(out, out_bytes, a, shared_a ? 8 * L : in_bytes) || ranges_overlap(out, out_bytes, b, in_bytes))
        return fail(ctx, GF2X_EINVAL, "result overlaps an operand");
    return GF2X_OK;
}

static gf2x_status launch(gf2x_ctx *ctx, const LaunchArgs &args, uint32_t S, unsigned threads, size_t smem,
                          size_t count, bool persistent, cudaStream_t stream, bool dynamic = false)
{
    LaunchFn fn = launcher_for(S);
    if (!fn)
        return fail(ctx, GF2X_EUNSUPPORTED, "leaf size not compiled");
    unsigned grid;
    LaunchArgs a = args;
    int ring_slot = -1;   // counter ring slot of an uncaptured dynamic launch
    if (persistent) {
        // cached so that launches inside a CUDA graph capture make no occupancy query
        const uint64_t okey = ((uint64_t)S << 48) | ((uint64_t)threads << 32) | (uint64_t)smem;
        int per_sm = 0;
        auto oc = ctx->occupancy.find(okey);
        if (oc != ctx->occupancy.end()) {
            per_sm = oc->second;
        } else {
            cudaError_t e = preparer_for(S)(&per_sm, threads, smem);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "occupancy query");
            ctx->occupancy[okey] = per_sm;
        }
        if (per_sm < 1)
            return fail(ctx, GF2X_EUNSUPPORTED, "kernel does not fit on an SM");
        grid = (unsigned)std::min<size_t>(count, (size_t)per_sm * ctx->sm_count);
        a.persistent = 1;
        if (dynamic && grid > 0) {   // items in order from a counter zeroed on the stream (a graph node too)
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            cudaError_t e = cudaStreamIsCapturing(stream, &cs);
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "capture status");
            uint32_t *c = nullptr;
            if (cs != cudaStreamCaptureStatusNone) {
                if (ctx->graph_counter_next < kGraphCounters)
                    c = ctx->counters + kCounters + ctx->graph_counter_next++;
            } else {
                ring_slot = (int)(ctx->counter_next++ % kCounters);
                if (ctx->counter_used[ring_slot])   // its previous launch (any stream) has finished with it
                    e = cudaStreamWaitEvent(stream, ctx->counter_ev[ring_slot], 0);
                if (e != cudaSuccess)
                    return cuda_fail(ctx, e, "work counter wait");
                c = ctx->counters + ring_slot;
            }
            if (c) {
                e = cudaMemsetAsync(c, 0, sizeof(uint32_t), stream);
                if (e != cudaSuccess)
                    return cuda_fail(ctx, e, "work counter reset");
                a.work_counter = c;
            }
        }
    } else {
        if (count > 0x7fffffffu)
            return fail(ctx, GF2X_EINVAL, "batch too large for one launch");
        grid = (unsigned)count;
        a.persistent = 0;
    }
    if (grid == 0)
        return GF2X_OK;
    cudaError_t e = fn(a, grid, threads, smem, stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "kernel launch");
    if (ring_slot >= 0) {
        e = cudaEventRecord(ctx->counter_ev[ring_slot], stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "work counter event");
        ctx->counter_used[ring_slot] = true;
    }
    return GF2X_OK;
}

// Scratch of at least `bytes` for split plans (grows only; waits for the
// device before replacing a smaller buffer).
static gf2x_status ensure_workspace(gf2x_ctx *ctx, size_t bytes)
{
    if (ctx->ws_bytes >= bytes)
        return GF2X_OK;
    if (ctx->fixed)   // chunks shrink to the fixed scratch; only one product that does not fit fails
        return fail(ctx, GF2X_ENOMEM, "fixed workspace too small for one product of this split plan");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "workspace wait");
    if (ctx->ws)
        cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    if (ctx_malloc(ctx, (void **)&ctx->ws, bytes) != cudaSuccess)
        return fail(ctx, GF2X_ENOMEM, "split workspace allocation");
    ctx->ws_bytes = bytes;
    return GF2X_OK;
}

// The three launches of a split plan over `count` products, in chunks whose
// scratch fits `ws_bytes` bytes at `ws`.  `top` describes the products
// (strided pointers or a device item array, plan = top_slot); chunk c0
// starts at product c0 of it.
static gf2x_status run_split_on(gf2x_ctx *ctx, uint32_t top_slot, uint32_t *ws, size_t ws_bytes,
                                const LaunchArgs &top, size_t count, bool persistent, cudaStream_t stream)
{
    auto ch = ctx->child_of.find(top_slot);
    if (ch == ctx->child_of.end())
        return fail(ctx, GF2X_EINVAL, "split plan without children plan");
    const GPlan &T = ctx->plans_host[top_slot];
    const GPlan &C = ctx->plans_host[ch->second];
    const uint32_t nch = T.lev[0].nch, E = T.lev[0].E;
    const size_t per = 4ull * nch * 2ull * E;
    const size_t chunk = std::min<size_t>(count, ws_bytes / per);
    if (chunk == 0)
        return fail(ctx, GF2X_EUNSUPPORTED, "scratch too small for one product");
    const unsigned top_threads = T.threads;
    const size_t top_smem = 4ull * T.smem_words;
    for (size_t c0 = 0; c0 < count; c0 += chunk) {
        const size_t k = std::min(chunk, count - c0);
        LaunchArgs ta = top;
        if (ta.mode == kItemsStrided) {
            if (!ta.shared_a)
                ta.base.a += c0 * ta.stride_in;
            ta.base.b += c0 * ta.stride_in;
            ta.base.out += c0 * ta.stride_out;
        } else {
            ta.items += c0;
        }
        ta.count = (uint32_t)k;
        ta.err = ctx->err_dev;
        ta.persistent = persistent ? 1u : 0u;
        const unsigned tgrid = (unsigned)(persistent ? std::min<size_t>(k, 4ull * ctx->sm_count) : k);
        cudaError_t e = launch_split_eval(ta, ws, tgrid, top_threads, top_smem, stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "split evaluation launch");
        // children: independent full products of E words, written over their operand slots
        LaunchArgs ca;
        memset(&ca, 0, sizeof(ca));
        ca.plans = ctx->plans_dev;
        ca.base = DevItem{reinterpret_cast<const uint64_t *>(ws), reinterpret_cast<const uint64_t *>(ws + E),
                          reinterpret_cast<uint64_t *>(ws), ch->second, 0u};
        ca.stride_in = E;    // 2E words = E limbs per slot
        ca.stride_out = E;
        ca.count = (uint32_t)(k * nch);
        ca.mode = kItemsStrided;
        ca.err = ctx->err_dev;
        // persistent: the children are taken in order from a counter, as the
        // products of an unsplit plan are
        gf2x_status st = launch(ctx, ca, C.S, C.threads, 4ull * C.smem_words, k * nch, persistent, stream,
                                persistent);
        if (st != GF2X_OK)
            return st;
        e = launch_split_interp(ta, ws, tgrid, top_threads, top_smem, stream);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "split interpolation launch");
    }
    return GF2X_OK;
}

static gf2x_status run_split_args(gf2x_ctx *ctx, uint32_t top_slot, const LaunchArgs &top, size_t count,
                                  bool persistent, cudaStream_t stream)
{
    const GPlan &T = ctx->plans_host[top_slot];
    const size_t per = 4ull * T.lev[0].nch * 2ull * T.lev[0].E;
    const size_t want = ctx->fixed ? per : std::max<size_t>(per, std::min<size_t>(count * per, kWorkspaceCap / per * per));
    gf2x_status st = ensure_workspace(ctx, want);
    if (st != GF2X_OK)
        return st;
    // the scratch is shared by every split call of the context: order this
    // call after the previous one when it came on another stream
    if (ctx->ws_used && ctx->ws_stream != stream) {
        cudaError_t e = cudaStreamWaitEvent(stream, ctx->ws_done, 0);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "workspace ordering");
    }
    st = run_split_on(ctx, top_slot, ctx->ws, ctx->ws_bytes, top, count, persistent, stream);
    if (st != GF2X_OK)
        return st;
    cudaError_t e = cudaEventRecord(ctx->ws_done, stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "workspace event");
    ctx->ws_used = true;
    ctx->ws_stream = stream;
    return GF2X_OK;
}

static gf2x_status run_split(gf2x_ctx *ctx, uint32_t top_slot, uint64_t *out, const uint64_t *a, const uint64_t *b,
                             size_t count, size_t stride_in, size_t stride_out, uint32_t flags, bool persistent,
                             cudaStream_t stream, bool shared_a = false)
{
    LaunchArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.plans = ctx->plans_dev;
    ta.base = DevItem{a, b, out, top_slot, flags};
    ta.stride_in = stride_in;
    ta.stride_out = stride_out;
    ta.mode = kItemsStrided;
    ta.shared_a = shared_a ? 1u : 0u;
    return run_split_args(ctx, top_slot, ta, count, persistent, stream);
}

static gf2x_status one_product(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n,
                               uint32_t flags, gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (n < 1 || n > GF2X_MAX_N)
        return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 131072]");
    gf2x_status st = check_operands(ctx, out, a, b, n, flags, 1, 0, 0);
    if (st != GF2X_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t slot;
    st = plan_for(ctx, n, s, &slot);
    if (st != GF2X_OK)
        return st;
    const GPlan &P = ctx->plans_host[slot];
    if (P.split)
        return run_split(ctx, slot, out, a, b, 1, 0, 0, flags, false, s);
    LaunchArgs args;
    memset(&args, 0, sizeof(args));
    args.plans = ctx->plans_dev;
    args.base = DevItem{a, b, out, slot, flags};
    args.count = 1;
    args.mode = kItemsSingle;
    args.err = ctx->err_dev;
    return launch(ctx, args, P.S, P.threads, 4ull * P.smem_words, 1, false, s);
}

extern "C" gf2x_status gf2x_mul(gf2x_ctx *ctx, uint64_t *c, const uint64_t *a, const uint64_t *b, uint32_t n,
                                gf2x_stream stream)
{
    return one_product(ctx, c, a, b, n, 0u, stream);
}

extern "C" gf2x_status gf2x_mulmod_xn1(gf2x_ctx *ctx, uint64_t *r, const uint64_t *a, const uint64_t *b,
                                       uint32_t n, gf2x_stream stream)
{
    return one_product(ctx, r, a, b, n, GF2X_REDUCE, stream);
}

static gf2x_status strided_on_slot(gf2x_ctx *ctx, uint32_t slot, uint64_t *out, const uint64_t *a,
                                   const uint64_t *b, size_t count, size_t stride_in, size_t stride_out,
                                   uint32_t flags, uint32_t batch_flags, cudaStream_t s);

extern "C" gf2x_status gf2x_mul_strided(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b,
                                        uint32_t n, size_t count, size_t stride_in, size_t stride_out,
                                        uint32_t flags, uint32_t batch_flags, gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (n < 1 || n > GF2X_MAX_N)
        return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 131072]");
    if (batch_flags & ~(uint32_t)(GF2X_BATCH_PERSISTENT | GF2X_BATCH_SHARED_A))
        return fail(ctx, GF2X_EINVAL, "unknown batch flag");
    const bool shared_a = (batch_flags & GF2X_BATCH_SHARED_A) != 0;
    gf2x_status st = check_operands(ctx, out, a, b, n, flags, count, stride_in, stride_out, shared_a);
    if (st != GF2X_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t slot;
    st = plan_for(ctx, n, s, &slot);
    if (st != GF2X_OK)
        return st;
    return strided_on_slot(ctx, slot, out, a, b, count, stride_in, stride_out, flags, batch_flags, s);
}

// The strided batch under plan `slot` (operands already checked).
static gf2x_status strided_on_slot(gf2x_ctx *ctx, uint32_t slot, uint64_t *out, const uint64_t *a,
                                   const uint64_t *b, size_t count, size_t stride_in, size_t stride_out,
                                   uint32_t flags, uint32_t batch_flags, cudaStream_t s)
{
    const bool shared_a = (batch_flags & GF2X_BATCH_SHARED_A) != 0;
    const GPlan &P = ctx->plans_host[slot];
    if (P.split)
        return run_split(ctx, slot, out, a, b, count, stride_in, stride_out, flags,
                         (batch_flags & GF2X_BATCH_PERSISTENT) != 0, s, shared_a);
    LaunchArgs args;
    memset(&args, 0, sizeof(args));
    args.plans = ctx->plans_dev;
    args.base = DevItem{a, b, out, slot, flags};
    args.stride_in = stride_in;
    args.stride_out = stride_out;
    args.count = (uint32_t)count;
    args.mode = kItemsStrided;
    args.shared_a = shared_a ? 1u : 0u;
    args.err = ctx->err_dev;
    if (count > 0xffffffffull)
        return fail(ctx, GF2X_EINVAL, "batch too large");
    // persistent: the CTAs take the products in order from a counter, which
    // measured faster than the static order i, i + grid, ... at every size
    // (4096 x 17669: 7.12 -> 7.50 M/s; 3648 x 17669: 7.22 -> 7.95; 12323:
    // 9.12 -> 10.04; 57637: 1.08 -> 1.14; 35851 unchanged)
    const bool persistent = (batch_flags & GF2X_BATCH_PERSISTENT) != 0;
    return launch(ctx, args, P.S, P.threads, 4ull * P.smem_words, count, persistent, s, persistent);
}

// The context scratch of the unbalanced and Toom-4 calls: at least `want`
// bytes (grows only; cudaFree synchronizes the device, so no call still
// uses the old buffer), ordered after the previous call that used it when
// that came on another stream.  scratch_release records the ordering event.
// Bytes of that scratch one call may use per group of products.
static size_t scratch_cap(const gf2x_ctx *ctx)
{
    return ctx->fixed ? ctx->ub_bytes : (size_t)kWorkspaceCap;
}

static gf2x_status scratch_acquire(gf2x_ctx *ctx, size_t want, cudaStream_t s)
{
    if (ctx->ub_bytes < want) {
        if (ctx->fixed)
            return fail(ctx, GF2X_ENOMEM, "fixed workspace too small for one product of this call");
        if (ctx->ub) {
            cudaError_t e = cudaFree(ctx->ub);
            ctx->ub = nullptr;
            ctx->ub_bytes = 0;
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "scratch");
        }
        cudaError_t e = ctx_malloc(ctx, (void **)&ctx->ub, want);
        if (e != cudaSuccess) {
            ctx->ub = nullptr;
            return e == cudaErrorMemoryAllocation ? fail(ctx, GF2X_ENOMEM, "scratch") : cuda_fail(ctx, e, "scratch");
        }
        ctx->ub_bytes = want;
    }
    if (ctx->ub_used && ctx->ub_stream != s) {
        cudaError_t e = cudaStreamWaitEvent(s, ctx->ub_done, 0);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "scratch ordering");
    }
    return GF2X_OK;
}

static gf2x_status scratch_release(gf2x_ctx *ctx, cudaStream_t s)
{
    cudaError_t e = cudaEventRecord(ctx->ub_done, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "scratch event");
    ctx->ub_used = true;
    ctx->ub_stream = s;
    return GF2X_OK;
}

// The plan slot and modelled operations of a product of size n in an
// unbalanced call: the context's current plan for n; for the chunk size m
// (= 64 ceil(nb/64)) without a plan of its own, the spec of nb's plan where
// it also covers m (the same limb count, so a plan tuned for nb serves its
// chunk products), else the default.  A borrowed spec gets a slot of its
// own but does not become the context's plan for m.
static gf2x_status unbalanced_plan(gf2x_ctx *ctx, uint32_t n, uint32_t borrow_from, cudaStream_t s,
                                   uint32_t *slot, uint64_t *ops)
{
    auto &map = ctx->checked ? ctx->by_n_checked : ctx->by_n;
    gf2x_plan_info info;
    gf2x_status st;
    if (borrow_from && borrow_from != n && map.find(n) == map.end()) {
        uint32_t unused;
        st = plan_for(ctx, borrow_from, s, &unused);
        if (st != GF2X_OK)
            return st;
        const gf2x_plan_spec spec = map.at(borrow_from).spec;
        if (gf2x_plan_info_get(n, &spec, &info) == GF2X_OK &&
            install_plan(ctx, n, spec, ctx->checked, s, slot) == GF2X_OK) {
            *ops = info.ops_full;
            return GF2X_OK;
        }
    }
    st = plan_for(ctx, n, s, slot);
    if (st != GF2X_OK)
        return st;
    st = gf2x_plan_info_get(n, &map.at(n).spec, &info);
    if (st != GF2X_OK)
        return fail(ctx, st, "plan description");
    *ops = info.ops_full;
    return GF2X_OK;
}

extern "C" gf2x_status gf2x_mul_unbalanced(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, uint32_t na,
                                           size_t stride_a, const uint64_t *b, uint32_t nb, size_t stride_b,
                                           size_t count, size_t stride_out, gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (na < 1 || nb < 1 || na > GF2X_MAX_N || nb > GF2X_MAX_N)
        return fail(ctx, GF2X_EUNSUPPORTED, "operand size outside [1, 131072]");
    if (!out || !a || !b)
        return fail(ctx, GF2X_EINVAL, "null operand or result pointer");
    if (((uintptr_t)out | (uintptr_t)a | (uintptr_t)b) & 7u)
        return fail(ctx, GF2X_EINVAL, "operands and results must be 8-byte aligned");
    const size_t La = (na + 63) / 64, Lb = (nb + 63) / 64;
    const uint32_t Lu = (uint32_t)(((uint64_t)na + nb - 1 + 63) / 64);
    if (count > 1 && (stride_a < La || stride_b < Lb || stride_out < Lu))
        return fail(ctx, GF2X_EINVAL, "stride smaller than the operand or result size");
    const size_t out_bytes = 8 * ((count - 1) * stride_out + Lu);
    if (ranges_overlap(out, out_bytes, a, 8 * ((count - 1) * stride_a + La)) ||
        ranges_overlap(out, out_bytes, b, 8 * ((count - 1) * stride_b + Lb)))
        return fail(ctx, GF2X_EINVAL, "result overlaps an operand");
    if (na < nb) {   // the product commutes: a is the longer operand from here on
        std::swap(a, b);
        std::swap(na, nb);
        std::swap(stride_a, stride_b);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // padded: one product of size na; chunked: k products of size m
    const uint32_t Lc = (uint32_t)((nb + 63) / 64), m = 64u * Lc;
    const uint32_t k = (na + m - 1) / m;
    uint32_t size = na, chunks = 1, Ld = (uint32_t)((na + 63) / 64), step = 0, slot = 0;
    uint64_t ops_pad = 0;
    gf2x_status pst = unbalanced_plan(ctx, na, 0u, s, &slot, &ops_pad);
    if (pst != GF2X_OK)
        return pst;
    if (k >= 2) {
        uint32_t chunk_slot = 0;
        uint64_t ops_chunk = 0;
        pst = unbalanced_plan(ctx, m, nb, s, &chunk_slot, &ops_chunk);
        if (pst != GF2X_OK)
            return pst;
        if ((uint64_t)k * ops_chunk < ops_pad) {
            size = m;
            chunks = k;
            Ld = Lc;
            step = Lc;
            slot = chunk_slot;
        }
    }
    const uint32_t Wp = (uint32_t)((2ull * size - 1 + 63) / 64);
    if (chunks == 1)
        step = Wp;
    // scratch per product: chunks x (two operand rows + one product row)
    const size_t per = 8ull * chunks * (2ull * Ld + Wp);
    const size_t group = std::max<size_t>(1, std::min<size_t>(count, scratch_cap(ctx) / per));
    gf2x_status sst = scratch_acquire(ctx, group * per, s);
    if (sst != GF2X_OK)
        return sst;
    for (size_t c0 = 0; c0 < count; c0 += group) {
        const size_t g = std::min(group, count - c0);
        uint64_t *A = ctx->ub, *B = A + g * chunks * Ld, *P = B + g * chunks * Ld;
        cudaError_t e = launch_pad_rows(A, a + c0 * stride_a, stride_a, na, g, chunks, Ld, chunks > 1 ? Lc : 0u,
                                        ctx->sm_count, s);
        if (e == cudaSuccess)
            e = launch_pad_rows(B, b + c0 * stride_b, stride_b, nb, g, chunks, Ld, 0u, ctx->sm_count, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "operand padding launch");
        if (g * chunks > 0xffffffffull)
            return fail(ctx, GF2X_EINVAL, "batch too large");
        // one CTA per chunk product: 1.95 against 1.84 M/s for persistent
        // launches at 2048 x (57637 x 17669)
        gf2x_status st = strided_on_slot(ctx, slot, P, A, B, g * chunks, Ld, Wp, 0u, 0u, s);
        if (st != GF2X_OK)
            return st;
        e = launch_overlap_add(out + c0 * stride_out, stride_out, Lu, P, Wp, g, chunks, step, ctx->sm_count, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "overlap-add launch");
    }
    return scratch_release(ctx, s);
}

extern "C" gf2x_status gf2x_mulmod_sparse(gf2x_ctx *ctx, uint64_t *r, const uint64_t *a, const uint32_t *pos,
                                          uint32_t w, uint32_t n, size_t count, size_t stride_a, size_t stride_pos,
                                          size_t stride_r, gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (n < 1 || n > kSparseMaxN)
        return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 65536] for the sparse product");
    if (!r || !a || (w && !pos))
        return fail(ctx, GF2X_EINVAL, "null operand or result pointer");
    if ((((uintptr_t)r | (uintptr_t)a) & 7u) || ((uintptr_t)pos & 3u))
        return fail(ctx, GF2X_EINVAL, "misaligned operand or result");
    const size_t L = (n + 63) / 64;
    if (count > 1 && (stride_a < L || stride_r < L || stride_pos < w))
        return fail(ctx, GF2X_EINVAL, "stride smaller than the operand, position list or result");
    if (count > 0xffffffffull)
        return fail(ctx, GF2X_EINVAL, "batch too large");
    const size_t r_bytes = 8 * ((count - 1) * stride_r + L);
    if (ranges_overlap(r, r_bytes, a, 8 * ((count - 1) * stride_a + L)) ||
        (w && ranges_overlap(r, r_bytes, pos, 4 * ((count - 1) * stride_pos + w))))
        return fail(ctx, GF2X_EINVAL, "result overlaps an operand");
    SparseShape sh;
    if (!sparse_shape(n, &sh))
        return fail(ctx, GF2X_EUNSUPPORTED, "no sparse kernel shape for this n");
    SparseArgs args;
    memset(&args, 0, sizeof(args));
    args.a = a;
    args.pos = pos;
    args.r = r;
    args.stride_a = stride_a;
    args.stride_pos = stride_pos;
    args.stride_r = stride_r;
    args.n = n;
    args.w = w;
    args.count = (uint32_t)count;
    args.T = sh.T;
    args.pre = sh.pre;
    args.d_words = sh.d_words;
    args.b_words = sh.b_words;
    cudaError_t e = launch_sparse_mulmod(args, sh, ctx->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "sparse product launch");
    return GF2X_OK;
}

extern "C" gf2x_status gf2x_sparse_info_get(uint32_t n, gf2x_sparse_info *info)
{
    if (!info)
        return GF2X_EINVAL;
    SparseShape sh;
    if (!sparse_shape(n, &sh))
        return GF2X_EUNSUPPORTED;
    info->n = n;
    info->words_per_lane = sh.C;
    info->result_words_per_lane = sh.R;
    info->shared_stages = sh.pre;
    uint32_t th = 0;
    while ((sh.QH >> th) != 0u)
        ++th;
    info->register_stages = th;
    info->lane_stages = 5;
    info->smem_bytes = (uint32_t)sparse_smem_bytes(sh);
    return GF2X_OK;
}

// A Toom-K top level (K = 4 or 5): evaluation kernel, the 2K - 1 child
// products of every row as one strided batch, interpolation kernel.
static gf2x_status run_toom(gf2x_ctx *ctx, uint32_t K, uint64_t *out, const uint64_t *a, const uint64_t *b,
                            uint32_t n, size_t count, size_t stride_in, size_t stride_out, uint32_t flags,
                            gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (n < 1 || n > GF2X_MAX_N)
        return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 131072]");
    gf2x_status st = check_operands(ctx, out, a, b, n, flags, count, stride_in, stride_out);
    if (st != GF2X_OK)
        return st;
    ToomArgs t;
    memset(&t, 0, sizeof(t));
    if (!toom_shape(K, n, &t))
        return fail(ctx, GF2X_EUNSUPPORTED, "no Toom shape for this n");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t NP = 2u * K - 1u;
    // the children: full products of 32 E bits, E/2 limbs per operand
    uint32_t slot;
    st = plan_for(ctx, 32u * t.E, s, &slot);
    if (st != GF2X_OK)
        return st;
    const size_t per = 4ull * 4u * NP * t.E;   // NP operand slots and NP products of 2E words
    const size_t group = std::max<size_t>(1, std::min<size_t>(count, scratch_cap(ctx) / per));
    st = scratch_acquire(ctx, group * per, s);
    if (st != GF2X_OK)
        return st;
    t.stride_in = stride_in;
    t.stride_out = stride_out;
    t.n = n;
    t.flags = flags;
    t.err = ctx->checked ? ctx->err_dev : nullptr;
    for (size_t c0 = 0; c0 < count; c0 += group) {
        const size_t g = std::min(group, count - c0);
        uint32_t *opnd = reinterpret_cast<uint32_t *>(ctx->ub);
        uint32_t *prod = opnd + g * 2u * NP * t.E;
        t.a = a + c0 * stride_in;
        t.b = b + c0 * stride_in;
        t.out = out + c0 * stride_out;
        t.count = (uint32_t)g;
        t.opnd = opnd;
        t.prod = prod;
        const unsigned grid = (unsigned)std::min<size_t>(g, 8ull * ctx->sm_count);
        cudaError_t e = launch_toom_eval(K, t, grid, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "Toom evaluation launch");
        const uint64_t *ca = reinterpret_cast<const uint64_t *>(opnd);
        st = strided_on_slot(ctx, slot, reinterpret_cast<uint64_t *>(prod), ca, ca + t.E / 2u, NP * g, t.E, t.E, 0u,
                             GF2X_BATCH_PERSISTENT, s);
        if (st != GF2X_OK)
            return st;
        e = launch_toom_interp(K, t, grid, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "Toom interpolation launch");
    }
    return scratch_release(ctx, s);
}

extern "C" gf2x_status gf2x_mul_toom4(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n,
                                      size_t count, size_t stride_in, size_t stride_out, uint32_t flags,
                                      gf2x_stream stream)
{
    return run_toom(ctx, 4u, out, a, b, n, count, stride_in, stride_out, flags, stream);
}

extern "C" gf2x_status gf2x_mul_toom5(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n,
                                      size_t count, size_t stride_in, size_t stride_out, uint32_t flags,
                                      gf2x_stream stream)
{
    return run_toom(ctx, 5u, out, a, b, n, count, stride_in, stride_out, flags, stream);
}

extern "C" gf2x_status gf2x_mulmod_shared_tc(gf2x_ctx *ctx, uint64_t *r, const uint64_t *a, const uint64_t *b,
                                             uint32_t n, size_t count, size_t stride_b, size_t stride_r,
                                             gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (n < 1 || n > kTcMaxN || !(n & 1u))
        return fail(ctx, GF2X_EUNSUPPORTED, "tensor-core circulant products need an odd n in [1, 65535]");
    if (!r || !a || !b)
        return fail(ctx, GF2X_EINVAL, "null operand or result pointer");
    if (((uintptr_t)r | (uintptr_t)a | (uintptr_t)b) & 7u)
        return fail(ctx, GF2X_EINVAL, "operands and results must be 8-byte aligned");
    const size_t L = (n + 63) / 64;
    if (count > 1 && (stride_b < L || stride_r < L))
        return fail(ctx, GF2X_EINVAL, "stride smaller than the operand or result size");
    if (count > 0x7fffffffull)
        return fail(ctx, GF2X_EINVAL, "batch too large");
    const size_t r_bytes = 8 * ((count - 1) * stride_r + L);
    if (ranges_overlap(r, r_bytes, a, 8 * L) || ranges_overlap(r, r_bytes, b, 8 * ((count - 1) * stride_b + L)))
        return fail(ctx, GF2X_EINVAL, "result overlaps an operand");
    TcShape sh;
    if (!tc_shape(n, count, &sh))
        return fail(ctx, GF2X_EUNSUPPORTED, "no tensor-core shape for this n");
    // scratch: R, then per group of products (a multiple of 128) the fp4
    // chunks of b and the parities in position-index order
    const size_t rbytes = (sh.rseq_bytes + 255) / 256 * 256;
    const size_t cap = scratch_cap(ctx);
    size_t group = (count + 127) / 128 * 128;
    while (group > 128 && rbytes + tc_group_bytes(sh, group) > cap)
        group = (group / 2 + 127) / 128 * 128;
    const size_t want = rbytes + tc_group_bytes(sh, std::min(group, count));
    if (want > cap)
        return fail(ctx, GF2X_ENOMEM, "scratch too small for one tile of 128 products");
    cudaStream_t s = (cudaStream_t)stream;
    gf2x_status st = scratch_acquire(ctx, want, s);
    if (st != GF2X_OK)
        return st;
    uint8_t *base = reinterpret_cast<uint8_t *>(ctx->ub);
    cudaError_t e = launch_tc_rseq(a, n, sh, base, ctx->sm_count, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "tensor-core sequence launch");
    for (size_t c0 = 0; c0 < count; c0 += group) {
        const size_t g = std::min(group, count - c0);
        e = launch_tc_group(b + c0 * stride_b, stride_b, r + c0 * stride_r, stride_r, n, (uint32_t)g, sh, base,
                            base + rbytes, ctx->err_dev, ctx->sm_count, s);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "tensor-core product launch");
    }
    return scratch_release(ctx, s);
}

// k rows of `width` limbs, `dpitch` / `spitch` limbs apart.
static cudaError_t copy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t k,
                             cudaMemcpyKind kind, cudaStream_t st)
{
    if (dpitch == width && spitch == width)
        return cudaMemcpyAsync(dst, src, 8 * width * k, kind, st);
    return cudaMemcpy2DAsync(dst, 8 * dpitch, src, 8 * spitch, 8 * width, k, kind, st);
}

static gf2x_status host_pipe_ready(gf2x_ctx *ctx, size_t bytes)
{
    HostPipe &hp = ctx->hp;
    cudaError_t e = cudaSuccess;
    if (!hp.ready)
        return fail(ctx, GF2X_ECUDA, "host pipeline streams missing");
    if (bytes > hp.bytes && ctx->fixed)
        return fail(ctx, GF2X_ENOMEM, "fixed workspace too small for one product of the host pipeline");
    if (bytes > hp.bytes) {
        if (hp.buf) {
            e = cudaFree(hp.buf);   // synchronizes the device: no copy or product still uses it
            hp.buf = nullptr;
            hp.bytes = 0;
            if (e != cudaSuccess)
                return cuda_fail(ctx, e, "host pipeline buffers");
        }
        e = ctx_malloc(ctx, (void **)&hp.buf, bytes);
        if (e != cudaSuccess) {
            hp.buf = nullptr;
            return e == cudaErrorMemoryAllocation ? fail(ctx, GF2X_ENOMEM, "host pipeline buffers")
                                                  : cuda_fail(ctx, e, "host pipeline buffers");
        }
        hp.bytes = bytes;
    }
    return GF2X_OK;
}

extern "C" gf2x_status gf2x_mul_strided_host(gf2x_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b,
                                             uint32_t n, size_t count, size_t stride_in, size_t stride_out,
                                             uint32_t flags, gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (n < 1 || n > GF2X_MAX_N)
        return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 131072]");
    const bool inputs_ready = (flags & GF2X_HOST_INPUTS_READY) != 0;
    flags &= ~(uint32_t)GF2X_HOST_INPUTS_READY;
    gf2x_status st = check_operands(ctx, out, a, b, n, flags, count, stride_in, stride_out);
    if (st != GF2X_OK)
        return st;
    const size_t L = (n + 63) / 64;
    const size_t Lo = (flags & GF2X_REDUCE) ? L : (size_t)((2ull * n - 1 + 63) / 64);
    // host strides (a single row may have any stride); the device rows are packed
    const size_t hi = count > 1 ? stride_in : L, ho = count > 1 ? stride_out : Lo;
    // chunks: the first chunk's copy in and the last one's copy out are not
    // overlapped with products; at 4096 x 17669 eight chunks measured slower
    // than four (5.40 vs 6.61 M products/s end to end: per-chunk launches)
    const size_t nchunk = count >= 2048 ? 4 : (count >= 512 ? 2 : 1);
    size_t K = (count + nchunk - 1) / nchunk;
    if (ctx->fixed)   // as many products per chunk as two buffer sets in the fixed workspace hold
        K = std::min(K, std::max<size_t>(1, ctx->hp.bytes / (2 * 8 * (2 * L + Lo))));
    const size_t in_w = K * L, set_w = 2 * in_w + K * Lo;
    st = host_pipe_ready(ctx, 2 * set_w * sizeof(uint64_t));
    if (st != GF2X_OK)
        return st;
    HostPipe &hp = ctx->hp;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!inputs_ready) {   // the operand copies wait for the work already on `stream`
        e = cudaEventRecord(hp.entry, s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(hp.h2d, hp.entry, 0);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "host pipeline ordering");
    }
    for (size_t c = 0, c0 = 0; c0 < count; ++c, c0 += K) {
        const int p = (int)(c & 1);
        const size_t k = std::min(K, count - c0);
        uint64_t *da = hp.buf + p * set_w, *db = da + in_w, *dout = db + in_w;
        // the set's previous product (this call or an earlier one) has read its operands
        e = cudaStreamWaitEvent(hp.h2d, hp.done[p], 0);
        // packed host rows: one flat copy; padded rows: one pitched copy moving
        // only the L limbs of each row
        if (e == cudaSuccess)
            e = copy_rows(da, L, a + c0 * hi, hi, L, k, cudaMemcpyHostToDevice, hp.h2d);
        if (e == cudaSuccess)
            e = copy_rows(db, L, b + c0 * hi, hi, L, k, cudaMemcpyHostToDevice, hp.h2d);
        if (e == cudaSuccess)
            e = cudaEventRecord(hp.in[p], hp.h2d);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(hp.comp[p], hp.in[p], 0);
        if (e == cudaSuccess)   // the set's previous results have been copied out
            e = cudaStreamWaitEvent(hp.comp[p], hp.out[p], 0);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "host pipeline copy in");
        // one CTA per product (end to end 8.29 against 8.27 M/s for persistent
        // launches at 4096 x 17669, 1.11 against 1.06 at 2048 x 57637)
        st = gf2x_mul_strided(ctx, dout, da, db, n, k, L, Lo, flags, 0u, hp.comp[p]);
        if (st != GF2X_OK)
            return st;
        e = cudaEventRecord(hp.done[p], hp.comp[p]);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(hp.d2h, hp.done[p], 0);
        if (e == cudaSuccess)   // the limbs between result rows are left as they are
            e = copy_rows(out + c0 * ho, ho, dout, Lo, Lo, k, cudaMemcpyDeviceToHost, hp.d2h);
        if (e == cudaSuccess)
            e = cudaEventRecord(hp.out[p], hp.d2h);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "host pipeline copy out");
    }
    e = cudaStreamWaitEvent(s, hp.out[0], 0);
    if (e == cudaSuccess && count > K)
        e = cudaStreamWaitEvent(s, hp.out[1], 0);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "host pipeline completion");
    return GF2X_OK;
}

// Take a staging buffer of at least `count` items; waits (host) for the
// buffer's previous copy to finish before it is reused.
static gf2x_status take_staging(gf2x_ctx *ctx, size_t count, Staging **out)
{
    Staging &r = ctx->ring[ctx->ring_next];
    ctx->ring_next = (ctx->ring_next + 1) % kRing;
    if (r.pending) {
        cudaError_t e = cudaEventSynchronize(r.done);
        if (e != cudaSuccess)
            return cuda_fail(ctx, e, "staging wait");
        r.pending = false;
    }
    if (r.cap < count) {
        if (ctx->fixed)
            return fail(ctx, GF2X_ENOMEM, "batch larger than the fixed item staging");
        size_t cap = std::max<size_t>(count, 1024);
        if (r.host)
            cudaFreeHost(r.host);
        if (r.dev)
            cudaFree(r.dev);
        r.host = nullptr;
        r.dev = nullptr;
        r.cap = 0;
        if (ctx_malloc_host(ctx, (void **)&r.host, cap * sizeof(DevItem)) != cudaSuccess ||
            ctx_malloc(ctx, (void **)&r.dev, cap * sizeof(DevItem)) != cudaSuccess)
            return fail(ctx, GF2X_ENOMEM, "staging allocation");
        r.cap = cap;
    }
    if (!r.done)
        return fail(ctx, GF2X_ECUDA, "staging event missing");
    *out = &r;
    return GF2X_OK;
}

extern "C" gf2x_status gf2x_mul_batched(gf2x_ctx *ctx, const gf2x_item *items, size_t count, uint32_t batch_flags,
                                        gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (!items)
        return fail(ctx, GF2X_EINVAL, "null item array");
    if (batch_flags & ~(uint32_t)(GF2X_BATCH_PERSISTENT | GF2X_BATCH_ITEMS_ON_DEVICE | GF2X_BATCH_LARGEST_FIRST |
                                  GF2X_BATCH_DYNAMIC))
        return fail(ctx, GF2X_EINVAL, "unknown batch flag");
    const bool dynamic = (batch_flags & GF2X_BATCH_DYNAMIC) != 0;
    if (count > 0xffffffffull)
        return fail(ctx, GF2X_EINVAL, "batch too large");
    cudaStream_t s = (cudaStream_t)stream;
    const bool persistent = (batch_flags & GF2X_BATCH_PERSISTENT) != 0;
    if (batch_flags & GF2X_BATCH_ITEMS_ON_DEVICE) {
        // one launch over the caller's device array; plans are looked up by n
        // on the device, so every size must have been prepared beforehand
        if (ctx->device_set.empty())
            return fail(ctx, GF2X_EINVAL, "no prepared sizes: call gf2x_ctx_prepare first");
        uint32_t S = 0;
        unsigned threads = 0;
        uint32_t smem_words = 0;
        for (uint32_t n : ctx->device_set) {
            uint32_t slot;
            gf2x_status st = plan_for(ctx, n, s, &slot);
            if (st != GF2X_OK)
                return st;
            const GPlan &P = ctx->plans_host[slot];
            if (P.split)
                return fail(ctx, GF2X_EUNSUPPORTED, "split plans run through gf2x_mul_strided / gf2x_mul only");
            if (S && P.S != S)
                return fail(ctx, GF2X_EUNSUPPORTED, "device item batches need one leaf size over the prepared plans");
            S = P.S;
            threads = std::max(threads, P.threads);
            smem_words = std::max(smem_words, P.smem_words);
        }
        static_assert(sizeof(gf2x_item) == sizeof(DevItem), "gf2x_item and DevItem share a layout");
        LaunchArgs args;
        memset(&args, 0, sizeof(args));
        args.plans = ctx->plans_dev;
        args.items = reinterpret_cast<const DevItem *>(items);
        args.count = (uint32_t)count;
        args.mode = kItemsUser;
        args.err = ctx->err_dev;
        args.plan_of_n = ctx->plan_of_n_dev;
        return launch(ctx, args, S, threads, 4ull * smem_words, count, persistent, s, dynamic);
    }

    if (ctx->fixed && count > kFixedStagingItems) {   // pieces that fit the fixed item staging
        for (size_t off = 0; off < count; off += kFixedStagingItems) {
            gf2x_status st = gf2x_mul_batched(ctx, items + off, std::min(kFixedStagingItems, count - off),
                                              batch_flags, stream);
            if (st != GF2X_OK)
                return st;
        }
        return GF2X_OK;
    }
    // resolve plans and check every item
    auto &dv = ctx->scratch_items;
    auto &Ss = ctx->scratch_S;
    dv.resize(count);
    Ss.resize(count);
    for (size_t i = 0; i < count; ++i) {
        const gf2x_item &it = items[i];
        if (it.n < 1 || it.n > GF2X_MAX_N)
            return fail(ctx, GF2X_EUNSUPPORTED, "item n outside [1, 131072]");
        gf2x_status st = check_operands(ctx, it.out, it.a, it.b, it.n, it.flags, 1, 0, 0);
        if (st != GF2X_OK)
            return st;
        uint32_t slot;
        st = plan_for(ctx, it.n, s, &slot);
        if (st != GF2X_OK)
            return st;
        dv[i] = DevItem{it.a, it.b, it.out, slot, it.flags};
        // launch groups: one per leaf size for in-CTA plans, one per plan for split plans
        Ss[i] = ctx->plans_host[slot].split ? (0x80000000u | slot) : ctx->plans_host[slot].S;
    }
    // group by leaf size (one launch per group), largest n first if asked
    std::vector<size_t> order(count);
    for (size_t i = 0; i < count; ++i)
        order[i] = i;
    const bool largest_first = (batch_flags & GF2X_BATCH_LARGEST_FIRST) != 0;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        if (Ss[x] != Ss[y])
            return Ss[x] < Ss[y];
        if (largest_first)
            return ctx->plans_host[dv[x].plan].n > ctx->plans_host[dv[y].plan].n;
        return false;
    });
    Staging *stg = nullptr;
    gf2x_status st = take_staging(ctx, count, &stg);
    if (st != GF2X_OK)
        return st;
    for (size_t i = 0; i < count; ++i)
        stg->host[i] = dv[order[i]];
    cudaError_t e = cudaMemcpyAsync(stg->dev, stg->host, count * sizeof(DevItem), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "item upload");
    e = cudaEventRecord(stg->done, s);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "event record");
    stg->pending = true;
    size_t g0 = 0;
    while (g0 < count) {
        const uint32_t S = Ss[order[g0]];
        size_t g1 = g0;
        if (S & 0x80000000u) {   // a split plan: its three launches over this group's items
            while (g1 < count && Ss[order[g1]] == S)
                ++g1;
            LaunchArgs ta;
            memset(&ta, 0, sizeof(ta));
            ta.plans = ctx->plans_dev;
            ta.items = stg->dev + g0;
            ta.mode = kItemsArray;
            st = run_split_args(ctx, S & 0x7fffffffu, ta, g1 - g0, persistent, s);
            if (st != GF2X_OK)
                return st;
            g0 = g1;
            continue;
        }
        unsigned threads = 0;
        uint32_t smem_words = 0;
        while (g1 < count && Ss[order[g1]] == S) {
            const GPlan &P = ctx->plans_host[dv[order[g1]].plan];
            threads = std::max(threads, P.threads);
            smem_words = std::max(smem_words, P.smem_words);
            ++g1;
        }
        LaunchArgs args;
        memset(&args, 0, sizeof(args));
        args.plans = ctx->plans_dev;
        args.items = stg->dev + g0;
        args.count = (uint32_t)(g1 - g0);
        args.mode = kItemsArray;
        args.err = ctx->err_dev;
        st = launch(ctx, args, S, threads, 4ull * smem_words, g1 - g0, persistent, s, dynamic);
        if (st != GF2X_OK)
            return st;
        g0 = g1;
    }
    return GF2X_OK;
}

extern "C" gf2x_status gf2x_ctx_sync_status(gf2x_ctx *ctx, gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "stream synchronize");
    uint32_t flags = 0;
    e = cudaMemcpy(&flags, ctx->err_dev, sizeof(flags), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "error word read");
    if (flags) {
        cudaMemset(ctx->err_dev, 0, sizeof(uint32_t));
        char buf[128];
        if (flags & kErrTimeout) {
            snprintf(buf, sizeof(buf), "a bounded wait in a kernel ran out (flags 0x%x)", flags);
            return fail(ctx, GF2X_ETIMEOUT, buf);
        }
        snprintf(buf, sizeof(buf), "checked kernel reported invariant violation flags 0x%x", flags);
        return fail(ctx, GF2X_EDEVICE, buf);
    }
    return GF2X_OK;
}

extern "C" gf2x_status gf2x_copy_rows(gf2x_ctx *ctx, const gf2x_copy_row *rows, size_t count, gf2x_stream stream)
{
    if (!ctx)
        return GF2X_EINVAL;
    if (count == 0)
        return GF2X_OK;
    if (!rows)
        return fail(ctx, GF2X_EINVAL, "null row list");
    cudaError_t e = launch_copy_rows(rows, count, ctx->sm_count, (cudaStream_t)stream);
    return e == cudaSuccess ? GF2X_OK : cuda_fail(ctx, e, "row copy launch");
}

extern "C" gf2x_status gf2x_ctx_wait(gf2x_ctx *ctx, gf2x_stream stream, uint32_t timeout_ms)
{
    if (!ctx)
        return GF2X_EINVAL;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        const cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
        if (e == cudaSuccess)
            break;
        if (e != cudaErrorNotReady)
            return cuda_fail(ctx, e, "stream query");
        if (std::chrono::steady_clock::now() >= deadline)
            return fail(ctx, GF2X_ETIMEOUT, "the stream's work did not finish within the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return gf2x_ctx_sync_status(ctx, stream);   // complete: the error word and asynchronous errors
}

extern "C" const char *gf2x_ctx_last_error(gf2x_ctx *ctx)
{
    if (!ctx)
        return "null context";
    return ctx->last_error.c_str();
}

extern "C" gf2x_status gf2x_ctx_prepare(gf2x_ctx *ctx, const uint32_t *sizes, size_t count, gf2x_stream stream)
{
    if (!ctx || (count && !sizes))
        return GF2X_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint32_t> next(sizes, sizes + count);
    for (uint32_t n : next)
        if (n < 1 || n > GF2X_MAX_N)
            return fail(ctx, GF2X_EUNSUPPORTED, "n outside [1, 131072]");
    // withdraw the previous device set, then publish the new one
    for (uint32_t n : ctx->device_set) {
        gf2x_status st = publish_plan(ctx, n, kNoPlan, s);
        if (st != GF2X_OK)
            return st;
    }
    ctx->device_set.clear();
    for (uint32_t n : next) {
        uint32_t slot;
        gf2x_status st = plan_for(ctx, n, s, &slot);
        if (st != GF2X_OK)
            return st;
        st = publish_plan(ctx, n, slot, s);
        if (st != GF2X_OK)
            return st;
        if (!in_device_set(ctx, n))
            ctx->device_set.push_back(n);
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? GF2X_OK : cuda_fail(ctx, e, "prepare");
}

extern "C" gf2x_status gf2x_ctx_launch_shape(gf2x_ctx *ctx, uint32_t n, uint32_t *threads, uint32_t *smem_bytes,
                                             uint32_t *blocks_per_sm, uint32_t *sm_count)
{
    if (!ctx)
        return GF2X_EINVAL;
    uint32_t slot;
    gf2x_status st = plan_for(ctx, n, nullptr, &slot);
    if (st != GF2X_OK)
        return st;
    auto chs = ctx->child_of.find(slot);
    const GPlan &P = ctx->plans_host[chs != ctx->child_of.end() ? chs->second : slot];
    int per_sm = 0;
    cudaError_t e = preparer_for(P.S)(&per_sm, P.threads, 4ull * P.smem_words);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "occupancy query");
    if (threads)
        *threads = P.threads;
    if (smem_bytes)
        *smem_bytes = 4u * P.smem_words;
    if (blocks_per_sm)
        *blocks_per_sm = (uint32_t)per_sm;
    if (sm_count)
        *sm_count = (uint32_t)ctx->sm_count;
    return GF2X_OK;
}

// Plan database: text lines "n batch_bucket spec [anything]"; '#' starts a comment.
// For every n the entry whose bucket is nearest (in log2) to batch_hint wins.
extern "C" gf2x_status gf2x_ctx_load_plan_db(gf2x_ctx *ctx, const char *path, size_t batch_hint)
{
    if (!ctx || !path)
        return GF2X_EINVAL;
    FILE *f = fopen(path, "r");
    if (!f)
        return fail(ctx, GF2X_EINVAL, std::string("cannot open plan database ") + path);
    struct Best {
        double dist;
        gf2x_plan_spec spec;
    };
    std::unordered_map<uint32_t, Best> best;
    char line[512];
    const double want = std::log2((double)std::max<size_t>(1, batch_hint));
    gf2x_status st = GF2X_OK;
    while (fgets(line, sizeof(line), f)) {
        char *hash = strchr(line, '#');
        if (hash)
            *hash = '\0';
        unsigned long n = 0, bucket = 0;
        char spec_text[256];
        if (sscanf(line, "%lu %lu %255s", &n, &bucket, spec_text) != 3)
            continue;
        gf2x_plan_spec spec;
        if (parse_spec(spec_text, &spec) != GF2X_OK || n < 1 || n > GF2X_MAX_N || bucket < 1) {
            st = GF2X_EINVAL;
            continue;
        }
        const double d = std::fabs(std::log2((double)bucket) - want);
        auto it = best.find((uint32_t)n);
        if (it == best.end() || d < it->second.dist)
            best[(uint32_t)n] = Best{d, spec};
    }
    fclose(f);
    for (auto &kv : best) {
        gf2x_status s2 = gf2x_ctx_set_plan(ctx, kv.first, &kv.second.spec);
        if (s2 != GF2X_OK)
            st = s2;
    }
    if (st != GF2X_OK)
        return fail(ctx, st, "some plan database entries were rejected");
    return GF2X_OK;
}
