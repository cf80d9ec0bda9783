// noalloc.cu -- gf2x_mul_strided_static: the split-plan product with its
// scratch and plans in file-scope device arrays, for callers that cannot
// allocate device memory (see the header).  Nothing here allocates.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "gf2x_gb300.h"
#include "launchers.h"
#include "plan.h"
#include "plan_host.h"

using namespace gf2x;

namespace {

constexpr int kMaxDevices = 64;

// Held by every GPU that loads the library, until the process exits.
__device__ __align__(256) uint32_t g_static_scratch[GF2X_STATIC_SCRATCH_BYTES / 4];
__device__ __align__(256) GPlan g_static_plans[2];   // [0] top level, [1] children

struct StaticSetup {
    bool done = false;
    uint32_t *scratch = nullptr;   // device address of g_static_scratch
    GPlan *plans = nullptr;        // device address of g_static_plans
};

StaticSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Both plans of one call, passed by value as a kernel parameter (3.3 KB,
// within the 4 KB parameter space): the launch copies them, so no host
// buffer has to outlive the call.
struct StaticPlans {
    GPlan p[2];
};
static_assert(sizeof(StaticPlans) <= 4096, "plans must fit the kernel parameter space");

// Writes the call's plans into g_static_plans (named directly: device code
// may use the array's own name), one 32-bit word per thread.
__global__ void __launch_bounds__(256) static_plans_kernel(const StaticPlans plans)
{
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&plans);
    uint32_t *dst = reinterpret_cast<uint32_t *>(g_static_plans);
    for (uint32_t w = threadIdx.x; w < sizeof(StaticPlans) / 4; w += blockDim.x)
        dst[w] = src[w];
}

// Once per device, with the device current: the arrays' device addresses
// (the host-side names are stand-ins, not device pointers) and the kernels'
// dynamic shared-memory limits.
gf2x_status setup_current_device(StaticSetup **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return GF2X_ECUDA;
    if (dev < 0 || dev >= kMaxDevices)
        return GF2X_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    StaticSetup &st = g_setup[dev];
    if (!st.done) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p)
            return GF2X_ECUDA;
        st.scratch = static_cast<uint32_t *>(p);
        p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_plans) != cudaSuccess || !p)
            return GF2X_ECUDA;
        st.plans = static_cast<GPlan *>(p);
        for (uint32_t S : kLeafSizes)
            if (preparer_for(S)(nullptr, 0, 0) != cudaSuccess)
                return GF2X_ECUDA;
        if (prepare_split() != cudaSuccess)
            return GF2X_ECUDA;
        st.done = true;
    }
    *out = &st;
    return GF2X_OK;
}

bool overlaps(const void *p, size_t pb, const void *q, size_t qb)
{
    const uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + qb && b < a + pb;
}

}  // namespace

extern "C" gf2x_status gf2x_mul_strided_static(uint64_t *out, const uint64_t *a, const uint64_t *b, uint32_t n,
                                               size_t count, size_t stride_in, size_t stride_out, uint32_t flags,
                                               const gf2x_plan_spec *spec, gf2x_stream stream)
{
    if (n < 1 || n > GF2X_MAX_N)
        return GF2X_EUNSUPPORTED;
    if (count == 0)
        return GF2X_OK;
    if (!out || !a || !b || (((uintptr_t)out | (uintptr_t)a | (uintptr_t)b) & 7u) || (flags & ~GF2X_REDUCE))
        return GF2X_EINVAL;
    if (count > 0x7fffffffull)
        return GF2X_EUNSUPPORTED;
    const size_t L = (n + 63) / 64;
    const size_t Lo = (flags & GF2X_REDUCE) ? L : (size_t)((2ull * n - 1 + 63) / 64);
    if (count > 1 && (stride_in < L || stride_out < Lo))
        return GF2X_EINVAL;
    const size_t in_bytes = 8 * ((count - 1) * stride_in + L), out_bytes = 8 * ((count - 1) * stride_out + Lo);
    if (overlaps(out, out_bytes, a, in_bytes) || overlaps(out, out_bytes, b, in_bytes))
        return GF2X_EINVAL;

    gf2x_plan_spec sp;
    if (spec) {
        if (!spec->split_top)
            return GF2X_EINVAL;
        sp = *spec;
    } else if (default_split_spec(n, &sp) != GF2X_OK) {
        return GF2X_EUNSUPPORTED;
    }
    StaticPlans sp2;
    GPlan *host = sp2.p;
    gf2x_plan_info info;
    gf2x_status st = build_plan(n, &sp, &host[0], &info, &host[1]);
    if (st != GF2X_OK)
        return st;
    if (!host[0].split || info.scratch_bytes == 0)
        return GF2X_EINVAL;
    if (count * info.scratch_bytes > GF2X_STATIC_SCRATCH_BYTES)
        return GF2X_EUNSUPPORTED;   // beyond the static scratch: split the batch

    StaticSetup *su = nullptr;
    st = setup_current_device(&su);
    if (st != GF2X_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the plans travel in the upload kernel's parameters, ordered before the
    // products on the same stream
    static_plans_kernel<<<1, 256, 0, s>>>(sp2);
    if (cudaGetLastError() != cudaSuccess)
        return GF2X_ECUDA;

    const GPlan &T = host[0], &C = host[1];
    const uint32_t nch = T.lev[0].nch, E = T.lev[0].E;
    LaunchArgs ta;
    memset(&ta, 0, sizeof(ta));
    ta.plans = su->plans;
    ta.base = DevItem{a, b, out, 0u, flags};
    ta.stride_in = stride_in;
    ta.stride_out = stride_out;
    ta.count = (uint32_t)count;
    ta.mode = kItemsStrided;
    ta.err = nullptr;   // no error word: see the header (device refusals cannot arise here)
    if (launch_split_eval(ta, su->scratch, (unsigned)count, T.threads, 4ull * T.smem_words, s) != cudaSuccess)
        return GF2X_ECUDA;
    LaunchArgs ca;
    memset(&ca, 0, sizeof(ca));
    ca.plans = su->plans;
    ca.base = DevItem{reinterpret_cast<const uint64_t *>(su->scratch),
                      reinterpret_cast<const uint64_t *>(su->scratch + E), reinterpret_cast<uint64_t *>(su->scratch),
                      1u, 0u};
    ca.stride_in = E;
    ca.stride_out = E;
    ca.count = (uint32_t)(count * nch);
    ca.mode = kItemsStrided;
    ca.err = nullptr;
    LaunchFn child = launcher_for(C.S);
    if (!child || child(ca, (unsigned)(count * nch), C.threads, 4ull * C.smem_words, s) != cudaSuccess)
        return GF2X_ECUDA;
    if (launch_split_interp(ta, su->scratch, (unsigned)count, T.threads, 4ull * T.smem_words, s) != cudaSuccess)
        return GF2X_ECUDA;
    return GF2X_OK;
}
