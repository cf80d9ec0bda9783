// tc_circulant.cu -- r_j = a * b_j mod (X^n - 1) for ONE polynomial a and
// many b_j (the shared-operand batch: an HQC/BIKE public key times many
// vectors, Sec. 1) as an integer GEMM on the fifth-generation tensor cores.
//
// Sec. 1 maps the product in F2[X]/(X^n - 1) to the circulant matrix of a
// times the vector b: r[p] = sum_k a[(p - k) mod n] b[k] over F2.  With one a
// for the whole batch this is D = B * T with B = [b_j] (count x n, 0/1) and
// T[k][p] = a[(p - k) mod n], and r_j[p] = D[j][p] mod 2.  The GEMM runs in
// block-scaled fp4 (tcgen05.mma kind::mxf4, every scale factor 1.0): the
// operands are the bits as e2m1 0.0 / 1.0 (nibble 0 / 2), the counts
// accumulate exactly in fp32 TMEM (at most n < 2^24), and the product bit
// is the count's parity.
//
// The circulant operand costs nothing per MMA.  Its row for output position
// p is a reversed window of a, and the rows of one MMA are the positions
// p0, p0 - 32, p0 - 64, ... (mod n): row q then starts exactly 16 bytes (32
// fp4 elements) after row q - 1 in ONE nibble sequence R[t] = a[(p0 - t) mod
// n], so a shared-memory descriptor with a 16-byte leading and a 128-byte
// stride offset reads the whole 224 x 64 operand tile out of R.  For odd n
// the stride -32 mod n visits every position once, so the positions are
// enumerated as q = 0, 1, 2, ... with p(q) = (n - 1 - 32 q) mod n.
//
// Kernels (all on the caller's stream):
//  tc_rseq_kernel     R, the nibble sequence of a (once per call);
//  tc_unpack_kernel   the b rows as fp4 nibbles in the UMMA K-major layout,
//                     one 4 KB chunk per tile of 128 rows and K-step of 64;
//  tc_gemm_kernel     persistent, one CTA per SM: a bulk-copy producer
//                     thread, an MMA thread, four epilogue warps reading the
//                     counts from TMEM; each unit is 128 products x 224
//                     positions over all n inputs, and TMEM holds two
//                     accumulator buffers, so a unit's parities are read
//                     while the next unit accumulates; the parities go out
//                     in position-index (q) order;
//  tc_assemble_kernel q order -> bit order: r_j[p] = parity[j][q(p)], the
//                     row staged in shared memory, a funnel-shift gather of
//                     each bit column and a warp butterfly transpose per 32
//                     output words.
// Constant time: every loop bound, address and branch depends on n, count
// and thread indices only; operand bits flow through data paths.
// Every wait on a barrier is bounded (globaltimer); on a timeout the CTA
// records kErrTimeout, drains its copies and MMAs (bounded) and frees TMEM.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "gf2x_gb300.h"
#include "launchers.h"

namespace gf2x {

namespace {

constexpr uint32_t kTcThreads = 256;          // warps: 0 producer, 1 MMA, 2-3 idle, 4-7 epilogue
// Pipeline shape (compile-time): the MMAs per barrier wait and commit are
// what counts -- measured at 4096 x 17669: 2 K-steps per stage 6.0 M/s, 4:
// 8.4, 8: 12.8, 16: 13.0 -- while the ring depth barely matters.
#ifndef GF2X_TC_KS
#define GF2X_TC_KS 16
#endif
#ifndef GF2X_TC_RING
#define GF2X_TC_RING 2
#endif
constexpr uint32_t kKS = GF2X_TC_KS;          // K-steps (of 64 inputs) per ring stage
constexpr uint32_t kRing = GF2X_TC_RING;      // A stages
constexpr uint32_t kChunk = 4096;             // bytes of one K-step of A: 128 rows x 64 fp4
constexpr uint32_t kStage = kKS * kChunk;
constexpr uint32_t kNT = 224;                 // N of one MMA = positions per unit (7 words of parities)
constexpr uint32_t kNU = kNT;
constexpr uint32_t kSfCol = 2 * kNT;          // TMEM: two accumulator buffers, then the scale factors (all 1.0)
constexpr uint32_t kRWinMax = 16 * (kNU - 1) + 32 * (kTcMaxN / 64);   // bytes of an R window
constexpr uint32_t kROff = kRing * kStage;
constexpr uint32_t kRBytes = (kRWinMax + 127) / 128 * 128;
constexpr uint32_t kBarOff = kROff + 2 * kRBytes;
constexpr uint32_t kSmemBytes = kBarOff + 512;   // > 114 KB: one CTA per SM (the whole TMEM)
constexpr uint64_t kWaitLimitNs = 2000000000ull; // 2 s per wait

// e2m1 1.0 = 0b0010; element 2i in the low nibble of byte i
__device__ __forceinline__ uint32_t spread8(uint32_t x)
{
    uint32_t t = x & 0xffu;
    t = (t | (t << 12)) & 0x000f000fu;
    t = (t | (t << 6)) & 0x03030303u;
    t = (t | (t << 3)) & 0x11111111u;
    return t << 1;
}

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtime()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// UMMA shared-memory descriptor, no swizzle: start, leading (K) byte offset,
// stride (M/N, 8-row group) byte offset, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3ffffu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | ((uint64_t)1 << 46);
}

// kind::mxf4 instruction descriptor: A and B e2m1 (1), K-major, N, M = 128,
// scale factors ue8m0 (bit 23), scale-factor ids 0.
constexpr uint32_t kIdesc = (1u << 7) | (1u << 10) | ((kNT >> 3) << 17) | (1u << 23) | ((128u >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// One test of a barrier phase (try_wait may suspend the thread briefly when
// the phase is not complete yet; a non-suspending test_wait measured the same).
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait on a barrier phase; false on a timeout or when another role
// has aborted (the shared abort word).  The clock is read only once the
// first test has failed; `nap` > 0 sleeps between tests (threads that wait
// long and have nothing else to issue).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t *abort_flag,
                                          uint32_t nap = 0)
{
    if (mbar_test(bar, parity))
        return true;
    const uint64_t t0 = gtime();
    for (;;) {
        if (mbar_test(bar, parity))
            return true;
        if (*abort_flag)
            return false;
        if (gtime() - t0 > kWaitLimitNs)
            return false;
        if (nap)
            __nanosleep(nap);
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mma_fp4(uint32_t d, uint64_t a, uint64_t b, uint32_t sfa, uint32_t sfb, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n}"
                 ::"r"(d), "l"(a), "l"(b), "r"(kIdesc), "r"(acc), "r"(sfa), "r"(sfb));
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

}  // namespace

// R[t] = a[(n - 1 - t) mod n] as fp4 nibbles, `words` 32-bit words of 8.
__global__ void __launch_bounds__(256) tc_rseq_kernel(const uint64_t *__restrict__ a, uint32_t n,
                                                      uint32_t *__restrict__ r, uint32_t words)
{
    const uint32_t top = n - 1;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        uint32_t i = (uint32_t)((top + (uint64_t)n - (8ull * w) % n) % n);   // (n-1-8w) mod n
#pragma unroll
        for (uint32_t e = 0; e < 8; ++e) {
            bits |= (uint32_t)((a[i >> 6] >> (i & 63u)) & 1u) << e;
            i = i == 0 ? top : i - 1;     // the index only, never the bit, decides
        }
        r[w] = spread8(bits);
    }
}

// b rows -> A chunks: chunk (tile, s) holds rows tile*128 .. +127, inputs
// 64 s .. 64 s + 63, core matrix (row group g, K half c) at g*256 + c*128,
// row r of it at + 16 r.  Rows past `count` and bits past n are zero.
__global__ void __launch_bounds__(256) tc_unpack_kernel(const uint64_t *__restrict__ b, size_t stride_b, uint32_t n,
                                                        uint32_t count, uint32_t S, uint32_t tiles,
                                                        uint8_t *__restrict__ chunks)
{
    const uint32_t L = (n + 63) / 64;
    const uint64_t top = (n & 63u) ? ((1ull << (n & 63u)) - 1ull) : ~0ull;
    const uint64_t total = (uint64_t)tiles * S * 128u;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t j = (uint32_t)(idx & 127u);
        const uint64_t ts = idx >> 7;
        const uint32_t s = (uint32_t)(ts % S), tile = (uint32_t)(ts / S);
        const uint32_t row = tile * 128u + j;
        uint64_t v = 0;
        if (row < count && s < L) {
            v = b[(size_t)row * stride_b + s];
            if (s == L - 1)
                v &= top;
        }
        const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
        uint4 q0, q1;
        q0.x = spread8(lo);
        q0.y = spread8(lo >> 8);
        q0.z = spread8(lo >> 16);
        q0.w = spread8(lo >> 24);
        q1.x = spread8(hi);
        q1.y = spread8(hi >> 8);
        q1.z = spread8(hi >> 16);
        q1.w = spread8(hi >> 24);
        uint8_t *base = chunks + ((uint64_t)tile * S + s) * kChunk + (j >> 3) * 256u + (j & 7u) * 16u;
        *reinterpret_cast<uint4 *>(base) = q0;
        *reinterpret_cast<uint4 *>(base + 128) = q1;
    }
}

struct TcGemmArgs {
    const uint8_t *chunks;    // A chunks (tc_unpack_kernel)
    const uint8_t *rseq;      // R (tc_rseq_kernel), 16-byte aligned
    uint32_t *qbits;          // per product qwords 32-bit words of parities in q order
    uint32_t *err;            // error word (kErrTimeout), may be null
    uint32_t S;               // K-steps (limbs of b)
    uint32_t V;               // position units per product tile
    uint32_t units;           // tiles x V
    uint32_t count;
    uint32_t qwords;          // V * kNU / 32
    uint32_t rwin;            // bytes of one unit's R window
};

__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const TcGemmArgs args)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t sbase = su32(sm);
    // barriers: full[kRing], empty[kRing], rfull[2], rempty[2], done[2], tfree[2], drain
    // (done / tfree per TMEM accumulator buffer: unit k uses buffer k & 1)
    const uint32_t bar0 = sbase + kBarOff;
    auto full = [&](uint32_t i) { return bar0 + 8u * i; };
    auto empty = [&](uint32_t i) { return bar0 + 8u * (kRing + i); };
    auto rfull = [&](uint32_t i) { return bar0 + 8u * (2 * kRing + i); };
    auto rempty = [&](uint32_t i) { return bar0 + 8u * (2 * kRing + 2 + i); };
    auto done = [&](uint32_t i) { return bar0 + 8u * (2 * kRing + 4 + i); };
    auto tfree = [&](uint32_t i) { return bar0 + 8u * (2 * kRing + 6 + i); };
    const uint32_t drain = bar0 + 8u * (2 * kRing + 8);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + kBarOff + 8u * (2 * kRing + 10));
    volatile uint32_t *abort_flag = tslot + 1;

    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < kRing; ++i) {
            mbar_init(full(i), 1);
            mbar_init(empty(i), 1);
        }
        for (uint32_t i = 0; i < 2; ++i) {
            mbar_init(rfull(i), 1);
            mbar_init(rempty(i), 1);
            mbar_init(done(i), 1);
            mbar_init(tfree(i), 4);   // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    if (warp >= 4) {   // scale factors: every byte 0x7F (ue8m0 1.0) in columns kSfCol..511
        const uint32_t v = 0x7f7f7f7fu;
        for (uint32_t c = kSfCol; c < 512u; c += 8)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};"
                         ::"r"(tmem + (((warp & 3u) * 32u) << 16) + c), "r"(v));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();

    const uint32_t S = args.S;
    bool failed = false;
    if (warp == 0 && lane == 0) {
        // ---- producer: R window per unit (two buffers), A chunks through the ring
        uint32_t g = 0, k = 0;
        for (uint32_t u = blockIdx.x; u < args.units && !failed; u += gridDim.x, ++k) {
            const uint32_t tile = u / args.V, v = u - tile * args.V;
            const uint32_t rb = k & 1u;
            if (k >= 2 && !mbar_wait(rempty(rb), ((k >> 1) - 1u) & 1u, abort_flag)) {
                failed = true;
                break;
            }
            bulk_load(sbase + kROff + rb * kRBytes, args.rseq + (size_t)v * (16u * kNU), args.rwin, rfull(rb));
            const uint8_t *src = args.chunks + (size_t)tile * S * kChunk;
            for (uint32_t s0 = 0; s0 < S; s0 += kKS, ++g) {   // one stage: up to kKS consecutive K-steps
                const uint32_t slot = g % kRing, ks = min(kKS, S - s0);
                if (g >= kRing && !mbar_wait(empty(slot), ((g / kRing) - 1u) & 1u, abort_flag)) {
                    failed = true;
                    break;
                }
                bulk_load(sbase + slot * kStage, src + (size_t)s0 * kChunk, ks * kChunk, full(slot));
            }
        }
        if (failed) {   // let the copies already issued land before the CTA can exit
            *abort_flag = 1;
            const uint64_t t0 = gtime();
            for (uint32_t h = (g > kRing ? g - kRing : 0); h < g; ++h)
                while (!mbar_test(full(h % kRing), (h / kRing) & 1u) && gtime() - t0 < 100000000ull) {
                }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        uint32_t g = 0, k = 0;
        bool issued = false;
        for (uint32_t u = blockIdx.x; u < args.units && !failed; u += gridDim.x, ++k) {
            const uint32_t rb = k & 1u, tb = k & 1u;
            // buffer tb was last read by the epilogue of unit k - 2
            if (!mbar_wait(rfull(rb), (k >> 1) & 1u, abort_flag) ||
                (k >= 2 && !mbar_wait(tfree(tb), ((k >> 1) - 1u) & 1u, abort_flag))) {
                failed = true;
                break;
            }
            fence_after();
            const uint32_t rwin = sbase + kROff + rb * kRBytes, d = tmem + tb * kNT;
            for (uint32_t s0 = 0; s0 < S; s0 += kKS, ++g) {
                const uint32_t slot = g % kRing, ks = min(kKS, S - s0);
                if (!mbar_wait(full(slot), (g / kRing) & 1u, abort_flag)) {
                    failed = true;
                    break;
                }
                fence_after();
                for (uint32_t i = 0; i < ks; ++i) {
                    const uint32_t s = s0 + i;
                    mma_fp4(d, sdesc(sbase + slot * kStage + i * kChunk, 128, 256), sdesc(rwin + 32u * s, 16, 128),
                            tmem + kSfCol, tmem + kSfCol + 16, s > 0);
                }
                issued = true;
                mma_commit(empty(slot));   // the stage is free once these MMAs have read it
            }
            if (failed)
                break;
            mma_commit(rempty(rb));
            mma_commit(done(tb));
        }
        if (failed) {
            *abort_flag = 1;
            if (issued) {   // wait (bounded) for the MMAs in flight before TMEM is freed
                mma_commit(drain);
                const uint64_t t0 = gtime();
                while (!mbar_test(drain, 0) && gtime() - t0 < 100000000ull) {
                }
            }
        }
    } else if (warp >= 4) {
        // ---- epilogue: counts -> parities, 224 positions of 32 products per warp
        const uint32_t wq = warp & 3u;
        uint32_t k = 0;
        for (uint32_t u = blockIdx.x; u < args.units; u += gridDim.x, ++k) {
            const uint32_t tile = u / args.V, v = u - tile * args.V, tb = k & 1u;
            const bool ok = mbar_wait(done(tb), (k >> 1) & 1u, abort_flag, 256);
            if (!__all_sync(0xffffffffu, ok)) {   // warp-uniform: the loads below are warp-synchronous
                failed = true;
                break;
            }
            fence_after();
            const uint32_t row = tile * 128u + wq * 32u + lane;
            uint32_t *dst = args.qbits + (size_t)row * args.qwords + (size_t)v * (kNU / 32u);
#pragma unroll 1
            for (uint32_t c = 0; c < kNU; c += 32) {
                uint32_t r[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(tmem + ((wq * 32u) << 16) + tb * kNT + c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                uint32_t word = 0;
#pragma unroll
                for (uint32_t i = 0; i < 32; ++i)   // exact integer count c < 2^23: bit 0 of 2^23 + c is its parity
                    word |= (__float_as_uint(__uint_as_float(r[i]) + 8388608.0f) & 1u) << i;
                if (row < args.count)
                    dst[c / 32u] = word;
            }
            fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(tfree(tb));
        }
        if (failed)
            *abort_flag = 1;
    }
    __syncwarp();
    if (failed && args.err && lane == 0)
        atomicOr(args.err, kErrTimeout);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// r_j in bit order from the parities in q order: for output words w0 .. w0+31
// and bit e, q(32 w + e) = (Q_e - w) mod n with Q_e = (n - 1 - e) inv32 mod n,
// a run of 32 q's read backwards from start = (Q_e - w0 - 31) mod n; lane e
// gathers it with one funnel shift, the warp transposes it.  One CTA per
// product at a time: the product's parity row is first copied to shared
// memory (coalesced), followed by its first bits again from bit n on, so
// that no run wraps past q = n - 1.  Warp k takes the 32-word blocks k, k + 8,
// ..., so a lane's run start moves down by 256 from one block to the next
// (start computed once per thread, no division per block).
__global__ void __launch_bounds__(256) tc_assemble_kernel(const uint32_t *__restrict__ qbits, uint32_t qwords,
                                                          uint32_t n, uint32_t inv32, uint32_t count,
                                                          uint64_t *__restrict__ out, size_t stride_out)
{
    extern __shared__ uint32_t srow[];   // (n >> 5) + 2 words
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t L32 = (n + 31) / 32, blocks = (L32 + 31) / 32, W32 = 2u * ((n + 63u) / 64u);
    const uint32_t nw = n >> 5, sft = n & 31u;   // n is odd: sft > 0
    // n <= 65535 and inv32 < n: the products stay below 2^32
    const uint32_t Qe = ((n - 1u - (lane % n)) * inv32) % n;
    const uint32_t start0 = (Qe + 32u * n - 32u * warp - 31u) % n;   // first block of this warp (32 warp < n)
    const uint32_t step = (32u * nwarps) % n;
    // per transpose stage s (16, 8, 4, 2, 1): a lane with bit s set takes the
    // partner's word shifted right by s into its low s-blocks, the others
    // its word shifted left into their high s-blocks; a rotation by the
    // lane's amount puts the wanted bits in place (the wrapped bits fall
    // under the mask), and `keep` selects the lane's own bits
    uint32_t keep[5], rot[5];
#pragma unroll
    for (uint32_t t = 0, sh = 16, m = 0x0000ffffu; t < 5; ++t, sh >>= 1, m ^= m << sh) {
        keep[t] = (lane & sh) ? ~m : m;
        rot[t] = (lane & sh) ? 32u - sh : sh;
    }
    for (uint32_t j = blockIdx.x; j < count; j += gridDim.x) {
        // the row's words below nw, then the two words from bit 32 nw on,
        // where bits n .. n + 62 repeat the row's bits 0 .. 62 (the row is
        // periodic in q with period n), so that no run wraps past q = n - 1
        const uint32_t *row = qbits + (size_t)j * qwords;
        for (uint32_t i = threadIdx.x; i < nw + 2u; i += blockDim.x) {
            uint32_t v;
            if (i < nw)
                v = row[i];
            else if (i == nw)   // bits below n, then the row's bits 0 .. 31 - sft
                v = (row[nw] & ((1u << sft) - 1u)) | (row[0] << sft);
            else
                v = (row[0] >> (32u - sft)) | (row[1] << sft);
            srow[i] = v;
        }
        __syncthreads();
        uint32_t *o = reinterpret_cast<uint32_t *>(out + (size_t)j * stride_out);
        uint32_t st = start0;
        for (uint32_t blk = warp; blk < blocks; blk += nwarps) {
            const uint32_t x = __funnelshift_r(srow[st >> 5], srow[(st >> 5) + 1u], st & 31u);
            st = st >= step ? st - step : st + n - step;
            // lane e holds bit e of words w0 .. w0+31 (bit i <-> word w0 + i);
            // a 32 x 32 bit transpose across the warp (swap the off-diagonal
            // s x s blocks for s = 16, 8, 4, 2, 1) leaves word w0 + lane in lane
            uint32_t mine = __brev(x);
#pragma unroll
            for (uint32_t t = 0, sh = 16; t < 5; ++t, sh >>= 1) {
                const uint32_t y = __shfl_xor_sync(0xffffffffu, mine, sh);
                const uint32_t r = __funnelshift_l(y, y, rot[t]);
                mine = (mine & keep[t]) | (r & ~keep[t]);
            }
            const uint32_t w = 32u * blk + lane;
            if (w < L32) {
                if (w == L32 - 1u)
                    mine &= (1u << sft) - 1u;
                o[w] = mine;
            } else if (w < W32) {
                o[w] = 0u;   // the top limb's upper half
            }
        }
        __syncthreads();   // srow is rewritten for the next product
    }
}

// ---------------------------------------------------------------- host side

bool tc_shape(uint32_t n, size_t count, TcShape *sh)
{
    if (n < 1 || n > kTcMaxN || !(n & 1u) || count == 0)
        return false;
    sh->S = (n + 63) / 64;
    sh->V = (n + kNU - 1) / kNU;
    sh->qwords = sh->V * (kNU / 32u);
    sh->rwin = 16u * (kNU - 1u) + 32u * sh->S;               // bytes of one unit's R window (multiple of 16)
    sh->rseq_bytes = (size_t)16u * kNU * (sh->V - 1u) + sh->rwin;
    // inverse of 32 mod n (n odd): extended Euclid
    int64_t t0 = 0, t1 = 1, r0 = n, r1 = 32 % n;
    while (r1) {
        const int64_t q = r0 / r1, r2 = r0 - q * r1, t2 = t0 - q * t1;
        r0 = r1;
        r1 = r2;
        t0 = t1;
        t1 = t2;
    }
    sh->inv32 = n == 1 ? 0u : (uint32_t)((t0 % (int64_t)n + n) % n);
    return true;
}

size_t tc_group_bytes(const TcShape &sh, size_t products)
{
    const size_t tiles = (products + 127) / 128;
    return tiles * sh.S * (size_t)kChunk + (products * sh.qwords + 2) * 4ull;
}

cudaError_t prepare_tc()
{
    return cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

cudaError_t launch_tc_rseq(const uint64_t *a, uint32_t n, const TcShape &sh, uint8_t *rseq, int sm_count,
                           cudaStream_t st)
{
    const uint32_t words = (uint32_t)((sh.rseq_bytes + 3) / 4);
    tc_rseq_kernel<<<(unsigned)std::min<uint32_t>(4u * sm_count, (words + 255) / 256), 256, 0, st>>>(
        a, n, reinterpret_cast<uint32_t *>(rseq), words);
    return cudaGetLastError();
}

cudaError_t launch_tc_group(const uint64_t *b, size_t stride_b, uint64_t *out, size_t stride_out, uint32_t n,
                            uint32_t count, const TcShape &sh, const uint8_t *rseq, uint8_t *scratch, uint32_t *err,
                            int sm_count, cudaStream_t st)
{
    const uint32_t tiles = (count + 127) / 128;
    uint8_t *chunks = scratch;
    uint32_t *qbits = reinterpret_cast<uint32_t *>(scratch + (size_t)tiles * sh.S * kChunk);
    const uint64_t threads = (uint64_t)tiles * sh.S * 128u;
    tc_unpack_kernel<<<(unsigned)std::min<uint64_t>(8ull * sm_count, (threads + 255) / 256), 256, 0, st>>>(
        b, stride_b, n, count, sh.S, tiles, chunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    TcGemmArgs g;
    g.chunks = chunks;
    g.rseq = rseq;
    g.qbits = qbits;
    g.err = err;
    g.S = sh.S;
    g.V = sh.V;
    g.units = tiles * sh.V;
    g.count = count;
    g.qwords = sh.qwords;
    g.rwin = sh.rwin;
    tc_gemm_kernel<<<std::min<uint32_t>(g.units, (uint32_t)sm_count), kTcThreads, kSmemBytes, st>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    tc_assemble_kernel<<<(unsigned)std::min<uint64_t>(8ull * sm_count, count), 256, 4u * (n / 32u + 2u), st>>>(
        qbits, sh.qwords, n, sh.inv32, count, out, stride_out);
    return cudaGetLastError();
}

}  // namespace gf2x
