// sparse.cu -- constant-time product of a dense a and a sparse b given by
// its w set positions, modulo X^n - 1: the operand shape of the HQC and BIKE
// operations of Sec. 1, where the sparse operand is secret.  Sec. 1 rules
// out methods that use the sparsity through branches or addresses; here the
// positions only enter masks and shift counts:
//   r = sum_j X^(p_j) a mod (X^n - 1) = sum_j rot(a, p_j),
// and rot(a, p) is the n-bit window at bit s = n - p of D = a + X^n a (the
// doubled vector, 2n bits).  The window's word offset q = s >> 5 is applied
// by a barrel shifter (stage t moves every word by 2^t under the mask of bit
// t of q, both candidates read, no secret address), its bit offset s & 31 by
// a funnel shift (constant time in the shift count), and the windows are
// XORed into the accumulator.
//
// One CTA per product; each of its four warps takes a quarter of the
// positions, and the four partial sums are XORed at the end.  Word
// i = lane C + k of a warp's cyclic window lives in register k of lane
// `lane` (C words per lane, 32 C >= the window); a shift by 2^t words is a
// register rename plus __shfl_sync from a fixed lane offset.  Small n keep D
// itself in registers; larger n first apply the largest shifts in shared
// memory, shrinking the window to what the register stages need.  Work per
// product: w x (stages x C) selects and shuffles per lane, independent of
// the operand bits.
#include <cstdint>

#include <cuda_runtime.h>

#include "launchers.h"

namespace gf2x {

constexpr int kSparseWarps = 4;
constexpr int kSparseMaxStages = 12;   // q < 2^12 words covers n <= 131072

// Cyclic shift of the 32 C-word window held by the warp: afterwards word w
// is the former word (w + q mod 2^stages) mod 32C, stage t taken under the
// mask of bit t of q (stages is uniform over the warp).
template <int C>
__device__ __forceinline__ void barrel(uint32_t (&y)[C], uint32_t q, uint32_t stages, uint32_t lane)
{
#pragma unroll
    for (int t = 0; t < kSparseMaxStages; ++t) {
        if ((uint32_t)t < stages) {
            const uint32_t m = 0u - ((q >> t) & 1u);
            uint32_t nv[C];
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const int g = k + (1 << t);
                const int d = g / C, kk = g % C;
                const uint32_t v = (d % 32 == 0) ? y[kk] : __shfl_sync(0xffffffffu, y[kk], (lane + d) & 31u);
                nv[k] = (v & m) | (y[k] & ~m);
            }
#pragma unroll
            for (int k = 0; k < C; ++k)
                y[k] = nv[k];
        }
    }
}

// acc ^= the n-bit window at bit offset b of the window held in y (word w of
// the result = bits [32w + b, 32w + b + 32) of y).
template <int C>
__device__ __forceinline__ void add_window(uint32_t (&acc)[C], const uint32_t (&y)[C], uint32_t b, uint32_t lane)
{
    const uint32_t next = __shfl_sync(0xffffffffu, y[0], (lane + 1u) & 31u);
#pragma unroll
    for (int k = 0; k < C; ++k)
        acc[k] ^= __funnelshift_r(y[k], k + 1 < C ? y[k + 1] : next, b);
}

// D = a + X^n a into `dst` (len words, zero past 2n bits); a masked to n bits.
__device__ __forceinline__ void build_doubled(uint32_t *dst, uint32_t len, const uint32_t *a32, uint32_t n,
                                              uint32_t first, uint32_t stride)
{
    const uint32_t N = (n + 31u) / 32u, q0 = n >> 5, r0 = n & 31u;
    const uint32_t top = r0 ? (1u << r0) - 1u : 0xffffffffu;
    for (uint32_t w = first; w < len; w += stride) {
        uint32_t v = 0;
        if (w < N)
            v = a32[w] & (w == N - 1u ? top : 0xffffffffu);
        if (w >= q0 && w - q0 <= N) {
            const uint32_t i = w - q0;
            const uint32_t x = i < N ? a32[i] & (i == N - 1u ? top : 0xffffffffu) : 0u;
            const uint32_t xp = (i >= 1u && i - 1u < N) ? a32[i - 1u] & (i - 1u == N - 1u ? top : 0xffffffffu) : 0u;
            v |= r0 ? (x << r0) | (xp >> (32u - r0)) : x;
        }
        dst[w] = v;
    }
}

template <int C>
__device__ __forceinline__ void store_result(uint64_t *r_row, const uint32_t (&acc)[C], uint32_t n, uint32_t lane)
{
    const uint32_t N = (n + 31u) / 32u, words = 2u * ((n + 63u) / 64u);
    const uint32_t top = (n & 31u) ? (1u << (n & 31u)) - 1u : 0xffffffffu;
    uint32_t *r32 = reinterpret_cast<uint32_t *>(r_row);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const uint32_t w = lane * C + k;
        if (w < words)
            r32[w] = w < N ? acc[k] & (w == N - 1u ? top : 0xffffffffu) : 0u;
    }
}

// The positions of product p that warp `warp` of its CTA takes: an equal
// share of the w (sizes only; the CTA's four partial sums are XORed).
__device__ __forceinline__ void warp_share(uint32_t w, uint32_t warp, uint32_t *jb, uint32_t *je)
{
    *jb = (uint32_t)(((uint64_t)w * warp) / kSparseWarps);
    *je = (uint32_t)(((uint64_t)w * (warp + 1u)) / kSparseWarps);
}

// The CTA's four partial sums into warp 0's acc (red: three buffers of
// 32 C words, one per other warp), then warp 0 stores the row.
template <int C>
__device__ __forceinline__ void reduce_and_store(uint32_t (&acc)[C], uint32_t *red, size_t red_stride,
                                                 uint64_t *r_row, uint32_t n, uint32_t lane, uint32_t warp)
{
    if (warp > 0) {
        uint32_t *mine = red + (warp - 1u) * red_stride;
#pragma unroll
        for (int k = 0; k < C; ++k)
            mine[lane * C + k] = acc[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (uint32_t g = 0; g + 1u < (uint32_t)kSparseWarps; ++g) {
#pragma unroll
            for (int k = 0; k < C; ++k)
                acc[k] ^= red[g * red_stride + lane * C + k];
        }
        store_result<C>(r_row, acc, n, lane);
    }
}

// One CTA per product (persistent over the batch), its four warps each
// taking a quarter of the positions.  Small n (32 C >= N + n/32 + 1): D is
// built once in shared memory and held in registers by every warp (dreg),
// every position runs all its stages there.
template <int C>
__global__ void __launch_bounds__(32 * kSparseWarps, 3) sparse_mulmod_regs_kernel(const SparseArgs args)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *D = smem;                       // 32 C words
    uint32_t *red = smem + 32u * C;           // 3 x 32 C words
    uint32_t jb, je;
    warp_share(args.w, warp, &jb, &je);
    for (uint32_t p = blockIdx.x; p < args.count; p += gridDim.x) {
        const uint32_t *a32 = reinterpret_cast<const uint32_t *>(args.a + (size_t)p * args.stride_a);
        const uint32_t *pos = args.pos + (size_t)p * args.stride_pos;
        build_doubled(D, 32u * C, a32, args.n, threadIdx.x, blockDim.x);
        __syncthreads();
        uint32_t dreg[C], acc[C];
#pragma unroll
        for (int k = 0; k < C; ++k) {
            dreg[k] = D[lane * C + k];
            acc[k] = 0u;
        }
        for (uint32_t j0 = jb; j0 < je; j0 += 32u) {
            const uint32_t mine = j0 + lane < je ? pos[j0 + lane] : 0u;
            const uint32_t cnt = je - j0 < 32u ? je - j0 : 32u;
            for (uint32_t jj = 0; jj < cnt; ++jj) {
                const uint32_t s = args.n - __shfl_sync(0xffffffffu, mine, jj);
                uint32_t y[C];
#pragma unroll
                for (int k = 0; k < C; ++k)
                    y[k] = dreg[k];
                barrel<C>(y, s >> 5, args.stages, lane);
                add_window<C>(acc, y, s & 31u, lane);
            }
        }
        reduce_and_store<C>(acc, red, 32u * C, args.r + (size_t)p * args.stride_r, args.n, lane, warp);
        __syncthreads();   // D and red are rewritten for the next product
    }
}

// Larger n: D in shared memory, built once per product; each warp applies
// the `pre` largest shifts of its positions in its own buffer B (the first
// from D into B, the rest in place in B), then its register window (32 C
// words of B, or of D when pre = 0) takes the remaining stages.  The B
// buffers of warps 1-3 (b_words >= 32 C) hold the partial sums at the end.
template <int C>
__global__ void __launch_bounds__(32 * kSparseWarps) sparse_mulmod_staged_kernel(const SparseArgs args)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *D = smem;
    uint32_t *B = smem + args.d_words + warp * args.b_words;
    const uint32_t N = (args.n + 31u) / 32u;
    uint32_t jb, je;
    warp_share(args.w, warp, &jb, &je);
    for (uint32_t p = blockIdx.x; p < args.count; p += gridDim.x) {
        const uint32_t *a32 = reinterpret_cast<const uint32_t *>(args.a + (size_t)p * args.stride_a);
        const uint32_t *pos = args.pos + (size_t)p * args.stride_pos;
        build_doubled(D, args.d_words, a32, args.n, threadIdx.x, blockDim.x);
        __syncthreads();
        uint32_t acc[C];
#pragma unroll
        for (int k = 0; k < C; ++k)
            acc[k] = 0u;
        const uint32_t *src = args.pre ? B : D;
        for (uint32_t j0 = jb; j0 < je; j0 += 32u) {
            const uint32_t mine = j0 + lane < je ? pos[j0 + lane] : 0u;
            const uint32_t cnt = je - j0 < 32u ? je - j0 : 32u;
            for (uint32_t jj = 0; jj < cnt; ++jj) {
                const uint32_t s = args.n - __shfl_sync(0xffffffffu, mine, jj);
                const uint32_t q = s >> 5;
                for (uint32_t u = 0; u < args.pre; ++u) {
                    const uint32_t t = args.stages + args.pre - 1u - u;   // largest first
                    const uint32_t sh = 1u << t, m = 0u - ((q >> t) & 1u);
                    const uint32_t len = N + sh;     // what the smaller shifts still need
                    const uint32_t *in = u == 0 ? D : B;
                    // in place: 256 words are read before any is written,
                    // and sh >= 256 (sparse_shape) keeps every read ahead of
                    // the writes; uniform trip count, every lane reaches
                    // each __syncwarp
                    for (uint32_t w0 = 0; w0 < len; w0 += 256u) {
                        uint32_t v[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const uint32_t w = w0 + 32u * e + lane;
                            v[e] = w < len ? (in[w + sh] & m) | (in[w] & ~m) : 0u;
                        }
                        __syncwarp();
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const uint32_t w = w0 + 32u * e + lane;
                            if (w < len)
                                B[w] = v[e];
                        }
                    }
                    __syncwarp();
                }
                uint32_t y[C];
#pragma unroll
                for (int k = 0; k < C; ++k)
                    y[k] = src[lane * C + k];
                __syncwarp();   // B is rewritten by the next position's first stage
                barrel<C>(y, q, args.stages, lane);
                add_window<C>(acc, y, s & 31u, lane);
            }
        }
        __syncthreads();   // every warp is done with D and with its B
        reduce_and_store<C>(acc, smem + args.d_words + args.b_words, args.b_words,
                            args.r + (size_t)p * args.stride_r, args.n, lane, warp);
        __syncthreads();   // D and the B buffers are rewritten for the next product
    }
}

template <int C>
static cudaError_t launch_regs(const SparseArgs &a, unsigned grid, cudaStream_t st)
{
    const size_t smem = 4ull * kSparseWarps * 32u * C;
    sparse_mulmod_regs_kernel<C><<<grid, 32 * kSparseWarps, smem, st>>>(a);
    return cudaGetLastError();
}

template <int C>
static cudaError_t launch_staged(const SparseArgs &a, unsigned grid, cudaStream_t st)
{
    const size_t smem = 4ull * (a.d_words + kSparseWarps * a.b_words);
    cudaError_t e = cudaFuncSetAttribute(sparse_mulmod_staged_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    sparse_mulmod_staged_kernel<C><<<grid, 32 * kSparseWarps, smem, st>>>(a);
    return cudaGetLastError();
}

// Window sizes C (words per lane) of the compiled variants.
constexpr int kRegsC[] = {9, 17, 35};
constexpr int kStagedC = 73;

bool sparse_shape(uint32_t n, SparseShape *sh)
{
    if (n < 1 || n > kSparseMaxN)
        return false;
    const uint32_t N = (n + 31u) / 32u, qmax = n >> 5;
    uint32_t T = 0;
    while (T < 32u && (qmax >> T) != 0u)
        ++T;
    sh->N = N;
    sh->T = T;
    for (int C : kRegsC) {
        if (32u * (uint32_t)C >= N + qmax + 1u) {
            sh->C = (uint32_t)C;
            sh->staged = 0;
            sh->pre = 0;
            sh->d_words = 0;
            sh->b_words = 0;
            return true;
        }
    }
    const uint32_t M = 32u * kStagedC;
    for (uint32_t pre = 0; pre <= T; ++pre) {
        // after the pre largest shifts the remaining offset is below 2^(T - pre)
        const uint32_t need = pre == 0 ? N + qmax + 1u : N + (1u << (T - pre));
        if (need <= M) {
            // the in-place shared stages read 256 words ahead of their writes
            if (pre > 0 && (1u << (T - pre)) < 256u)
                return false;
            sh->C = kStagedC;
            sh->staged = 1;
            sh->pre = pre;
            sh->d_words = pre == 0 ? M : (N + (1u << T) > M ? N + (1u << T) : M);
            // B: the shared stages' buffer, and the partial sums at the end
            sh->b_words = pre == 0 ? M : (N + (1u << (T - 1u)) > M ? N + (1u << (T - 1u)) : M);
            return true;
        }
    }
    return false;
}

size_t sparse_smem_bytes(const SparseShape &sh)
{
    return sh.staged ? 4ull * (sh.d_words + kSparseWarps * sh.b_words) : 4ull * kSparseWarps * 32u * sh.C;
}

cudaError_t launch_sparse_mulmod(const SparseArgs &args, const SparseShape &sh, int sm_count, cudaStream_t st)
{
    const size_t ctas = args.count;   // one CTA per product
    const size_t cap = (size_t)(sm_count > 0 ? sm_count : 1) * 8u;
    const unsigned grid = (unsigned)(ctas < cap ? ctas : cap);
    if (grid == 0)
        return cudaSuccess;
    if (!sh.staged) {
        switch (sh.C) {
        case 9: return launch_regs<9>(args, grid, st);
        case 17: return launch_regs<17>(args, grid, st);
        case 35: return launch_regs<35>(args, grid, st);
        default: return cudaErrorInvalidValue;
        }
    }
    return sh.C == kStagedC ? launch_staged<kStagedC>(args, grid, st) : cudaErrorInvalidValue;
}

}  // namespace gf2x
