// sparse.cu -- constant-time product of a dense a and a sparse b given by
// its w set positions, modulo X^n - 1: the operand shape of the HQC and BIKE
// operations of Sec. 1, where the sparse operand is secret.  Sec. 1 rules out
// methods that use the sparsity through branches or addresses; here the
// positions only enter select masks and a funnel-shift count:
//   r = sum_j X^(p_j) a mod (X^n - 1) = sum_j rot(a, p_j),
// and rot(a, p) is the n-bit window at bit s = n - p of D = a + X^n a (the
// doubled vector, 2n bits).  With q = s >> 5 the window's word offset and
// s & 31 its bit offset, word w of the window is the low half of
// (D[w + q + 1] : D[w + q]) >> (s & 31).
//
// Layout: a warp holds 32 C words of D, word w = lane + 32 k in register k
// of lane `lane`.  The word offset q = 32 qh + ql is applied in two parts,
// each as a barrel shifter whose stages are all executed and select under
// the mask of one bit of q (both candidates read, no secret address, no
// secret shuffle lane):
//  * qh (whole registers): stage t moves register k + 2^t into register k.
//    A pure register rename, so a select per register; the stages run
//    largest first, and each only computes the registers that the later
//    stages can still read.
//  * ql (lanes): five stages of a cyclic lane rotation by 2^t (a shuffle
//    from a fixed lane offset, then a select), then lanes with
//    lane + ql >= 32 take the next register (their word came round from
//    the following 32-word row).
// The bit offset is one funnel shift per word with the neighbouring word,
// which is lane + 1 (a shuffle from a fixed offset; lane 31 takes lane 0 of
// the next register).  The R accumulator registers of a lane hold result
// words lane + 32 k; 32 R >= N + 1.
//
// Larger n first apply the top bits of q in shared memory (each warp its own
// buffer B, shifts >= 256 words with public addresses), so that the register
// window stays at C = R + QH + 1 registers.  One CTA per product; its four
// warps take a quarter of the positions each and XOR their partial sums.
// Work per product: fixed by n, w and the kernel shape.
#include <cstdint>

#include <cuda_runtime.h>

#include "launchers.h"

namespace gf2x {

constexpr int kSparseWarps = 4;

__host__ __device__ constexpr int bit_length(int x)
{
    return x == 0 ? 0 : 1 + bit_length(x >> 1);
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

// The positions of product p that warp `warp` of its CTA takes: an equal
// share of the w (sizes only; the CTA's four partial sums are XORed).
__device__ __forceinline__ void warp_share(uint32_t w, uint32_t warp, uint32_t *jb, uint32_t *je)
{
    *jb = (uint32_t)(((uint64_t)w * warp) / kSparseWarps);
    *je = (uint32_t)(((uint64_t)w * (warp + 1u)) / kSparseWarps);
}

// Shapes compiled with the shared stages: the offsets they leave, below
// 32 (QH + 1) words, form a power of two >= 256 (every shared shift >= 256).
__host__ __device__ constexpr bool shared_capable(int R, int QH)
{
    return QH + 1 >= 8 && ((QH + 1) & QH) == 0 && QH + 1 < R;
}

// The top `pre` bits of the word offset q in shared memory: afterwards
// B[w] = D[w + (q with its low T - pre bits cleared)] for w < wpad + (the
// smallest shared shift), wpad = the register window rounded up to 128
// words.  Stage u moves by 2^(T - 1 - u) words (>= 256), the first from D
// into B, the rest in place in B.  Each lane moves 4 words per 16-byte
// access; a warp reads a 128-word chunk (and the chunk one shift ahead)
// before it writes the chunk, and the chunks go up, so every read precedes
// the write of its word.  Lengths are multiples of 128 words, the trip
// counts uniform over the warp.  (Four accesses in flight per lane measured
// 1.7% slower at n = 57637.)
__device__ __forceinline__ void shared_stages(const uint32_t *D, uint32_t *B, uint32_t q, uint32_t T, uint32_t pre,
                                              uint32_t wpad, uint32_t lane)
{
    uint4 *B4 = reinterpret_cast<uint4 *>(B);
    for (uint32_t u = 0; u < pre; ++u) {
        const uint32_t t = T - 1u - u;
        const uint32_t sh4 = (1u << t) >> 2, m = 0u - ((q >> t) & 1u);
        const uint32_t len4 = (wpad >> 2) + sh4;     // what the smaller shifts still read
        const uint4 *in = reinterpret_cast<const uint4 *>(u == 0 ? D : B);
        for (uint32_t w = lane; w < len4; w += 32u) {
            const uint4 x = in[w], y = in[w + sh4];
            uint4 v;
            v.x = (y.x & m) | (x.x & ~m);
            v.y = (y.y & m) | (x.y & ~m);
            v.z = (y.z & m) | (x.z & ~m);
            v.w = (y.w & m) | (x.w & ~m);
            __syncwarp();
            B4[w] = v;
        }
        __syncwarp();
    }
}

// Register stages t = T - 1, ..., 0 of the whole-register barrel (largest
// first; one compile-time instance per stage, so that every register index
// is a constant).  Stage t computes registers 0 .. R + the largest offset
// the later stages can still apply, min(QH, 2^t - 1).  (Bounding that by
// QH - 2^t when the stage moves saves 14 selects per position at R = 18
// but measured 0.4% slower.)
template <int R, int QH, int T>
__device__ __forceinline__ void register_stages(uint32_t (&y)[R + QH + 1], uint32_t qh)
{
    if constexpr (T > 0) {
        constexpr int C = R + QH + 1, t = T - 1, sh = 1 << t;
        constexpr int later = QH < sh - 1 ? QH : sh - 1;
        constexpr int dest = R + 1 + later < C ? R + 1 + later : C;
        const uint32_t m = 0u - ((qh >> t) & 1u);
#pragma unroll
        for (int k = 0; k < dest; ++k) {
            if (k + sh < C)
                y[k] = (y[k + sh] & m) | (y[k] & ~m);
        }
        register_stages<R, QH, T - 1>(y, qh);
    }
}

// Lane stages t = T - 1, ..., 0: registers 0 .. R rotate cyclically by 2^t
// lanes under bit t of ql.
template <int R, int QH, int T>
__device__ __forceinline__ void lane_stages(uint32_t (&y)[R + QH + 1], uint32_t ql, uint32_t lane)
{
    if constexpr (T > 0) {
        constexpr int t = T - 1;
        const uint32_t m = 0u - ((ql >> t) & 1u);
        const uint32_t from = (lane + (1u << t)) & 31u;
#pragma unroll
        for (int k = 0; k <= R; ++k) {
            const uint32_t z = __shfl_sync(0xffffffffu, y[k], from);
            y[k] = (z & m) | (y[k] & ~m);
        }
        lane_stages<R, QH, T - 1>(y, ql, lane);
    }
}

// acc ^= the window at word offset q (q < 32 (QH + 1) after the shared
// stages) and bit offset b of the 32 C words held in y (word lane + 32 k in
// y[k]).  y is consumed.
template <int R, int QH>
__device__ __forceinline__ void add_rotated(uint32_t (&acc)[R], uint32_t (&y)[R + QH + 1], uint32_t q, uint32_t b,
                                            uint32_t lane, uint32_t lane0)
{
    const uint32_t qh = q >> 5, ql = q & 31u;
    register_stages<R, QH, bit_length(QH)>(y, qh);
    // lanes: cyclic rotation by ql, then the wrapped lanes take the next register
    lane_stages<R, QH, 5>(y, ql, lane);
    const uint32_t wm = 0u - ((lane + ql) >> 5);
#pragma unroll
    for (int k = 0; k < R; ++k)
        y[k] = (y[k + 1] & wm) | (y[k] & ~wm);
    // bit offset: funnel with the next word (lane + 1; lane 31 reads lane 0
    // of the next register, which lane 0 sends)
    const uint32_t from = (lane + 1u) & 31u;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const uint32_t v = k + 1 < R ? (y[k + 1] & lane0) | (y[k] & ~lane0) : y[k];
        const uint32_t nb = __shfl_sync(0xffffffffu, v, from);
        acc[k] ^= __funnelshift_r(y[k], nb, b);
    }
}

// One CTA per product (persistent over the batch), its four warps each
// taking a quarter of the positions.  Shared memory: D (d_words), then
// either the four warps' stage buffers B (b_words each; pre > 0) or the
// three partial-sum buffers of warps 1-3 (pre = 0).
template <int R, int QH, int MINB>
__global__ void __launch_bounds__(32 * kSparseWarps, MINB) sparse_mulmod_kernel(const SparseArgs args)
{
    constexpr int C = R + QH + 1;
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lane0 = 0u - (lane == 0u ? 1u : 0u);
    uint32_t *D = smem;
    uint32_t *B = smem + args.d_words + warp * args.b_words;
    uint32_t *red = smem + args.d_words + (args.pre ? args.b_words : 0u);
    const uint32_t red_stride = args.pre ? args.b_words : 32u * R;
    const uint32_t wpad = (32u * C + 127u) & ~127u;
    const uint32_t qmask = (1u << (args.T - args.pre)) - 1u;
    uint32_t jb, je;
    warp_share(args.w, warp, &jb, &je);
    for (uint32_t p = blockIdx.x; p < args.count; p += gridDim.x) {
        const uint32_t *a32 = reinterpret_cast<const uint32_t *>(args.a + (size_t)p * args.stride_a);
        const uint32_t *pos = args.pos + (size_t)p * args.stride_pos;
        build_doubled(D, args.d_words, a32, args.n, threadIdx.x, blockDim.x);
        __syncthreads();
        uint32_t acc[R];
#pragma unroll
        for (int k = 0; k < R; ++k)
            acc[k] = 0u;
        const uint32_t *src = args.pre ? B : D;
        for (uint32_t j0 = jb; j0 < je; j0 += 32u) {
            const uint32_t mine = j0 + lane < je ? pos[j0 + lane] : 0u;
            const uint32_t cnt = je - j0 < 32u ? je - j0 : 32u;
            for (uint32_t jj = 0; jj < cnt; ++jj) {
                const uint32_t s = args.n - __shfl_sync(0xffffffffu, mine, jj);
                const uint32_t q = s >> 5;
                if constexpr (shared_capable(R, QH))
                    if (args.pre)
                        shared_stages(D, B, q, args.T, args.pre, wpad, lane);
                uint32_t y[C];
#pragma unroll
                for (int k = 0; k < C; ++k)
                    y[k] = src[lane + 32u * k];
                __syncwarp();   // B is rewritten by the next position's first stage
                add_rotated<R, QH>(acc, y, q & qmask, s & 31u, lane, lane0);
            }
        }
        __syncthreads();   // every warp is done with D and with its B
        if (warp > 0) {
            uint32_t *mine = red + (warp - 1u) * red_stride;
#pragma unroll
            for (int k = 0; k < R; ++k)
                mine[lane + 32u * k] = acc[k];
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t N = (args.n + 31u) / 32u, words = 2u * ((args.n + 63u) / 64u);
            const uint32_t top = (args.n & 31u) ? (1u << (args.n & 31u)) - 1u : 0xffffffffu;
            uint32_t *r32 = reinterpret_cast<uint32_t *>(args.r + (size_t)p * args.stride_r);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                uint32_t v = acc[k];
#pragma unroll
                for (uint32_t g = 0; g + 1u < (uint32_t)kSparseWarps; ++g)
                    v ^= red[g * red_stride + lane + 32u * k];
                const uint32_t w = lane + 32u * k;
                if (w < words)
                    r32[w] = w < N ? v & (w == N - 1u ? top : 0xffffffffu) : 0u;
            }
        }
        __syncthreads();   // D, B and the partial sums are rewritten for the next product
    }
}

// The compiled shapes: R result registers per lane, register offsets up to
// QH, CTAs per SM the register budget allows.  The first seven keep D's
// whole window in registers (QH = R - 1 covers every offset of the n they
// serve); the last three take the top bits of q in shared memory first.
struct Variant {
    uint32_t R, QH;
};
constexpr Variant kVariants[] = {{2, 1},  {5, 4},   {9, 8},   {13, 12}, {18, 17},
                                 {26, 25}, {36, 35}, {46, 15}, {57, 15}, {65, 7}};

template <int R, int QH, int MINB>
static cudaError_t launch_variant(const SparseArgs &a, size_t smem, unsigned grid, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(sparse_mulmod_kernel<R, QH, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    sparse_mulmod_kernel<R, QH, MINB><<<grid, 32 * kSparseWarps, smem, st>>>(a);
    return cudaGetLastError();
}

bool sparse_shape(uint32_t n, SparseShape *sh)
{
    if (n < 1 || n > kSparseMaxN)
        return false;
    const uint32_t N = (n + 31u) / 32u, qmax = n >> 5;
    uint32_t T = 0;
    while (T < 32u && (qmax >> T) != 0u)
        ++T;
    const uint32_t R = (N + 1u + 31u) / 32u;   // 32 R >= N + 1
    for (const Variant &v : kVariants) {
        if (v.R < R)
            continue;
        // pre = 0 when every register offset qmax / 32 fits QH; else the
        // shared stages leave offsets below 32 (QH + 1) = 2^(T - pre)
        uint32_t pre = 0;
        if ((qmax >> 5) > v.QH) {
            if (!shared_capable((int)v.R, (int)v.QH))
                continue;
            const uint32_t span = 32u * (v.QH + 1u);
            uint32_t lg = 0;
            while ((1u << lg) < span)
                ++lg;
            if ((1u << lg) != span || lg < 8u || T <= lg)
                continue;   // shared shifts must be >= 256 words
            pre = T - lg;
        }
        const uint32_t C = v.R + v.QH + 1u;
        sh->N = N;
        sh->T = T;
        sh->R = v.R;
        sh->QH = v.QH;
        sh->C = C;
        sh->pre = pre;
        // the shared stages move 128-word chunks: the window rounded up to
        // 128 words plus the first shift's reach (D), plus the second's (B)
        const uint32_t wpad = (32u * C + 127u) & ~127u;
        sh->d_words = pre ? wpad + (1u << T) : 32u * C;
        sh->b_words = pre ? wpad + (1u << (T - 1u)) : 0u;
        return true;
    }
    return false;
}

size_t sparse_smem_bytes(const SparseShape &sh)
{
    const size_t tail = sh.pre ? (size_t)kSparseWarps * sh.b_words : (size_t)(kSparseWarps - 1) * 32u * sh.R;
    return 4ull * (sh.d_words + tail);
}

cudaError_t launch_sparse_mulmod(const SparseArgs &args, const SparseShape &sh, int sm_count, cudaStream_t st)
{
    const size_t ctas = args.count;   // one CTA per product
    const size_t cap = (size_t)(sm_count > 0 ? sm_count : 1) * 8u;
    const unsigned grid = (unsigned)(ctas < cap ? ctas : cap);
    if (grid == 0)
        return cudaSuccess;
    const size_t smem = sparse_smem_bytes(sh);
    switch (sh.R) {
    case 2: return launch_variant<2, 1, 8>(args, smem, grid, st);
    case 5: return launch_variant<5, 4, 8>(args, smem, grid, st);
    case 9: return launch_variant<9, 8, 8>(args, smem, grid, st);
    case 13: return launch_variant<13, 12, 6>(args, smem, grid, st);
    case 18: return launch_variant<18, 17, 6>(args, smem, grid, st);
    case 26: return launch_variant<26, 25, 5>(args, smem, grid, st);
    case 36: return launch_variant<36, 35, 4>(args, smem, grid, st);
    case 46: return launch_variant<46, 15, 3>(args, smem, grid, st);
    case 57: return launch_variant<57, 15, 3>(args, smem, grid, st);
    case 65: return launch_variant<65, 7, 2>(args, smem, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gf2x
