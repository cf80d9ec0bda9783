// toom.cu -- Toom-4 and Toom-5 top levels over F2[X] (Toom-Cook 4-7 and
// 5-9, the members of Sec. 3's Toom-Cook family after the paper's Toom-3).
// Operands are cut into K parts of m 32-bit words,
// A(t) = A0 + A1 t + ... + A(K-1) t^(K-1), and evaluated at 2K - 1 points:
// 0, inf and 1, x, x+1, x^2, x^2+1 (K = 4), plus x^2+x, x^2+x+1 (K = 5),
// with x = X^32, so that every product by a power of a point is a sum of
// word shifts.  The 2K - 1 products of E-word operands (E = m + 2(K-1),
// even) run as one batch of equal-size products; toom_interp_kernel solves
// for the inner coefficients C1..C(2K-3) of the product polynomial C(t) and
// recomposes c = sum_k C_k X^(32 m k), folding mod X^n - 1 on request.
//
// Interpolation.  With S_j = R(p_j) - C0 - C(2K-2) p_j^(2K-2) for the
// finite nonzero points, C_k = (sum_j P_kj(x) S_j) / D_k(x), the
// Vandermonde system's solution over F2(x) in common-denominator form
// (the tables below; gen_toom_tables.py prints them), where
// D_k = x^a (x+1)^b (x^2+x+1)^c: the points' differences factor into these
// three only.  The numerators are sums of word shifts; dividing by x^a
// drops a words, by x+1 is a prefix XOR over words, and by x^2+x+1 =
// (x^3+1)/(x+1) is a product by 1+x followed by a prefix XOR with a stride
// of three words.  Every division is exact.  All loops and addresses depend
// on the sizes only (constant time in the operand bits).
//
// Checked mode (a non-null error word): the interpolation verifies every
// division -- the a words dropped by x^a are zero, each prefix XOR of a
// division by x+1 ends in a zero word, each division by x^2+x+1 leaves its
// last three words zero -- and that every C_k fits its 2m words, so that a
// wrong table entry is reported, not only seen as a wrong product.
#include <cstdint>

#include <cuda_runtime.h>

#include "gf2x_gb300.h"
#include "launchers.h"

namespace gf2x {

namespace {

constexpr int kT4Threads = 256;

struct ExpSet {
    uint8_t n, e[6];
};
// C_k = (sum_j P_kj S_j) / (x^a (x+1)^b (x^2+x+1)^c)
struct Interp {
    uint8_t a, b, c;
    uint8_t n[7];
    uint8_t e[7][6];
};

// kPowK[j][i]: exponents of p_j^i (points 0, the finite nonzero ones, inf);
// kTopK[j]: exponents of p_j^(2K-2); kInterpK[k]: C_(k+1).
// Toom-4
__constant__ ExpSet kPow4[7][4] = {
    {{1, {0}}, {0, {0}}, {0, {0}}, {0, {0}}},
    {{1, {0}}, {1, {0}}, {1, {0}}, {1, {0}}},
    {{1, {0}}, {1, {1}}, {1, {2}}, {1, {3}}},
    {{1, {0}}, {2, {0, 1}}, {2, {0, 2}}, {4, {0, 1, 2, 3}}},
    {{1, {0}}, {1, {2}}, {1, {4}}, {1, {6}}},
    {{1, {0}}, {2, {0, 2}}, {2, {0, 4}}, {4, {0, 2, 4, 6}}},
    {{0, {0}}, {0, {0}}, {0, {0}}, {1, {0}}},
};
__constant__ ExpSet kTop4[5] = {{1, {0}}, {1, {6}}, {4, {0, 2, 4, 6}}, {1, {12}}, {4, {0, 4, 8, 12}}};
__constant__ Interp kInterp4[5] = {
    {2, 3, 1, {4, 2, 4, 4, 2}, {{2, 4, 5, 7}, {2, 6}, {3, 4, 5, 6}, {0, 1, 2, 3}, {2, 3}}},
    {3, 3, 1, {6, 6, 2, 4, 3}, {{1, 2, 3, 4, 5, 6}, {1, 3, 4, 5, 6, 7}, {2, 7}, {0, 2, 3, 4}, {1, 3, 4}}},
    {3, 3, 1, {5, 6, 6, 3, 3}, {{0, 3, 4, 5, 6}, {1, 2, 3, 4, 5, 6}, {1, 2, 3, 4, 5, 6}, {0, 1, 2}, {0, 1, 2}}},
    {3, 3, 1, {0, 2, 2, 2, 1}, {{0}, {1, 3}, {2, 3}, {0, 2}, {2}}},
    {3, 3, 1, {3, 2, 2, 1, 1}, {{0, 1, 2}, {1, 2}, {1, 2}, {0}, {0}}},
};
// Toom-5
__constant__ ExpSet kPow5[9][5] = {
    {{1, {0}}, {0, {0}}, {0, {0}}, {0, {0}}, {0, {0}}},
    {{1, {0}}, {1, {0}}, {1, {0}}, {1, {0}}, {1, {0}}},
    {{1, {0}}, {1, {1}}, {1, {2}}, {1, {3}}, {1, {4}}},
    {{1, {0}}, {2, {0, 1}}, {2, {0, 2}}, {4, {0, 1, 2, 3}}, {2, {0, 4}}},
    {{1, {0}}, {1, {2}}, {1, {4}}, {1, {6}}, {1, {8}}},
    {{1, {0}}, {2, {0, 2}}, {2, {0, 4}}, {4, {0, 2, 4, 6}}, {2, {0, 8}}},
    {{1, {0}}, {2, {1, 2}}, {2, {2, 4}}, {4, {3, 4, 5, 6}}, {2, {4, 8}}},
    {{1, {0}}, {3, {0, 1, 2}}, {3, {0, 2, 4}}, {5, {0, 1, 3, 5, 6}}, {3, {0, 4, 8}}},
    {{0, {0}}, {0, {0}}, {0, {0}}, {0, {0}}, {1, {0}}},
};
__constant__ ExpSet kTop5[7] = {{1, {0}}, {1, {8}}, {2, {0, 8}}, {1, {16}}, {2, {0, 16}}, {2, {8, 16}}, {3, {0, 8, 16}}};
__constant__ Interp kInterp5[7] = {
    {2, 4, 1, {6, 6, 4, 6, 4, 4, 2}, {{2, 3, 4, 6, 7, 8}, {1, 2, 3, 5, 6, 7}, {2, 4, 5, 7}, {0, 1, 2, 4, 5, 6}, {2, 3, 5, 6}, {1, 3, 4, 6}, {2, 6}}},
    {3, 4, 1, {6, 6, 6, 6, 4, 6, 2}, {{1, 2, 3, 4, 5, 7}, {0, 2, 3, 5, 6, 8}, {1, 3, 4, 6, 7, 8}, {1, 3, 4, 5, 6, 7}, {1, 2, 6, 7}, {0, 1, 2, 4, 5, 7}, {1, 7}}},
    {4, 4, 1, {6, 6, 5, 6, 5, 5, 4}, {{2, 3, 4, 5, 6, 8}, {0, 2, 3, 5, 6, 8}, {2, 3, 5, 6, 8}, {0, 2, 3, 4, 5, 6}, {2, 3, 4, 5, 6}, {0, 2, 3, 5, 6}, {2, 3, 5, 6}}},
    {4, 4, 1, {1, 1, 4, 1, 4, 4, 5}, {{0}, {3}, {0, 1, 2, 3}, {6}, {0, 2, 4, 6}, {3, 4, 5, 6}, {0, 1, 3, 5, 6}}},
    {4, 4, 1, {1, 1, 2, 1, 2, 2, 3}, {{0}, {2}, {0, 2}, {4}, {0, 4}, {2, 4}, {0, 2, 4}}},
    {4, 4, 1, {1, 1, 2, 1, 2, 2, 3}, {{0}, {1}, {0, 1}, {2}, {0, 2}, {1, 2}, {0, 1, 2}}},
    {4, 4, 1, {1, 1, 1, 1, 1, 1, 1}, {{0}, {0}, {0}, {0}, {0}, {0}, {0}}},
};

template <int K> __device__ __forceinline__ const ExpSet &pow_set(uint32_t j, uint32_t i);
template <> __device__ __forceinline__ const ExpSet &pow_set<4>(uint32_t j, uint32_t i) { return kPow4[j][i]; }
template <> __device__ __forceinline__ const ExpSet &pow_set<5>(uint32_t j, uint32_t i) { return kPow5[j][i]; }
template <int K> __device__ __forceinline__ const ExpSet &top_set(uint32_t j);
template <> __device__ __forceinline__ const ExpSet &top_set<4>(uint32_t j) { return kTop4[j]; }
template <> __device__ __forceinline__ const ExpSet &top_set<5>(uint32_t j) { return kTop5[j]; }
template <int K> __device__ __forceinline__ const Interp &interp(uint32_t k);
template <> __device__ __forceinline__ const Interp &interp<4>(uint32_t k) { return kInterp4[k]; }
template <> __device__ __forceinline__ const Interp &interp<5>(uint32_t k) { return kInterp5[k]; }

__device__ __forceinline__ uint32_t operand_word(const uint32_t *x32, uint32_t g, uint32_t L32, uint32_t top)
{
    return g < L32 ? x32[g] & (g == L32 - 1u ? top : 0xffffffffu) : 0u;
}

// v[r + s u] <- XOR of v[r + s u'] over u' <= u, for r < s (v of W words):
// a division by 1 + X^(32 s).  Each thread scans a contiguous run of u;
// the runs' totals are combined by a block-wide exclusive XOR scan.
__device__ void prefix_xor(uint32_t *v, uint32_t W, uint32_t s, uint32_t *carry)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t r = 0; r < s; ++r) {
        const uint32_t U = W > r ? (W - r + s - 1u) / s : 0u;
        const uint32_t per = (U + blockDim.x - 1u) / blockDim.x;
        const uint32_t u0 = threadIdx.x * per;
        const uint32_t u1 = u0 + per < U ? u0 + per : U;
        uint32_t tot = 0;
        for (uint32_t u = u0; u < u1; ++u)
            tot ^= v[r + s * u];
        uint32_t x = tot;   // inclusive scan within the warp
#pragma unroll
        for (uint32_t o = 1; o < 32u; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x ^= y;
        }
        if (lane == 31u)
            carry[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t c = lane < nwarps ? carry[lane] : 0u;
#pragma unroll
            for (uint32_t o = 1; o < 32u; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, c, o);
                if (lane >= o)
                    c ^= y;
            }
            if (lane < nwarps)
                carry[32u + lane] = c;
        }
        __syncthreads();
        uint32_t run = (x ^ tot) ^ (warp > 0 ? carry[32u + warp - 1u] : 0u);   // exclusive prefix
        for (uint32_t u = u0; u < u1; ++u) {
            run ^= v[r + s * u];
            v[r + s * u] = run;
        }
        __syncthreads();
    }
}

}  // namespace

// One CTA per product: the 2K - 1 evaluated operand pairs into `opnd`
// (per product 2K - 1 slots of 2E words: A(p_j) | B(p_j)).
template <int K>
__global__ void __launch_bounds__(kT4Threads) toom_eval_kernel(const ToomArgs args)
{
    constexpr uint32_t NP = 2u * K - 1u;
    const uint32_t L32 = (args.n + 31u) / 32u, m = args.m, E = args.E;
    const uint32_t top = (args.n & 31u) ? (1u << (args.n & 31u)) - 1u : 0xffffffffu;
    for (uint32_t p = blockIdx.x; p < args.count; p += gridDim.x) {
        const uint32_t *a32 = reinterpret_cast<const uint32_t *>(args.a + (size_t)p * args.stride_in);
        const uint32_t *b32 = reinterpret_cast<const uint32_t *>(args.b + (size_t)p * args.stride_in);
        uint32_t *slot = args.opnd + (size_t)p * 2u * NP * E;
        for (uint32_t idx = threadIdx.x; idx < NP * E; idx += blockDim.x) {
            const uint32_t j = idx / E, t = idx - j * E;
            uint32_t va = 0, vb = 0;
#pragma unroll
            for (uint32_t i = 0; i < (uint32_t)K; ++i) {
                const ExpSet &P = pow_set<K>(j, i);
                for (uint32_t q = 0; q < P.n; ++q) {
                    const uint32_t e = P.e[q];
                    if (t >= e && t - e < m) {
                        const uint32_t g = i * m + (t - e);
                        va ^= operand_word(a32, g, L32, top);
                        vb ^= operand_word(b32, g, L32, top);
                    }
                }
            }
            slot[j * 2u * E + t] = va;
            slot[j * 2u * E + E + t] = vb;
        }
    }
}

// One CTA per product: interpolation, recomposition, fold / store.
template <int K>
__global__ void __launch_bounds__(kT4Threads) toom_interp_kernel(const ToomArgs args)
{
    constexpr uint32_t NP = 2u * K - 1u, NF = 2u * K - 3u, TOP = 2u * K - 2u;
    extern __shared__ __align__(16) uint32_t sm[];
    const uint32_t L32 = (args.n + 31u) / 32u, m = args.m, E = args.E, W = args.W, OW = args.OW;
    uint32_t *S = sm;                 // NF x W
    uint32_t *C0 = S + NF * W;        // W
    uint32_t *CT = C0 + W;            // W: the top coefficient C(2K-2)
    uint32_t *num = CT + W;           // W
    uint32_t *tmp = num + W;          // W
    uint32_t *O = tmp + W;            // OW: the product c
    uint32_t *carry = O + OW;         // 64
    for (uint32_t p = blockIdx.x; p < args.count; p += gridDim.x) {
        const uint32_t *R = args.prod + (size_t)p * 2u * NP * E;   // NP products of 2E words
        for (uint32_t t = threadIdx.x; t < W; t += blockDim.x) {
            C0[t] = t < 2u * E ? R[t] : 0u;
            CT[t] = t < 2u * E ? R[(NP - 1u) * 2u * E + t] : 0u;
        }
        __syncthreads();
        for (uint32_t idx = threadIdx.x; idx < NF * W; idx += blockDim.x) {
            const uint32_t j = idx / W, t = idx - j * W;
            uint32_t v = (t < 2u * E ? R[(j + 1u) * 2u * E + t] : 0u) ^ C0[t];
            const ExpSet &PT = top_set<K>(j);
            for (uint32_t q = 0; q < PT.n; ++q)
                v ^= t >= PT.e[q] ? CT[t - PT.e[q]] : 0u;
            S[idx] = v;
        }
        for (uint32_t t = threadIdx.x; t < OW; t += blockDim.x)
            O[t] = (t < W ? C0[t] : 0u) ^ (t >= TOP * m && t - TOP * m < W ? CT[t - TOP * m] : 0u);
        __syncthreads();
        for (uint32_t k = 0; k < NF; ++k) {
            const Interp &I = interp<K>(k);
            // numerator, already divided by x^a
            for (uint32_t t = threadIdx.x; t < W; t += blockDim.x) {
                uint32_t v = 0;
                for (uint32_t j = 0; j < NF; ++j)
                    for (uint32_t q = 0; q < I.n[j]; ++q) {
                        const uint32_t s = t + I.a - I.e[j][q];   // used only when t + a >= e
                        if (t + I.a >= I.e[j][q] && s < W)
                            v ^= S[j * W + s];
                    }
                num[t] = v;
            }
            if (args.err) {   // the words the division by x^a drops are zero
                for (uint32_t t = threadIdx.x; t < I.a; t += blockDim.x) {
                    uint32_t v = 0;
                    for (uint32_t j = 0; j < NF; ++j)
                        for (uint32_t q = 0; q < I.n[j]; ++q)
                            if (t >= I.e[j][q])
                                v ^= S[j * W + t - I.e[j][q]];
                    if (v)
                        atomicOr(args.err, kErrDivX);
                }
            }
            __syncthreads();
            for (uint32_t u = 0; u < I.b; ++u) {
                prefix_xor(num, W, 1u, carry);
                if (args.err && threadIdx.x == 0 && num[W - 1u])   // remainder by x+1
                    atomicOr(args.err, kErrDivX1);
            }
            for (uint32_t u = 0; u < I.c; ++u) {
                for (uint32_t t = threadIdx.x; t < W; t += blockDim.x) {
                    tmp[t] = num[t] ^ (t >= 1u ? num[t - 1u] : 0u);
                    if (args.err && t == W - 1u && num[t])   // the product by 1+x must fit W words
                        atomicOr(args.err, kErrDivX2X1);
                }
                __syncthreads();
                prefix_xor(tmp, W, 3u, carry);
                for (uint32_t t = threadIdx.x; t < W; t += blockDim.x) {
                    num[t] = tmp[t];
                    if (args.err && t + 3u >= W && tmp[t])   // remainder by x^3+1
                        atomicOr(args.err, kErrDivX2X1);
                }
                __syncthreads();
            }
            if (args.err) {   // C_k is a sum of products of m-word parts: 2m words
                for (uint32_t t = 2u * m + threadIdx.x; t < W; t += blockDim.x)
                    if (num[t])
                        atomicOr(args.err, kErrPad);
            }
            const uint32_t off = (k + 1u) * m;
            for (uint32_t t = threadIdx.x; t < W; t += blockDim.x)
                if (off + t < OW)
                    O[off + t] ^= num[t];
            __syncthreads();
        }
        uint32_t *out32 = reinterpret_cast<uint32_t *>(args.out + (size_t)p * args.stride_out);
        if (args.flags & GF2X_REDUCE) {
            const uint32_t words = 2u * ((args.n + 63u) / 64u);
            const uint32_t q0 = args.n >> 5, r0 = args.n & 31u;
            const uint32_t top = r0 ? (1u << r0) - 1u : 0xffffffffu;
            for (uint32_t t = threadIdx.x; t < words; t += blockDim.x) {
                uint32_t v = 0;
                if (t < L32) {
                    const uint32_t hi = __funnelshift_r(O[q0 + t], O[q0 + t + 1u], r0);
                    v = (O[t] ^ hi) & (t == L32 - 1u ? top : 0xffffffffu);
                }
                out32[t] = v;
            }
        } else {
            const uint32_t words = 2u * (uint32_t)((2ull * args.n - 1u + 63u) / 64u);
            for (uint32_t t = threadIdx.x; t < words; t += blockDim.x)
                out32[t] = O[t];
        }
        __syncthreads();   // O and the buffers are rewritten for the next product
    }
}

bool toom_shape(uint32_t K, uint32_t n, ToomArgs *a)
{
    if ((K != 4u && K != 5u) || n < 1 || n > GF2X_MAX_N)
        return false;
    const uint32_t L32 = (n + 31u) / 32u;
    a->m = (L32 + K - 1u) / K;
    const uint32_t e = a->m + 2u * (K - 1u);   // p^(K-1) has degree up to 2(K-1) in x
    a->E = e + (e & 1u);
    a->W = 2u * a->E + 8u * (K - 2u);        // room for C(2K-2) p^(2K-2), degree up to 4(K-1)
    a->OW = (2u * K - 2u) * a->m + a->W;
    return true;
}

size_t toom_interp_smem(uint32_t K, const ToomArgs &a)
{
    return 4ull * ((2ull * K + 1u) * a.W + a.OW + 64u);
}

template <int K>
static cudaError_t launch_pair(const ToomArgs &a, unsigned grid, cudaStream_t st, bool eval)
{
    if (eval) {
        toom_eval_kernel<K><<<grid, kT4Threads, 0, st>>>(a);
        return cudaGetLastError();
    }
    const size_t smem = toom_interp_smem(K, a);
    cudaError_t e = cudaFuncSetAttribute(toom_interp_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    toom_interp_kernel<K><<<grid, kT4Threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_toom_eval(uint32_t K, const ToomArgs &a, unsigned grid, cudaStream_t st)
{
    return K == 4u ? launch_pair<4>(a, grid, st, true) : K == 5u ? launch_pair<5>(a, grid, st, true)
                                                                 : cudaErrorInvalidValue;
}

cudaError_t launch_toom_interp(uint32_t K, const ToomArgs &a, unsigned grid, cudaStream_t st)
{
    return K == 4u ? launch_pair<4>(a, grid, st, false) : K == 5u ? launch_pair<5>(a, grid, st, false)
                                                                  : cudaErrorInvalidValue;
}

}  // namespace gf2x
