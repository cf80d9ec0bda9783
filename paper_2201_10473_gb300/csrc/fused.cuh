// fused.cuh -- one CTA multiplies one pair of binary polynomials entirely
// in shared memory: stage -> evaluate (Toom-3 / Karatsuba, breadth first)
// -> leaf products -> interpolate (bottom up) -> fold mod X^n - 1 -> store.
//
// Constant time: every loop bound, branch and shared/global address below
// depends only on the plan (n, sizes) and on thread indices, never on
// operand bits.  Operand bits only flow through XOR/AND/shift data paths.
#pragma once
#include <stdint.h>

#include "plan.h"

namespace gf2x {

__device__ __forceinline__ uint32_t fdiv(const FastDiv &f, uint32_t x)
{
    return f.m ? __umulhi(x, f.m) : x;
}

// ---------------------------------------------------------------- leaf
// Mask of bit 8q+7 of x (all ones or all zeros) by byte-sign replication:
// prmt with selector nibbles 8|q copies the sign of byte q into every byte.
template <uint32_t Q>
__device__ __forceinline__ uint32_t byte_sign_mask(uint32_t x)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(x), "n"(0x8888u | (Q * 0x1111u)));
    return d;
}

// a * X^s as S+1 words (0 < s < 32)
template <int S>
__device__ __forceinline__ void shift_words(const uint32_t (&a)[S], uint32_t (&r)[S + 1], uint32_t s)
{
    r[0] = a[0] << s;
#pragma unroll
    for (int k = 1; k < S; ++k)
        r[k] = __funnelshift_l(a[k - 1], a[k], s);
    r[S] = a[S - 1] >> (32u - s);
}

// S x S-word carry-less product by the comb method, in registers.  Bit
// 8q+7-u of a word of b contributes a * X^{8q} * X^{7-u}: eight steps u
// (high to low) shift the 2S-word accumulator left by one (funnel shifts),
// and in each, every word b[i] gives four masks -- the byte signs of
// b[i] << u, bits 31-u, 23-u, 15-u, 7-u -- that select a, a X^8, a X^16 and
// a X^24 (precomputed) into the accumulator at word i (AND with the mask:
// no branch).  32 S^2 + 83 S + 3 integer operations for (32S)^2 bit
// products, against 32 S^2 + 128 S for one accumulator shift, one mask and
// one b shift per bit (measured 3-5% faster on GB300 for S = 4..10).  This
// replaces the paper's Mult64 (Sec. 2.1, PCLMULQDQ), which the GPU does not
// have.  (Moving shifts to the FMA pipe with mul.hi measured slower: mul.hi
// issues at half rate.)  b is consumed.
template <int S>
__device__ __forceinline__ void comb(const uint32_t (&a)[S], uint32_t (&b)[S], uint32_t (&c)[2 * S])
{
    uint32_t a8[S + 1], a16[S + 1], a24[S + 1];
    shift_words<S>(a, a8, 8u);
    shift_words<S>(a, a16, 16u);
    shift_words<S>(a, a24, 24u);
#pragma unroll
    for (int i = 0; i < 2 * S; ++i)
        c[i] = 0u;
#pragma unroll 2
    for (int u = 0; u < 8; ++u) {
#pragma unroll
        for (int k = 2 * S - 1; k > 0; --k)
            c[k] = __funnelshift_l(c[k - 1], c[k], 1);
        c[0] <<= 1;
#pragma unroll
        for (int i = 0; i < S; ++i) {
            const uint32_t m3 = byte_sign_mask<3>(b[i]), m2 = byte_sign_mask<2>(b[i]);
            const uint32_t m1 = byte_sign_mask<1>(b[i]), m0 = byte_sign_mask<0>(b[i]);
            b[i] <<= 1;
#pragma unroll
            for (int k = 0; k <= S; ++k)
                c[i + k] ^= a24[k] & m3;
#pragma unroll
            for (int k = 0; k <= S; ++k)
                c[i + k] ^= a16[k] & m2;
#pragma unroll
            for (int k = 0; k <= S; ++k)
                c[i + k] ^= a8[k] & m1;
#pragma unroll
            for (int k = 0; k < S; ++k)
                c[i + k] ^= a[k] & m0;
        }
    }
}

template <int N>
__device__ __forceinline__ void load_words(uint32_t (&r)[N], const uint32_t *p)
{
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p + i);
        r[i] = t.x;
        r[i + 1] = t.y;
    }
}

template <int N>
__device__ __forceinline__ void store_words(uint32_t *p, const uint32_t (&r)[N])
{
#pragma unroll
    for (int i = 0; i < N; i += 2)
        *reinterpret_cast<uint2 *>(p + i) = make_uint2(r[i], r[i + 1]);
}

// Leaf slot: A (S words) then B (S words); the 2S-word product replaces them.
template <int S>
__device__ __forceinline__ void leaf_plain(uint32_t *slot)
{
    uint32_t a[S], b[S], c[2 * S];
    load_words<S>(a, slot);
    load_words<S>(b, slot + S);
    comb<S>(a, b, c);
    store_words<2 * S>(slot, c);
}

// Leaf slot of a 2-way Karatsuba node (Alg. 1, one level): A = A0 + X^{32S} A1,
// B likewise (2S words each); R = R0 + (R0 + R1 + R2) X^{32S} + R1 X^{64S}
// with R0 = A0 B0, R1 = A1 B1, R2 = (A0 + A1)(B0 + B1), all in registers.
template <int S>
__device__ __forceinline__ void leaf_k2(uint32_t *slot)
{
    uint32_t C[4 * S], r[2 * S], a[S], b[S];
    load_words<S>(a, slot);
    load_words<S>(b, slot + 2 * S);
    comb<S>(a, b, r);
#pragma unroll
    for (int k = 0; k < 2 * S; ++k)
        C[k] = r[k];
#pragma unroll
    for (int k = 2 * S; k < 4 * S; ++k)
        C[k] = 0u;
#pragma unroll
    for (int k = 0; k < 2 * S; ++k)
        C[S + k] ^= r[k];
    load_words<S>(a, slot + S);
    load_words<S>(b, slot + 3 * S);
    comb<S>(a, b, r);
#pragma unroll
    for (int k = 0; k < 2 * S; ++k) {
        C[2 * S + k] ^= r[k];
        C[S + k] ^= r[k];
    }
    {
        uint32_t a1[S], b1[S];
        load_words<S>(a, slot);
        load_words<S>(a1, slot + S);
        load_words<S>(b, slot + 2 * S);
        load_words<S>(b1, slot + 3 * S);
#pragma unroll
        for (int k = 0; k < S; ++k) {
            a[k] ^= a1[k];
            b[k] ^= b1[k];
        }
    }
    comb<S>(a, b, r);
#pragma unroll
    for (int k = 0; k < 2 * S; ++k)
        C[S + k] ^= r[k];
    store_words<4 * S>(slot, C);
}

template <int S>
__device__ __forceinline__ void leaf_pass(const GPlan &P, uint32_t *base, uint32_t nleaf)
{
    if (P.fuse_k2) {
        if constexpr (S <= 10) {
            for (uint32_t l = threadIdx.x; l < nleaf; l += blockDim.x)
                leaf_k2<S>(base + l * (4u * S));
        }
    } else {
        for (uint32_t l = threadIdx.x; l < nleaf; l += blockDim.x)
            leaf_plain<S>(base + l * (2u * S));
    }
}

// ---------------------------------------------------------------- staging
// Words 0..T0-1 of an operand: the caller's ceil(n/64) limbs read as 32-bit
// words, bits >= n cleared, zero padding up to the plan size.  A row that
// starts on a 16-byte boundary is read with 128-bit loads (four words per
// thread), any other (8-byte aligned) row with 64-bit loads; the choice
// depends on the address only.  Loads stay inside the row's ceil(n/64) limbs.
__device__ __forceinline__ uint32_t stage_word(uint32_t v, uint32_t w, uint32_t L32, uint32_t r)
{
    v = w < L32 ? v : 0u;
    return (w == L32 - 1 && r) ? (v & ((1u << r) - 1u)) : v;
}

__device__ __forceinline__ void stage_operand(uint32_t *dst, const uint64_t *src, const GPlan &P)
{
    const uint32_t L32 = P.L32, T0 = P.T0, r = P.n & 31u, W = 2u * P.L64;   // W: words in the row
    if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        for (uint32_t q = threadIdx.x; 4u * q < T0; q += blockDim.x) {
            const uint32_t w = 4u * q;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (w + 3u < W) {
                v = __ldg(s4 + q);
            } else if (w < W) {   // the row's last words (W is even)
                const uint2 h = __ldg(reinterpret_cast<const uint2 *>(src) + 2u * q);
                v.x = h.x;
                v.y = h.y;
            }
            const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k)
                if (w + k < T0)
                    dst[w + k] = stage_word(vv[k], w + k, L32, r);
        }
    } else {
        const uint2 *s2 = reinterpret_cast<const uint2 *>(src);
        for (uint32_t q = threadIdx.x; 2u * q < T0; q += blockDim.x) {
            const uint32_t w = 2u * q;
            const uint2 v = w < W ? __ldg(s2 + q) : make_uint2(0u, 0u);
            dst[w] = stage_word(v.x, w, L32, r);
            if (w + 1u < T0)
                dst[w + 1u] = stage_word(v.y, w + 1u, L32, r);
        }
    }
}

// ---------------------------------------------------------------- evaluation
// Children c_begin .. c_begin+c_count-1 (numbered over all parents of the
// pass) of one level: operand word e of child j of parent p.
__device__ __forceinline__ void eval_level(const GLevel &L, const uint32_t *__restrict__ par,
                                           uint32_t *__restrict__ ch, uint32_t c_begin, uint32_t c_count)
{
    const uint32_t E = L.E, twoE = 2u * E, T = L.T;
    const uint32_t total = c_count * twoE;
    for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const uint32_t cl = fdiv(L.div2E, idx);
        const uint32_t r = idx - cl * twoE;
        const uint32_t c = c_begin + cl;
        const uint32_t p = fdiv(L.divnch, c);
        const uint32_t j = c - p * L.nch;
        const uint32_t half = r >= E ? 1u : 0u;
        const uint32_t e = r - half * E;
        const uint32_t *X = par + p * (2u * T) + half * T;
        uint32_t v;
        if (L.kind == kKaratsuba) {
            // Alg. 1-3: child j multiplies A_i (single) or A_i + A_j (pair)
            const uint32_t s0 = L.sel[j][0], s1 = L.sel[j][1];
            v = X[s0 * E + e];
            if (s1 != 255u)
                v ^= X[s1 * E + e];
        } else {
            // Appendix D evaluation at 0, 1, x, x+1, inf, x = X^w (word shift W)
            const uint32_t np = L.np, W = L.W;
            const bool in = e < np;
            const uint32_t a0 = in ? X[e] : 0u;
            const uint32_t a1 = in ? X[np + e] : 0u;
            const uint32_t a2 = in ? X[2u * np + e] : 0u;
            const uint32_t a1x = (e >= W && e - W < np) ? X[np + e - W] : 0u;          // a1 * x
            const uint32_t a2x = (e >= 2u * W && e - 2u * W < np) ? X[2u * np + e - 2u * W] : 0u;  // a2 * x^2
            switch (j) {
            case 0: v = a0; break;                              // C(0)
            case 1: v = a0 ^ a1 ^ a2; break;                    // C(1)
            case 2: v = a0 ^ a1x ^ a2x; break;                  // C(x)
            case 3: v = a0 ^ a1 ^ a2 ^ a1x ^ a2x; break;        // C(x+1)
            default: v = a2; break;                             // C(inf)
            }
        }
        ch[cl * twoE + r] = v;
    }
}

// 2-way Karatsuba evaluation (Alg. 1), two words per thread: children
// (A0, B0), (A1, B1), (A0 + A1, B0 + B1) of every parent of the pass.
__device__ __forceinline__ void eval_k2(const GLevel &L, const uint32_t *__restrict__ par, uint32_t *__restrict__ ch,
                                        uint32_t npar)
{
    const uint32_t E = L.E, hE = E / 2u;
    const uint32_t total = npar * hE;
    for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const uint32_t p = fdiv(L.divhE, idx);
        const uint32_t e = 2u * (idx - p * hE);
        const uint32_t *X = par + p * (4u * E);
        const uint2 a0 = *reinterpret_cast<const uint2 *>(X + e);
        const uint2 a1 = *reinterpret_cast<const uint2 *>(X + E + e);
        const uint2 b0 = *reinterpret_cast<const uint2 *>(X + 2u * E + e);
        const uint2 b1 = *reinterpret_cast<const uint2 *>(X + 3u * E + e);
        uint32_t *C = ch + p * (6u * E);
        *reinterpret_cast<uint2 *>(C + e) = a0;
        *reinterpret_cast<uint2 *>(C + E + e) = b0;
        *reinterpret_cast<uint2 *>(C + 2u * E + e) = a1;
        *reinterpret_cast<uint2 *>(C + 3u * E + e) = b1;
        *reinterpret_cast<uint2 *>(C + 4u * E + e) = make_uint2(a0.x ^ a1.x, a0.y ^ a1.y);
        *reinterpret_cast<uint2 *>(C + 5u * E + e) = make_uint2(b0.x ^ b1.x, b0.y ^ b1.y);
    }
}

// 2-way Karatsuba reconstruction (Alg. 1): with M = R0 + R1 + R2,
// C[x] = R0[x], C[E+x] = R0[E+x] + M[x], C[2E+x] = M[E+x] + R1[x], C[3E+x] = R1[E+x].
__device__ __forceinline__ void interp_k2(const GLevel &L, const uint32_t *__restrict__ ch, uint32_t *__restrict__ par,
                                          uint32_t npar)
{
    const uint32_t E = L.E, hE = E / 2u;
    const uint32_t total = npar * hE;
    for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const uint32_t p = fdiv(L.divhE, idx);
        const uint32_t x = 2u * (idx - p * hE);
        const uint32_t *R = ch + p * (6u * E);
        const uint2 r0l = *reinterpret_cast<const uint2 *>(R + x);
        const uint2 r0h = *reinterpret_cast<const uint2 *>(R + E + x);
        const uint2 r1l = *reinterpret_cast<const uint2 *>(R + 2u * E + x);
        const uint2 r1h = *reinterpret_cast<const uint2 *>(R + 3u * E + x);
        const uint2 r2l = *reinterpret_cast<const uint2 *>(R + 4u * E + x);
        const uint2 r2h = *reinterpret_cast<const uint2 *>(R + 5u * E + x);
        const uint2 ml = make_uint2(r0l.x ^ r1l.x ^ r2l.x, r0l.y ^ r1l.y ^ r2l.y);
        const uint2 mh = make_uint2(r0h.x ^ r1h.x ^ r2h.x, r0h.y ^ r1h.y ^ r2h.y);
        uint32_t *C = par + p * (4u * E);
        *reinterpret_cast<uint2 *>(C + x) = r0l;
        *reinterpret_cast<uint2 *>(C + E + x) = make_uint2(r0h.x ^ ml.x, r0h.y ^ ml.y);
        *reinterpret_cast<uint2 *>(C + 2u * E + x) = make_uint2(mh.x ^ r1l.x, mh.y ^ r1l.y);
        *reinterpret_cast<uint2 *>(C + 3u * E + x) = r1h;
    }
}

// Two 2-way Karatsuba levels in one pass (Alg. 1 applied twice): parent
// operands of 4G words (quarters q0..q3) give the nine grandchildren
// (j1, j2), child j1 = (q0 q1), (q2 q3) or (q0+q2, q1+q3) and grandchild j2
// its low half, high half or their sum -- each grandchild word the XOR of 1,
// 2 or 4 quarter words at one offset.  Two words per thread.
__device__ __forceinline__ void eval_k2x2(const GLevel &L1, const GLevel &L2, const uint32_t *__restrict__ par,
                                          uint32_t *__restrict__ ch, uint32_t npar)
{
    const uint32_t G = L2.E, T = L1.T;   // T = 4G
    const uint32_t total = npar * (G / 2u);
    for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const uint32_t p = fdiv(L2.divhE, idx);
        const uint32_t e = 2u * idx - p * G;
        const uint32_t *X = par + p * (2u * T);
        uint32_t *C = ch + p * (18u * G);
#pragma unroll
        for (uint32_t op = 0; op < 2; ++op) {   // A, then B
            const uint32_t *Q = X + op * T;
            const uint2 q0 = *reinterpret_cast<const uint2 *>(Q + e);
            const uint2 q1 = *reinterpret_cast<const uint2 *>(Q + G + e);
            const uint2 q2 = *reinterpret_cast<const uint2 *>(Q + 2u * G + e);
            const uint2 q3 = *reinterpret_cast<const uint2 *>(Q + 3u * G + e);
            const uint2 q01 = make_uint2(q0.x ^ q1.x, q0.y ^ q1.y), q23 = make_uint2(q2.x ^ q3.x, q2.y ^ q3.y);
            const uint2 q02 = make_uint2(q0.x ^ q2.x, q0.y ^ q2.y), q13 = make_uint2(q1.x ^ q3.x, q1.y ^ q3.y);
            const uint2 v[9] = {q0, q1, q01, q2, q3, q23, q02, q13, make_uint2(q01.x ^ q23.x, q01.y ^ q23.y)};
            uint32_t *D = C + op * G + e;
#pragma unroll
            for (uint32_t g = 0; g < 9; ++g)
                *reinterpret_cast<uint2 *>(D + g * (2u * G)) = v[g];
        }
    }
}

// The reconstruction of such a pair: with Q the grandchild products (2G
// words, blocks of G), child j is R = Q0 + X^G (Q0+Q1+Q2) + X^2G Q1 and the
// parent P = R0 + X^2G (R0+R1+R2) + X^4G R1, eight blocks of G words per
// offset in registers.
__device__ __forceinline__ void interp_k2x2(const GLevel &L1, const GLevel &L2, const uint32_t *__restrict__ ch,
                                            uint32_t *__restrict__ par, uint32_t npar)
{
    const uint32_t G = L2.E, T = L1.T;
    const uint32_t total = npar * (G / 2u);
    for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const uint32_t p = fdiv(L2.divhE, idx);
        const uint32_t e = 2u * idx - p * G;
        const uint32_t *Q = ch + p * (18u * G) + e;
        uint2 R[3][4];
#pragma unroll
        for (uint32_t j = 0; j < 3; ++j) {
            const uint32_t *q = Q + j * (6u * G);
            const uint2 a0 = *reinterpret_cast<const uint2 *>(q);
            const uint2 a1 = *reinterpret_cast<const uint2 *>(q + G);
            const uint2 b0 = *reinterpret_cast<const uint2 *>(q + 2u * G);
            const uint2 b1 = *reinterpret_cast<const uint2 *>(q + 3u * G);
            const uint2 c0 = *reinterpret_cast<const uint2 *>(q + 4u * G);
            const uint2 c1 = *reinterpret_cast<const uint2 *>(q + 5u * G);
            const uint2 m0 = make_uint2(a0.x ^ b0.x ^ c0.x, a0.y ^ b0.y ^ c0.y);
            const uint2 m1 = make_uint2(a1.x ^ b1.x ^ c1.x, a1.y ^ b1.y ^ c1.y);
            R[j][0] = a0;
            R[j][1] = make_uint2(a1.x ^ m0.x, a1.y ^ m0.y);
            R[j][2] = make_uint2(m1.x ^ b0.x, m1.y ^ b0.y);
            R[j][3] = b1;
        }
        uint32_t *C = par + p * (2u * T) + e;
#pragma unroll
        for (uint32_t b = 0; b < 8; ++b) {
            uint2 v = make_uint2(0u, 0u);
            if (b < 4)
                v = R[0][b];
            if (b >= 2 && b < 6)
                v = make_uint2(v.x ^ R[0][b - 2].x ^ R[1][b - 2].x ^ R[2][b - 2].x,
                               v.y ^ R[0][b - 2].y ^ R[1][b - 2].y ^ R[2][b - 2].y);
            if (b >= 4)
                v = make_uint2(v.x ^ R[1][b - 4].x, v.y ^ R[1][b - 4].y);
            *reinterpret_cast<uint2 *>(C + b * G) = v;
        }
    }
}

// ---------------------------------------------------------------- interpolation
// k-way Karatsuba reconstruction: word q of the parent product is the XOR of
// term_p[q - pE] for the (at most two) positions p covering q.
__device__ __forceinline__ void interp_karatsuba(const GLevel &L, const uint32_t *__restrict__ ch,
                                                 uint32_t *__restrict__ par, uint32_t npar)
{
    const uint32_t E = L.E, twoE = 2u * E, twoT = 2u * L.T, k = L.k;
    const uint32_t total = npar * twoT;
    for (uint32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const uint32_t p = fdiv(L.div2T, idx);
        const uint32_t q = idx - p * twoT;
        const uint32_t *R = ch + p * L.nch * twoE;
        const uint32_t hi = fdiv(L.divE, q);
        uint32_t v = 0u;
#pragma unroll
        for (uint32_t u = 0; u < 2; ++u) {
            if (hi < u)
                continue;
            const uint32_t pos = hi - u;
            if (pos > 2u * k - 2u)
                continue;
            const uint32_t x = q - pos * E;
            const uint32_t nt = L.nterms[pos];
            for (uint32_t t = 0; t < nt; ++t)
                v ^= R[L.terms[pos][t] * twoE + x];
        }
        par[idx] = v;
    }
}

// In-place prefix XOR over W-word blocks (division by x+1 = X^w + 1, Sec. 3.2:
// the quotient is the product with sum_i X^{wi}, i.e. Q[i] = P[i] ^ Q[i-W]),
// for nseg segments `stride` words apart, each `len` words long.  Three
// passes: chunk totals, exclusive scan of the totals, chunk rescans.
static __device__ void scan_xor_blocks(uint32_t *base, uint32_t nseg, uint32_t stride, uint32_t len, uint32_t W,
                                uint32_t *part, uint32_t part_words)
{
    const uint32_t rows = (len + W - 1) / W;
    uint32_t nchunk = part_words / (nseg * W);
    nchunk = nchunk < 1u ? 1u : (nchunk > 32u ? 32u : nchunk);
    if (nchunk > rows)
        nchunk = rows;
    const uint32_t rpc = (rows + nchunk - 1) / nchunk;
    const uint32_t per_seg = W * nchunk;
    const uint32_t ntask = nseg * per_seg;
    for (uint32_t t = threadIdx.x; t < ntask; t += blockDim.x) {
        const uint32_t seg = t / per_seg, rem = t - seg * per_seg, c = rem / W, col = rem - c * W;
        const uint32_t *a = base + seg * stride;
        const uint32_t r0 = c * rpc, r1 = min(rows, r0 + rpc);
        uint32_t acc = 0u;
        for (uint32_t r = r0; r < r1; ++r) {
            const uint32_t i = r * W + col;
            if (i < len)
                acc ^= a[i];
        }
        part[t] = acc;
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < nseg * W; s += blockDim.x) {
        const uint32_t seg = s / W, col = s - seg * W;
        uint32_t run = 0u;
        for (uint32_t c = 0; c < nchunk; ++c) {
            const uint32_t t = seg * per_seg + c * W + col;
            const uint32_t v = part[t];
            part[t] = run;
            run ^= v;
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < ntask; t += blockDim.x) {
        const uint32_t seg = t / per_seg, rem = t - seg * per_seg, c = rem / W, col = rem - c * W;
        uint32_t *a = base + seg * stride;
        const uint32_t r0 = c * rpc, r1 = min(rows, r0 + rpc);
        uint32_t acc = part[t];
        for (uint32_t r = r0; r < r1; ++r) {
            const uint32_t i = r * W + col;
            if (i < len) {
                acc ^= a[i];
                a[i] = acc;
            }
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void flag_error(uint32_t *err, uint32_t code)
{
    if (err)
        atomicOr(err, code);
}

// Toom-3 interpolation (Appendix D), as the sequence
//   c3 = ((v0+v1+vx+vx1)/x)/(x+1)
//   c2 = ((vx+v0)/x + c3 x^2 + c4 x^3 + v1 + v0 + c3 + c4)/(x+1)
//   c1 = v1 + v0 + c2 + c3 + c4,   c0 = v0,  c4 = v_inf
// (two word shifts and two prefix-XOR scans; it reproduces the rows of
// M^-1), then C = sum_i c_i X^{32 n' i}.
static __device__ void interp_toom3(const GPlan &P, const GLevel &L, const uint32_t *__restrict__ ch,
                             uint32_t *__restrict__ par, uint32_t *tmp, uint32_t *part, uint32_t npar,
                             uint32_t *err)
{
    const uint32_t E = L.E, twoE = 2u * E, W = L.W, np = L.np, twonp = 2u * np;
    const uint32_t len = P.checked ? twoE - W : twonp;  // words of c3, c2 computed
    const uint32_t tstride = 4u * E;                     // per parent: c3 at [0,2E), c2 at [2E,4E)
    // (1) t = (v0 + v1 + vx + vx1) / x
    for (uint32_t idx = threadIdx.x; idx < npar * len; idx += blockDim.x) {
        const uint32_t p = idx / len, x = idx - p * len;
        const uint32_t *R = ch + p * 5u * twoE;
        tmp[p * tstride + x] = R[x + W] ^ R[twoE + x + W] ^ R[2u * twoE + x + W] ^ R[3u * twoE + x + W];
    }
    if (P.checked) {
        for (uint32_t idx = threadIdx.x; idx < npar * W; idx += blockDim.x) {
            const uint32_t p = idx / W, x = idx - p * W;
            const uint32_t *R = ch + p * 5u * twoE;
            if ((R[x] ^ R[twoE + x] ^ R[2u * twoE + x] ^ R[3u * twoE + x]) | (R[2u * twoE + x] ^ R[x]))
                flag_error(err, kErrDivX);
        }
    }
    __syncthreads();
    // (2) c3 = t / (x+1)
    scan_xor_blocks(tmp, npar, tstride, len, W, part, P.part_words);
    // (3) numerator of c2
    for (uint32_t idx = threadIdx.x; idx < npar * len; idx += blockDim.x) {
        const uint32_t p = idx / len, x = idx - p * len;
        const uint32_t *R = ch + p * 5u * twoE;
        const uint32_t *c3 = tmp + p * tstride;
        const uint32_t *c4 = R + 4u * twoE;
        uint32_t v = R[2u * twoE + x + W] ^ R[x + W];          // (vx + v0) / x
        if (x >= 2u * W)
            v ^= c3[x - 2u * W];                                // c3 x^2
        if (x >= 3u * W)
            v ^= c4[x - 3u * W];                                // c4 x^3
        v ^= R[twoE + x] ^ R[x] ^ c3[x] ^ c4[x];                // v1 + v0 + c3 + c4
        tmp[p * tstride + twoE + x] = v;
    }
    if (P.checked) {
        for (uint32_t idx = threadIdx.x; idx < npar * (len - twonp); idx += blockDim.x) {
            const uint32_t p = idx / (len - twonp), x = twonp + idx % (len - twonp);
            if (tmp[p * tstride + x])
                flag_error(err, kErrDivX1);
        }
    }
    __syncthreads();
    // (4) c2 = numerator / (x+1)
    scan_xor_blocks(tmp + twoE, npar, tstride, len, W, part, P.part_words);
    if (P.checked) {
        for (uint32_t idx = threadIdx.x; idx < npar * (len - twonp); idx += blockDim.x) {
            const uint32_t p = idx / (len - twonp), x = twonp + idx % (len - twonp);
            if (tmp[p * tstride + twoE + x])
                flag_error(err, kErrDivX1);
        }
    }
    // (5) recomposition C = c0 + c1 X^n' + c2 X^2n' + c3 X^3n' + c4 X^4n'
    const uint32_t twoT = 2u * L.T;  // = 6 n'
    for (uint32_t idx = threadIdx.x; idx < npar * twoT; idx += blockDim.x) {
        const uint32_t p = idx / twoT, q = idx - p * twoT;
        const uint32_t *R = ch + p * 5u * twoE;
        const uint32_t *c3 = tmp + p * tstride;
        const uint32_t *c2 = c3 + twoE;
        uint32_t v = 0u;
#pragma unroll
        for (uint32_t i = 0; i < 5; ++i) {
            if (q < i * np)
                continue;
            const uint32_t y = q - i * np;
            if (y >= twonp)
                continue;
            switch (i) {
            case 0: v ^= R[y]; break;
            case 1: v ^= R[twoE + y] ^ R[y] ^ c3[y] ^ R[4u * twoE + y] ^ c2[y]; break;
            case 2: v ^= c2[y]; break;
            case 3: v ^= c3[y]; break;
            default: v ^= R[4u * twoE + y]; break;
            }
        }
        par[idx] = v;
    }
    __syncthreads();
}

__device__ __forceinline__ void interp_level(const GPlan &P, const GLevel &L, const uint32_t *ch, uint32_t *par,
                                             uint32_t *sm, uint32_t npar, uint32_t *err)
{
    if (L.kind == kKaratsuba && L.k == 2u && !(L.E & 1u)) {
        interp_k2(L, ch, par, npar);
        __syncthreads();
    } else if (L.kind == kKaratsuba) {
        interp_karatsuba(L, ch, par, npar);
        __syncthreads();
    } else {
        interp_toom3(P, L, ch, par, sm + P.tmp_off, sm + P.part_off, npar, err);
    }
}

// ---------------------------------------------------------------- epilogue
// Full product: the first ceil((2n-1)/64) limbs.  Reduced product:
// r = (c mod X^n) + (c >> n), since X^n = 1 in F2[X]/(X^n - 1) and deg c <= 2n-2
// (Sec. 1, circulant isomorphism).
__device__ __forceinline__ uint32_t fold_word(const GPlan &P, const uint32_t *C, uint32_t q, uint32_t twoT)
{
    const uint32_t sh = P.n >> 5, s = P.n & 31u, L32 = P.L32;
    const uint32_t lo = q < twoT ? C[q] : 0u;
    const uint32_t i0 = q + sh;
    const uint32_t h0 = i0 < twoT ? C[i0] : 0u;
    const uint32_t h1 = i0 + 1u < twoT ? C[i0 + 1u] : 0u;
    uint32_t v = lo ^ __funnelshift_r(h0, h1, s);
    if (q >= L32)
        v = 0u;
    else if (q == L32 - 1 && s)
        v &= (1u << s) - 1u;
    return v;
}

// Results leave as whole 64-bit limbs (one 8-byte store per limb).
__device__ __forceinline__ void epilogue(const GPlan &P, const DevItem &it, const uint32_t *C, uint32_t *err)
{
    uint2 *o2 = reinterpret_cast<uint2 *>(it.out);
    const uint32_t twoT = 2u * P.T0;
    if (it.flags & 1u) {
        for (uint32_t l = threadIdx.x; l < P.L64; l += blockDim.x)
            o2[l] = make_uint2(fold_word(P, C, 2u * l, twoT), fold_word(P, C, 2u * l + 1u, twoT));
    } else {
        for (uint32_t l = threadIdx.x; l < P.Lfull64; l += blockDim.x) {
            const uint32_t q = 2u * l;
            o2[l] = make_uint2(q < twoT ? C[q] : 0u, q + 1u < twoT ? C[q + 1u] : 0u);
        }
    }
    if (P.checked) {
        const uint32_t top = 2u * P.n - 1u;  // first bit that must be zero
        for (uint32_t q = (top >> 5) + threadIdx.x; q < twoT; q += blockDim.x) {
            const uint32_t mask = (q == (top >> 5)) ? ~((1u << (top & 31u)) - 1u) : ~0u;
            if (C[q] & mask)
                flag_error(err, kErrPad);
        }
    }
}

// ---------------------------------------------------------------- one product
__device__ __forceinline__ void eval_pass(const GLevel &L, const uint32_t *par, uint32_t *ch, uint32_t c_begin,
                                          uint32_t c_count, uint32_t npar)
{
    if (L.kind == kKaratsuba && L.k == 2u && !(L.E & 1u) && c_begin == 0u && c_count == 3u * npar)
        eval_k2(L, par, ch, npar);
    else
        eval_level(L, par, ch, c_begin, c_count);
}

// One level's evaluation pass (a pair's first level runs both; its second none).
__device__ __forceinline__ void eval_step(const GPlan &P, uint32_t l, uint32_t *sm)
{
    const GLevel &L = P.lev[l];
    if (L.pair == 2u)
        return;
    if (L.pair == 1u)
        eval_k2x2(L, P.lev[l + 1], sm + L.in_off, sm + L.ch_off, L.npar);
    else
        eval_pass(L, sm + L.in_off, sm + L.ch_off, 0u, L.npar * L.nch, L.npar);
    __syncthreads();
}

__device__ __forceinline__ void interp_step(const GPlan &P, uint32_t l, uint32_t *sm, uint32_t *err)
{
    const GLevel &L = P.lev[l];
    if (L.pair == 2u)
        return;
    if (L.pair == 1u) {
        interp_k2x2(L, P.lev[l + 1], sm + L.ch_off, sm + L.in_off, L.npar);
        __syncthreads();
    } else {
        interp_level(P, L, sm + L.ch_off, sm + L.in_off, sm, L.npar, err);
    }
}

template <int S>
__device__ void run_product(const GPlan &P, const DevItem &it, uint32_t *sm, uint32_t *err)
{
    uint32_t *top = sm + P.top_off;
    stage_operand(top, it.a, P);
    stage_operand(top + P.T0, it.b, P);
    __syncthreads();
    const uint32_t nlev = P.nlev;
    const uint32_t ne = nlev - P.fuse_k2;   // levels run as shared-memory passes
    if (nlev == 0) {
        if (threadIdx.x == 0)
            leaf_plain<S>(top);
        __syncthreads();
    } else {
        uint32_t *leaf_base = sm + (P.fuse_k2 ? P.lev[nlev - 1].in_off : P.lev[nlev - 1].ch_off);
        if (!P.seq_top) {
            for (uint32_t l = 0; l < ne; ++l)
                eval_step(P, l, sm);
            leaf_pass<S>(P, leaf_base, P.nleaf_pass);
            __syncthreads();
            for (int l = (int)ne - 1; l >= 0; --l)
                interp_step(P, (uint32_t)l, sm, err);
        } else {
            const GLevel &L0 = P.lev[0];
            const uint32_t twoE0 = 2u * L0.E;
            for (uint32_t j = 0; j < L0.nch; ++j) {
                eval_level(L0, sm + L0.in_off, sm + L0.ch_off, j, 1u);
                __syncthreads();
                for (uint32_t l = 1; l < ne; ++l)
                    eval_step(P, l, sm);
                leaf_pass<S>(P, leaf_base, P.nleaf_pass);
                __syncthreads();
                for (int l = (int)ne - 1; l >= 1; --l)
                    interp_step(P, (uint32_t)l, sm, err);
                const uint32_t *src = sm + L0.ch_off;
                uint32_t *dst = sm + P.prod_off + j * twoE0;
                for (uint32_t w = threadIdx.x; w < twoE0; w += blockDim.x)
                    dst[w] = src[w];
                __syncthreads();
            }
            interp_level(P, L0, sm + P.prod_off, sm + L0.in_off, sm, 1u, err);
        }
    }
    epilogue(P, it, top, err);
}

__device__ __forceinline__ DevItem fetch_item(const LaunchArgs &args, uint32_t i)
{
    if (args.mode == kItemsArray)
        return args.items[i];
    if (args.mode == kItemsUser) {
        DevItem it = args.items[i];
        it.plan = it.plan == 0u ? kEmptyItem : (it.plan <= 131072u ? __ldg(args.plan_of_n + it.plan) : kNoPlan);
        return it;
    }
    DevItem it = args.base;
    if (args.mode == kItemsStrided) {
        if (!args.shared_a)
            it.a += (uint64_t)i * args.stride_in;
        it.b += (uint64_t)i * args.stride_in;
        it.out += (uint64_t)i * args.stride_out;
    }
    return it;
}

template <int S>
struct LeafTraits {
    static constexpr int kMaxThreads = S <= 6 ? 768 : 512;
};

__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

template <int S>
__global__ void __launch_bounds__(LeafTraits<S>::kMaxThreads, 1)
fused_mul_kernel(const LaunchArgs args)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ GPlan P;
    __shared__ uint32_t next_item;
    const uint32_t smem_avail = dynamic_smem_bytes();
    const uint32_t step = args.persistent ? gridDim.x : args.count;
    uint32_t loaded = kEmptyItem;   // plan slot currently in P (none)
    uint32_t i = blockIdx.x;
    if (args.work_counter) {   // dynamic order: items are taken from the counter (sizes only decide the cost)
        if (threadIdx.x == 0)
            next_item = atomicAdd(args.work_counter, 1u);
        __syncthreads();
        i = next_item;
    }
    while (i < args.count) {
        const DevItem it = fetch_item(args, i);
        bool run = true;
        if (it.plan >= kEmptyItem) {  // uniform over the CTA: every thread read the same item
            if (it.plan == kNoPlan && threadIdx.x == 0)
                flag_error(args.err, kErrNoPlan);
            run = false;
        } else {
            __syncthreads();   // the previous product is done with shared memory
            if (it.plan != loaded) {   // uniform: a persistent CTA of a uniform batch loads its plan once
                const uint32_t *src = reinterpret_cast<const uint32_t *>(args.plans + it.plan);
                uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
                for (uint32_t w = threadIdx.x; w < sizeof(GPlan) / 4; w += blockDim.x)
                    dst[w] = __ldg(src + w);
                loaded = it.plan;
                __syncthreads();
            }
            // a plan made for another leaf size or more shared memory than this
            // launch has is refused (uniform over the CTA), never run
            if (P.S != (uint32_t)S || 4u * P.smem_words > smem_avail || P.nlev > (uint32_t)kMaxLevels) {
                if (threadIdx.x == 0)
                    flag_error(args.err, kErrPlanMismatch);
                run = false;
            }
        }
        if (run)
            run_product<S>(P, it, sm, args.err);
        if (args.work_counter) {
            __syncthreads();   // every thread has read next_item
            if (threadIdx.x == 0)
                next_item = atomicAdd(args.work_counter, 1u);
            __syncthreads();
            i = next_item;
        } else {
            i += step;
        }
    }
}

// Host launcher, one instantiation per compiled leaf size.
template <int S>
cudaError_t launch_fused(const LaunchArgs &args, unsigned grid, unsigned block, size_t smem, cudaStream_t stream)
{
    fused_mul_kernel<S><<<grid, block, smem, stream>>>(args);
    return cudaGetLastError();
}

template <int S>
cudaError_t prepare_fused(int *max_blocks_per_sm, unsigned block, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(fused_mul_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         232448 - (int)sizeof(GPlan) - 256);
    if (e != cudaSuccess)
        return e;
    if (max_blocks_per_sm)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, fused_mul_kernel<S>, (int)block, smem);
    return e;
}

}  // namespace gf2x
