// launchers.h -- per-leaf-size entry points of the fused kernel.
#pragma once
#include <cuda_runtime.h>

#include "gf2x_gb300.h"
#include "plan.h"

namespace gf2x {
#define GF2X_DECLARE_LEAF(S)                                                                              \
    cudaError_t launch_fused_s##S(const LaunchArgs &a, unsigned g, unsigned b, size_t sm, cudaStream_t st); \
    cudaError_t prepare_fused_s##S(int *blocks, unsigned b, size_t sm);
GF2X_DECLARE_LEAF(4)
GF2X_DECLARE_LEAF(6)
GF2X_DECLARE_LEAF(8)
GF2X_DECLARE_LEAF(10)
GF2X_DECLARE_LEAF(12)
GF2X_DECLARE_LEAF(16)
#undef GF2X_DECLARE_LEAF

cudaError_t launch_split_eval(const LaunchArgs &a, uint32_t *scratch, unsigned grid, unsigned block, size_t smem,
                              cudaStream_t st);
cudaError_t launch_split_interp(const LaunchArgs &a, const uint32_t *scratch, unsigned grid, unsigned block,
                                size_t smem, cudaStream_t st);
cudaError_t prepare_split();

// operands of different sizes (unbalanced.cu)
cudaError_t launch_pad_rows(uint64_t *dst, const uint64_t *src, size_t stride_src, uint32_t nsrc, size_t count,
                            uint32_t k, uint32_t Ld, uint32_t step, int sm_count, cudaStream_t st);
cudaError_t launch_overlap_add(uint64_t *out, size_t stride_out, uint32_t Lu, const uint64_t *prod, uint32_t Wp,
                               size_t count, uint32_t k, uint32_t step, int sm_count, cudaStream_t st);

// constant-time sparse x dense product mod X^n - 1 (sparse.cu)
constexpr uint32_t kSparseMaxN = 65536;
struct SparseArgs {
    const uint64_t *a;        // dense rows, ceil(n/64) limbs, stride_a limbs apart
    const uint32_t *pos;      // w positions per product, stride_pos entries apart
    uint64_t *r;              // result rows, ceil(n/64) limbs, stride_r limbs apart
    size_t stride_a, stride_pos, stride_r;
    uint32_t n, w, count;
    uint32_t T;               // bits of the largest word offset n/32
    uint32_t pre;             // its top bits applied in shared memory first
    uint32_t d_words, b_words; // shared words: doubled vector, each warp's stage buffer
};
struct SparseShape {
    uint32_t N, T;            // words of a, bits of the largest word offset n/32
    uint32_t R, QH, C;        // result registers per lane, register offsets up to QH, window registers
    uint32_t pre, d_words, b_words;
};
bool sparse_shape(uint32_t n, SparseShape *sh);
size_t sparse_smem_bytes(const SparseShape &sh);
cudaError_t launch_sparse_mulmod(const SparseArgs &args, const SparseShape &sh, int sm_count, cudaStream_t st);

// Toom-4 and Toom-5 top levels (toom.cu)
struct ToomArgs {
    const uint64_t *a, *b;    // operand rows, stride_in limbs apart
    uint64_t *out;            // result rows, stride_out limbs apart
    size_t stride_in, stride_out;
    uint32_t n, count, flags;
    uint32_t m, E, W, OW;     // part words, child operand words, interpolation and product buffer words
    uint32_t *opnd;           // per product 2K - 1 slots of 2E words (A(p_j) | B(p_j))
    const uint32_t *prod;     // per product 2K - 1 child products of 2E words
    uint32_t *err;            // checked mode: error word for inexact divisions (else null)
};
bool toom_shape(uint32_t K, uint32_t n, ToomArgs *a);
size_t toom_interp_smem(uint32_t K, const ToomArgs &a);
cudaError_t launch_toom_eval(uint32_t K, const ToomArgs &a, unsigned grid, cudaStream_t st);
cudaError_t launch_toom_interp(uint32_t K, const ToomArgs &a, unsigned grid, cudaStream_t st);

// shared-operand circulant products on the tensor cores (tc_circulant.cu)
constexpr uint32_t kTcMaxN = 65536;
struct TcShape {
    uint32_t S;               // K-steps of 64 inputs (limbs of b)
    uint32_t V;               // units of 480 positions
    uint32_t qwords;          // 32-bit words of parities per product (q order)
    uint32_t rwin;            // bytes of one unit's window of R
    uint32_t inv32;           // 32^-1 mod n
    size_t rseq_bytes;        // bytes of R
};
bool tc_shape(uint32_t n, size_t count, TcShape *sh);   // n odd, 1 <= n <= kTcMaxN
size_t tc_group_bytes(const TcShape &sh, size_t products);
cudaError_t prepare_tc();
cudaError_t launch_tc_rseq(const uint64_t *a, uint32_t n, const TcShape &sh, uint8_t *rseq, int sm_count,
                           cudaStream_t st);
cudaError_t launch_tc_group(const uint64_t *b, size_t stride_b, uint64_t *out, size_t stride_out, uint32_t n,
                            uint32_t count, const TcShape &sh, const uint8_t *rseq, uint8_t *scratch, uint32_t *err,
                            int sm_count, cudaStream_t st);

// row copies of the serving loop (copy_rows.cu)
cudaError_t launch_copy_rows(const gf2x_copy_row *rows, size_t count, int sm_count, cudaStream_t st);

typedef cudaError_t (*LaunchFn)(const LaunchArgs &, unsigned, unsigned, size_t, cudaStream_t);
typedef cudaError_t (*PrepareFn)(int *, unsigned, size_t);

// launcher for leaf size S (null if not compiled)
inline LaunchFn launcher_for(uint32_t S)
{
    switch (S) {
    case 4: return launch_fused_s4;
    case 6: return launch_fused_s6;
    case 8: return launch_fused_s8;
    case 10: return launch_fused_s10;
    case 12: return launch_fused_s12;
    case 16: return launch_fused_s16;
    default: return nullptr;
    }
}
inline PrepareFn preparer_for(uint32_t S)
{
    switch (S) {
    case 4: return prepare_fused_s4;
    case 6: return prepare_fused_s6;
    case 8: return prepare_fused_s8;
    case 10: return prepare_fused_s10;
    case 12: return prepare_fused_s12;
    case 16: return prepare_fused_s16;
    default: return nullptr;
    }
}
}  // namespace gf2x
