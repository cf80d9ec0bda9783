// split.cu -- the top level of a split plan across CTAs.  split_eval_kernel
// evaluates level 0 of every product (Toom-3 points or Karatsuba sums) into
// global scratch; the children are then multiplied in place by the fused
// kernel as independent full products; split_interp_kernel reads the
// children's products back, interpolates level 0 and folds / stores the
// result.  Same constant-time rules as the fused kernel.
#include "fused.cuh"
#include "launchers.h"

namespace gf2x {

// one item's scratch: nch slots of 2E words (operands A|B, later the product)
__device__ __forceinline__ uint32_t *item_scratch(uint32_t *scratch, const GLevel &L, uint32_t i)
{
    return scratch + (size_t)i * L.nch * 2u * L.E;
}

__device__ __forceinline__ void copy_words(uint32_t *dst, const uint32_t *src, uint32_t words)
{
    // 16-byte aligned, words a multiple of 4 (slots are 2E words with E even)
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (uint32_t w = threadIdx.x; w < words / 4u; w += blockDim.x)
        d4[w] = s4[w];
    for (uint32_t w = (words & ~3u) + threadIdx.x; w < words; w += blockDim.x)
        dst[w] = src[w];
}

__device__ __forceinline__ bool load_top_plan(GPlan &P, const LaunchArgs &args, const DevItem &it)
{
    const uint32_t *src = reinterpret_cast<const uint32_t *>(args.plans + it.plan);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
    for (uint32_t w = threadIdx.x; w < sizeof(GPlan) / 4; w += blockDim.x)
        dst[w] = __ldg(src + w);
    __syncthreads();
    return P.split == 1u && P.nlev == 1u && 4u * P.smem_words <= dynamic_smem_bytes();
}

__global__ void __launch_bounds__(512, 1) split_eval_kernel(const LaunchArgs args, uint32_t *scratch)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ GPlan P;
    const uint32_t step = args.persistent ? gridDim.x : args.count;
    for (uint32_t i = blockIdx.x; i < args.count; i += step) {
        const DevItem it = fetch_item(args, i);
        __syncthreads();
        if (!load_top_plan(P, args, it)) {
            if (threadIdx.x == 0)
                flag_error(args.err, kErrPlanMismatch);
            continue;
        }
        const GLevel &L = P.lev[0];
        uint32_t *top = sm + P.top_off;
        stage_operand(top, it.a, P);
        stage_operand(top + P.T0, it.b, P);
        __syncthreads();
        eval_level(L, sm + L.in_off, sm + L.ch_off, 0u, L.nch);
        __syncthreads();
        copy_words(item_scratch(scratch, L, i), sm + L.ch_off, L.nch * 2u * L.E);
    }
}

__global__ void __launch_bounds__(512, 1) split_interp_kernel(const LaunchArgs args, const uint32_t *scratch)
{
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ GPlan P;
    const uint32_t step = args.persistent ? gridDim.x : args.count;
    for (uint32_t i = blockIdx.x; i < args.count; i += step) {
        const DevItem it = fetch_item(args, i);
        __syncthreads();
        if (!load_top_plan(P, args, it)) {
            if (threadIdx.x == 0)
                flag_error(args.err, kErrPlanMismatch);
            continue;
        }
        const GLevel &L = P.lev[0];
        copy_words(sm + L.ch_off, item_scratch(const_cast<uint32_t *>(scratch), L, i), L.nch * 2u * L.E);
        __syncthreads();
        interp_level(P, L, sm + L.ch_off, sm + L.in_off, sm, 1u, args.err);
        epilogue(P, it, sm + P.top_off, args.err);
    }
}

cudaError_t launch_split_eval(const LaunchArgs &a, uint32_t *scratch, unsigned grid, unsigned block, size_t smem,
                              cudaStream_t st)
{
    split_eval_kernel<<<grid, block, smem, st>>>(a, scratch);
    return cudaGetLastError();
}

cudaError_t launch_split_interp(const LaunchArgs &a, const uint32_t *scratch, unsigned grid, unsigned block,
                                size_t smem, cudaStream_t st)
{
    split_interp_kernel<<<grid, block, smem, st>>>(a, scratch);
    return cudaGetLastError();
}

cudaError_t prepare_split()
{
    const int smem = 232448 - (int)sizeof(GPlan) - 256;
    cudaError_t e = cudaFuncSetAttribute(split_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(split_interp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

}  // namespace gf2x
