// unbalanced.cu -- operands of different sizes.  The product of a (na bits)
// and b (nb bits, nb <= na) is assembled from equal-size products:
//   padded:  both operands zero-extended to na bits, one product of size na
//            (the zero padding Sec. 3.2 applies to the Toom-3 evaluation
//            products, whose operands differ by 2w bits);
//   chunked: a cut into k chunks a_i of m = 64 ceil(nb/64) bits, so that
//            a = sum_i a_i X^(i m) and a b = sum_i (a_i b) X^(i m), the
//            splitting of Sec. 2.1 applied to one operand only; the k
//            products of size m run as one batch and overlap-add into the
//            result.
// pad_rows_kernel writes the operand rows of those products,
// overlap_add_kernel the result.  Both are memory-bound copies whose loops
// and addresses depend on the sizes only (constant time in the operand bits).
#include <cstdint>

#include <cuda_runtime.h>

namespace gf2x {

// Row r = p k + i of dst (Ld limbs) takes limbs [i step, i step + Ld) of
// source row p, with the bits at and above nsrc cleared and zeros past the
// source's ceil(nsrc/64) limbs.  step = 0 repeats the row k times.
__global__ void __launch_bounds__(256) pad_rows_kernel(uint64_t *dst, const uint64_t *src, size_t stride_src,
                                                       uint32_t nsrc, size_t count, uint32_t k, uint32_t Ld,
                                                       uint32_t step)
{
    const uint32_t Ls = (nsrc + 63u) / 64u;
    const uint64_t top = (nsrc & 63u) ? ((1ull << (nsrc & 63u)) - 1ull) : ~0ull;
    const size_t total = count * k * Ld;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / Ld;
        const uint32_t t = (uint32_t)(e - r * Ld);
        const size_t p = r / k;
        const uint32_t i = (uint32_t)(r - p * k);
        const uint64_t g = (uint64_t)i * step + t;
        uint64_t v = 0;
        if (g < Ls) {
            v = src[p * stride_src + g];
            if (g == Ls - 1u)
                v &= top;
        }
        dst[e] = v;
    }
}

// Limb j < Lu of result row p: the XOR of limb j - i step of product rows
// p k + i (Wp limbs each) over the chunks i whose product covers j.
__global__ void __launch_bounds__(256) overlap_add_kernel(uint64_t *out, size_t stride_out, uint32_t Lu,
                                                          const uint64_t *prod, uint32_t Wp, size_t count,
                                                          uint32_t k, uint32_t step)
{
    const size_t total = count * Lu;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const size_t p = e / Lu;
        const uint32_t j = (uint32_t)(e - p * Lu);
        const uint32_t hi = k - 1u < j / step ? k - 1u : j / step;
        const uint64_t *row = prod + p * k * (size_t)Wp;
        uint64_t v = 0;
        for (int32_t i = (int32_t)hi; i >= 0 && j - (uint32_t)i * step < Wp; --i)
            v ^= row[(size_t)i * Wp + (j - (uint32_t)i * step)];
        out[p * stride_out + j] = v;
    }
}

static unsigned grid_for(size_t total, int sm_count)
{
    const size_t blocks = (total + 255) / 256;
    const size_t cap = (size_t)(sm_count > 0 ? sm_count : 1) * 8;   // 8 CTAs of 256 per SM
    return (unsigned)(blocks < cap ? (blocks ? blocks : 1) : cap);
}

cudaError_t launch_pad_rows(uint64_t *dst, const uint64_t *src, size_t stride_src, uint32_t nsrc, size_t count,
                            uint32_t k, uint32_t Ld, uint32_t step, int sm_count, cudaStream_t st)
{
    pad_rows_kernel<<<grid_for(count * k * Ld, sm_count), 256, 0, st>>>(dst, src, stride_src, nsrc, count, k, Ld,
                                                                        step);
    return cudaGetLastError();
}

cudaError_t launch_overlap_add(uint64_t *out, size_t stride_out, uint32_t Lu, const uint64_t *prod, uint32_t Wp,
                               size_t count, uint32_t k, uint32_t step, int sm_count, cudaStream_t st)
{
    overlap_add_kernel<<<grid_for(count * Lu, sm_count), 256, 0, st>>>(out, stride_out, Lu, prod, Wp, count, k,
                                                                       step);
    return cudaGetLastError();
}

}  // namespace gf2x
