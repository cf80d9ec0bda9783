// copy_rows.cu -- gf2x_copy_rows: a device list of (src, dst, limbs) row
// copies in one launch.  The serving loop stages the operands of the requests
// it admits into their slots of its device-memory budget with it (one launch
// per batch, capturable in a CUDA graph with the products).  Not part of the
// paper's method: plumbing of the request loop, kept in CUDA so that no
// library or framework kernel runs on the serving path.
#include <cstdint>

#include <cuda_runtime.h>

#include "gf2x_gb300.h"

namespace gf2x {

// One CTA per row (grid-stride over rows), 8-byte words; entries with
// limbs = 0 are padding.
__global__ void __launch_bounds__(128) copy_rows_kernel(const gf2x_copy_row *__restrict__ rows, uint64_t count)
{
    for (uint64_t r = blockIdx.x; r < count; r += gridDim.x) {
        const gf2x_copy_row e = rows[r];
        for (uint64_t i = threadIdx.x; i < e.limbs; i += blockDim.x)
            e.dst[i] = e.src[i];
    }
}

cudaError_t launch_copy_rows(const gf2x_copy_row *rows, size_t count, int sm_count, cudaStream_t st)
{
    const unsigned grid = (unsigned)(count < 8ull * (unsigned)sm_count ? count : 8ull * (unsigned)sm_count);
    if (grid == 0)
        return cudaSuccess;
    copy_rows_kernel<<<grid, 128, 0, st>>>(rows, count);
    return cudaGetLastError();
}

}  // namespace gf2x
