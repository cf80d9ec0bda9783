// Instantiates the fused multiplication kernel for a leaf of 16 32-bit words.
#include "fused.cuh"
#include "launchers.h"

namespace gf2x {
cudaError_t launch_fused_s16(const LaunchArgs &a, unsigned g, unsigned b, size_t sm, cudaStream_t st)
{
    return launch_fused<16>(a, g, b, sm, st);
}
cudaError_t prepare_fused_s16(int *blocks, unsigned b, size_t sm) { return prepare_fused<16>(blocks, b, sm); }
}  // namespace gf2x
