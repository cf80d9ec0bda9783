// Warp-level tensor MMA throughput (mma.sync) on sm_103a: s8, f16 and e4m3 inputs.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
template <int KIND>
__global__ void probe(float* out, int iters) {
  uint32_t a[4], b[2];
  for (int i = 0; i < 4; ++i) a[i] = 0x3c003c00u ^ (threadIdx.x * (i + 1));
  for (int i = 0; i < 2; ++i) b[i] = 0x3c003c00u ^ (threadIdx.x * (i + 7));
  float acc[4][4] = {};
  int iacc[4][4] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (KIND == 0) {
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
          : "+r"(iacc[u][0]), "+r"(iacc[u][1]), "+r"(iacc[u][2]), "+r"(iacc[u][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
      } else if (KIND == 1) {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
          : "+f"(acc[u][0]), "+f"(acc[u][1]), "+f"(acc[u][2]), "+f"(acc[u][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
      } else {
        asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
          : "+f"(acc[u][0]), "+f"(acc[u][1]), "+f"(acc[u][2]), "+f"(acc[u][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
      }
    }
  }
  float s = 0;
  for (int u = 0; u < 4; ++u) for (int i = 0; i < 4; ++i) s += acc[u][i] + (float)iacc[u][i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  float* out; cudaMalloc(&out, 4 << 24);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* names[] = {"mma.sync s8 m16n8k32", "mma.sync f16 m16n8k16", "mma.sync e4m3 m16n8k32"};
  const double macs[] = {16.0 * 8 * 32, 16.0 * 8 * 16, 16.0 * 8 * 32};
  for (int kind = 0; kind < 3; ++kind) {
    int threads = 256, blocks = sms * 8, iters = 4000;
    auto launch = [&]() {
      if (kind == 0) probe<0><<<blocks, threads>>>(out, iters);
      if (kind == 1) probe<1><<<blocks, threads>>>(out, iters);
      if (kind == 2) probe<2><<<blocks, threads>>>(out, iters);
    };
    launch(); cudaDeviceSynchronize();
    cudaEventRecord(e0); launch(); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double warps = (double)blocks * threads / 32;
    double total = warps * iters * 4 * macs[kind];
    printf("%-26s ms=%.3f TMAC/s=%.1f (T%s/s=%.1f)\n", names[kind], ms, total / ms / 1e9, kind == 0 ? "OP" : "FLOP", 2 * total / ms / 1e9);
  }
  printf("err=%s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
