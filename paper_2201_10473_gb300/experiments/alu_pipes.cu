// ALU pipe throughput probe: independent LOP3 (c ^= a & m), funnel shift and IMAD chains, and a LOP3 + IMAD mix.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
template <int KIND>
__global__ void probe(uint32_t* out, uint32_t seed, int iters) {
  uint32_t c[16], a[16];
  for (int i = 0; i < 16; ++i) { a[i] = seed * (i + 1) + threadIdx.x; c[i] = a[i] ^ 0x9e3779b9u; }
  uint32_t m = seed ^ blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (KIND == 0) c[i] ^= a[i] & m;                      // LOP3
        if (KIND == 1) c[i] = __funnelshift_l(c[i], a[i], 1); // SHF
        if (KIND == 2) c[i] = c[i] * a[i] + m;                // IMAD
        if (KIND == 3) { if (i & 1) c[i] ^= a[i] & m; else c[i] = c[i] * a[i] + m; } // mix
      }
      m = (m << 1) | (m >> 31);
    }
  }
  uint32_t s = 0;
  for (int i = 0; i < 16; ++i) s ^= c[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  uint32_t* out; cudaMalloc(&out, 4 << 24);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* names[] = {"LOP3 c^=a&m", "SHF.L funnel", "IMAD", "LOP3+IMAD mix"};
  for (int kind = 0; kind < 4; ++kind) {
    for (int threads : {256, 512, 1024}) {
      int blocks = sms * (2048 / threads);
      int iters = 2000;
      auto launch = [&]() {
        if (kind == 0) probe<0><<<blocks, threads>>>(out, 7, iters);
        if (kind == 1) probe<1><<<blocks, threads>>>(out, 7, iters);
        if (kind == 2) probe<2><<<blocks, threads>>>(out, 7, iters);
        if (kind == 3) probe<3><<<blocks, threads>>>(out, 7, iters);
      };
      launch(); cudaDeviceSynchronize();
      cudaEventRecord(e0); launch(); cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      double ops = (double)blocks * threads * iters * 8 * 16;
      printf("%-16s threads=%4d blocks=%d ms=%.3f Tops/s=%.2f ops/clk/SM@2070=%.1f\n", names[kind], threads, blocks, ms,
             ops / ms / 1e9, ops / (ms * 1e-3) / sms / 2.07e9);
    }
  }
  printf("err=%s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
