// FMA pipe probe: IMAD.WIDE (mad.wide.u32), IMAD.HI (mul.hi.u32), and mixes with LOP3.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ uint64_t madw(uint32_t a, uint32_t b, uint64_t c) { uint64_t d; asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c)); return d; }
__device__ __forceinline__ uint64_t mulw(uint32_t a, uint32_t b) { uint64_t d; asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b)); return d; }
__device__ __forceinline__ uint32_t mulhi(uint32_t a, uint32_t b) { uint32_t d; asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b)); return d; }
template <int KIND>
__global__ void probe(uint32_t* out, uint32_t seed, int iters) {
  uint32_t c[16], a[16]; uint64_t w[8];
  for (int i = 0; i < 16; ++i) { a[i] = seed * (i + 1) + threadIdx.x; c[i] = a[i] ^ 0x9e3779b9u; }
  for (int i = 0; i < 8; ++i) w[i] = c[i];
  uint32_t m = seed ^ blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (KIND == 0) {   // 8 IMAD.WIDE accumulate chains
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = madw(a[i], m, w[i]);
      }
      if (KIND == 1) {   // 16 IMAD.HI
#pragma unroll
        for (int i = 0; i < 16; ++i) c[i] = mulhi(c[i], a[i]) ^ 0;
      }
      if (KIND == 2) {   // 8 mul.wide + 8 LOP3 xor-accumulate of the two halves
#pragma unroll
        for (int i = 0; i < 8; ++i) { uint64_t p = mulw(a[i], m); c[2*i] ^= (uint32_t)p ^ c[2*i+1]; c[2*i+1] ^= (uint32_t)(p >> 32); }
      }
      if (KIND == 3) {   // 8 mad.wide (FMA) interleaved with 16 LOP3 (ALU)
#pragma unroll
        for (int i = 0; i < 8; ++i) { w[i] = madw(a[i], m, w[i]); c[2*i] ^= a[2*i] & m; c[2*i+1] ^= a[2*i+1] & m; }
      }
      m = (m << 1) | (m >> 31);
    }
  }
  uint32_t s = 0;
  for (int i = 0; i < 16; ++i) s ^= c[i];
  for (int i = 0; i < 8; ++i) s ^= (uint32_t)w[i] ^ (uint32_t)(w[i] >> 32);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  uint32_t* out; cudaMalloc(&out, 4 << 24);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* names[] = {"IMAD.WIDE acc (8/iter)", "IMAD.HI (16/iter)", "mul.wide+2xLOP3 (8/iter)", "mad.wide+2LOP3 (8/iter)"};
  const int per[] = {8, 16, 8, 8};
  for (int kind = 0; kind < 4; ++kind) {
    int threads = 512, blocks = sms * 4, iters = 2000;
    auto launch = [&]() {
      if (kind == 0) probe<0><<<blocks, threads>>>(out, 7, iters);
      if (kind == 1) probe<1><<<blocks, threads>>>(out, 7, iters);
      if (kind == 2) probe<2><<<blocks, threads>>>(out, 7, iters);
      if (kind == 3) probe<3><<<blocks, threads>>>(out, 7, iters);
    };
    launch(); cudaDeviceSynchronize();
    cudaEventRecord(e0); launch(); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double units = (double)blocks * threads * iters * 8 * per[kind];
    printf("%-28s ms=%.3f units/clk/SM@2070=%.1f\n", names[kind], ms, units / (ms * 1e-3) / sms / 2.07e9);
  }
  printf("err=%s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
