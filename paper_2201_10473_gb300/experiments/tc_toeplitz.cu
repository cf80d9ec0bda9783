// Tensor-core Toeplitz experiment: 512 x 512-bit carry-less products through fp8 (e4m3) mma.sync on
// bit-unpacked Toeplitz tiles (counts in fp32, parity = the bit), one warp per
// product, against the library's comb leaf (2-way Karatsuba over 256-bit
// combs, one thread per product).  Bit-exact check, then timing.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>
#include "../csrc/fused.cuh"

constexpr int S = 16;            // 32-bit words per operand
constexpr int SB = 32 * S;       // bits
constexpr int WARPS = 8;
constexpr int AR_PAD = 2, AR_W = S + 4;     // ar words [-2, S+2)
constexpr int B_PAD = 8, B_W = S + 16;      // b words [-8, S+8)

__device__ __forceinline__ uint32_t expand4(uint32_t x) { return ((x * 0x00204081u) & 0x01010101u) * 0x38u; }
__device__ __forceinline__ uint32_t extract8(uint32_t x, uint32_t t) {
  uint32_t y = (x >> t) & 0x11111111u;
  y = (y | (y >> 3)) & 0x03030303u;
  y = (y | (y >> 6)) & 0x000F000Fu;
  y = (y | (y >> 12)) & 0xFFu;
  return y;
}
__device__ __forceinline__ uint32_t parity_bit(float v) { return __float_as_uint(v + 8388608.0f) & 1u; }

__global__ void __launch_bounds__(32 * WARPS) tc_mul(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B,
                                                     uint32_t* __restrict__ C, int count) {
  __shared__ uint32_t s_ar[WARPS][AR_W];
  __shared__ uint32_t s_b[WARPS][B_W];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int p = blockIdx.x * WARPS + warp; p < count; p += gridDim.x * WARPS) {
    const uint32_t* a = A + (size_t)p * S;
    const uint32_t* b = B + (size_t)p * S;
    // stage: ar[i] = bit-reverse of a[S-1-i]; zero padding around both
    for (int i = lane; i < AR_W; i += 32) {
      const int w = i - AR_PAD;
      s_ar[warp][i] = (w >= 0 && w < S) ? __brev(a[S - 1 - w]) : 0u;
    }
    for (int i = lane; i < B_W; i += 32) {
      const int w = i - B_PAD;
      s_b[warp][i] = (w >= 0 && w < S) ? b[w] : 0u;
    }
    __syncwarp();
    // B fragments for every column start J0 in [-7, S-1]
    uint32_t bf0[S + 7], bf1[S + 7];
#pragma unroll
    for (int j = 0; j < S + 7; ++j) {
      const uint32_t bw = s_b[warp][j - 7 + g + B_PAD];
      bf0[j] = expand4((bw >> (4 * t)) & 15u);
      bf1[j] = expand4((bw >> (16 + 4 * t)) & 15u);
    }
    float acc[8][4];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[q][r] = 0.f;
#pragma unroll
    for (int e = 0; e <= 2 * S + 1; ++e) {
      const int par = e & 1;
      // A fragment: Toeplitz tile T_e, rows 16e + r - k of a, from reversed a
      const int Q = SB - 1 - 16 * e - g + 4 * t;
      const int base = Q - 8 + 64;
      const int w = (base >> 5) - 2;
      const uint32_t off = base & 31;
      const uint32_t lo = s_ar[warp][w + AR_PAD], hi = s_ar[warp][w + 1 + AR_PAD];
      const uint32_t W = __funnelshift_r(lo, hi, off);
      const uint32_t a1 = expand4(W & 15u), a0 = expand4((W >> 8) & 15u);
      const uint32_t a3 = expand4((W >> 16) & 15u), a2 = expand4((W >> 24) & 15u);
#pragma unroll
      for (int m = 0; m < S / 4; ++m) {
        const int K0 = 16 * m + par;
        if (e < K0 - 2 * S + 2 || e > K0 + 14) continue;    // compile-time after unrolling
        const int J0 = (K0 - e) / 2;
        const int gi = m + 4 * par;
        asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                     : "+f"(acc[gi][0]), "+f"(acc[gi][1]), "+f"(acc[gi][2]), "+f"(acc[gi][3])
                     : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(bf0[J0 + 7]), "r"(bf1[J0 + 7]));
      }
    }
    // parity of the counts, gathered with ballots into output words
    uint32_t* c = C + (size_t)p * 2 * S;
#pragma unroll
    for (int m = 0; m < S / 4; ++m) {
      uint32_t be[4], bo[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        be[r] = __ballot_sync(0xffffffffu, parity_bit(acc[m][r]));
        bo[r] = __ballot_sync(0xffffffffu, parity_bit(acc[m + 4][r]));
      }
      if (lane < 8) {
        const uint32_t tc = lane >> 1, odd = lane & 1;
        const uint32_t e_lo = odd ? be[1] : be[0], e_hi = odd ? be[3] : be[2];
        const uint32_t o_lo = odd ? bo[1] : bo[0], o_hi = odd ? bo[3] : bo[2];
        const uint32_t low16 = extract8(e_lo, tc) | (extract8(e_hi, tc) << 8);
        const uint32_t high16 = extract8(o_lo, tc) | (extract8(o_hi, tc) << 8);
        c[8 * m + lane] = low16 | (high16 << 16);
      }
    }
    __syncwarp();
  }
}

// the library's comb: one thread per product, 2-way Karatsuba over 256-bit combs
__global__ void __launch_bounds__(256) comb_mul(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B,
                                                uint32_t* __restrict__ C, int count) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < count; p += gridDim.x * blockDim.x) {
    uint32_t slot[4 * (S / 2)];
    for (int i = 0; i < S; ++i) { slot[i] = A[(size_t)p * S + i]; slot[S + i] = B[(size_t)p * S + i]; }
    gf2x::leaf_k2<S / 2>(slot);
    for (int i = 0; i < 2 * S; ++i) C[(size_t)p * 2 * S + i] = slot[i];
  }
}

static void clmul_ref(const uint32_t* a, const uint32_t* b, uint32_t* c) {
  for (int i = 0; i < 2 * S; ++i) c[i] = 0;
  for (int i = 0; i < SB; ++i)
    if ((b[i >> 5] >> (i & 31)) & 1)
      for (int j = 0; j < SB; ++j)
        if ((a[j >> 5] >> (j & 31)) & 1) c[(i + j) >> 5] ^= 1u << ((i + j) & 31);
}

#ifdef GF2X_EXPERIMENT_LIB
// Test entry points (built into libgf2x_exp_tc.so by build.py): `count`
// full 512 x 512-bit products, operands of 16 words per row, results of 32
// words per row, device pointers, asynchronous on `stream`.  0 on success.
extern "C" int gf2x_exp_tc_mul512(const uint32_t* A, const uint32_t* B, uint32_t* C, int count, void* stream) {
  if (count <= 0) return 0;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
  tc_mul<<<sms * 8, 32 * WARPS, 0, (cudaStream_t)stream>>>(A, B, C, count);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
extern "C" int gf2x_exp_comb_mul512(const uint32_t* A, const uint32_t* B, uint32_t* C, int count, void* stream) {
  if (count <= 0) return 0;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
  comb_mul<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(A, B, C, count);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
#else
int main() {
  const int count = 1 << 20;
  std::vector<uint32_t> ha((size_t)count * S), hb((size_t)count * S);
  uint64_t x = 0x9E3779B97F4A7C15ull;
  for (auto& v : ha) { x ^= x << 13; x ^= x >> 7; x ^= x << 17; v = (uint32_t)x; }
  for (auto& v : hb) { x ^= x << 13; x ^= x >> 7; x ^= x << 17; v = (uint32_t)x; }
  for (int i = 0; i < S; ++i) { ha[i] = 0xFFFFFFFFu; hb[i] = 0xFFFFFFFFu; }      // product 0: all ones
  uint32_t *dA, *dB, *dC1, *dC2;
  cudaMalloc(&dA, ha.size() * 4); cudaMalloc(&dB, hb.size() * 4);
  cudaMalloc(&dC1, (size_t)count * 2 * S * 4); cudaMalloc(&dC2, (size_t)count * 2 * S * 4);
  cudaMemcpy(dA, ha.data(), ha.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, hb.data(), hb.size() * 4, cudaMemcpyHostToDevice);
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int tc_blocks = sms * 8, comb_blocks = sms * 8;
  tc_mul<<<tc_blocks, 32 * WARPS>>>(dA, dB, dC1, count);
  comb_mul<<<comb_blocks, 256>>>(dA, dB, dC2, count);
  cudaError_t err = cudaDeviceSynchronize();
  printf("launch: %s\n", cudaGetErrorString(err));
  if (err != cudaSuccess) return 1;
  std::vector<uint32_t> c1((size_t)count * 2 * S), c2((size_t)count * 2 * S);
  cudaMemcpy(c1.data(), dC1, c1.size() * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(c2.data(), dC2, c2.size() * 4, cudaMemcpyDeviceToHost);
  size_t mism = 0;
  for (size_t i = 0; i < c1.size(); ++i) mism += c1[i] != c2[i];
  int refbad = 0;
  for (int p = 0; p < 16; ++p) {
    uint32_t r[2 * S]; clmul_ref(&ha[(size_t)p * S], &hb[(size_t)p * S], r);
    for (int i = 0; i < 2 * S; ++i) refbad += r[i] != c1[(size_t)p * 2 * S + i];
  }
  printf("tensor vs comb mismatching words: %zu of %zu; tensor vs CPU reference (16 products): %d bad words\n",
         mism, c1.size(), refbad);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0); for (int k = 0; k < 5; ++k) tc_mul<<<tc_blocks, 32 * WARPS>>>(dA, dB, dC1, count);
    cudaEventRecord(e1); cudaEventSynchronize(e1); float ms1; cudaEventElapsedTime(&ms1, e0, e1);
    cudaEventRecord(e0); for (int k = 0; k < 5; ++k) comb_mul<<<comb_blocks, 256>>>(dA, dB, dC2, count);
    cudaEventRecord(e1); cudaEventSynchronize(e1); float ms2; cudaEventElapsedTime(&ms2, e0, e1);
    printf("512x512-bit products: tensor (mma.sync e4m3) %.3e /s   comb (ALU, K2 over 256-bit) %.3e /s\n",
           5.0 * count / (ms1 * 1e-3), 5.0 * count / (ms2 * 1e-3));
  }
  return 0;
}
#endif
