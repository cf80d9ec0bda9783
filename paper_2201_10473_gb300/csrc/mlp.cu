// mlp.cu -- the plan cost model's network: y = w2 . relu(W1 x + b1) + b2 in
// fp32, trained with mean squared error and Adam by the kernels below.
//
// Parameter vector (fp32, device): W1 [H x D] row-major, b1 [H], w2 [H], b2 [1].
// One warp per sample: lane l owns hidden units l, l+32, ... (H <= 128).
#include <cuda_runtime.h>

#include "gf2x_gb300.h"

namespace {

constexpr int kMaxHidden = 128;
constexpr int kMaxIn = 64;
constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void mlp_forward_kernel(const float *__restrict__ P, const float *__restrict__ X, float *__restrict__ Y,
                                   int B, int D, int H)
{
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (s >= B)
        return;
    const float *W1 = P, *b1 = P + H * D, *w2 = b1 + H, *b2 = w2 + H;
    const float *x = X + (size_t)s * D;
    float acc = 0.f;
    for (int h = lane; h < H; h += 32) {
        float z = b1[h];
        for (int i = 0; i < D; ++i)
            z = fmaf(W1[h * D + i], x[i], z);
        acc = fmaf(w2[h], fmaxf(z, 0.f), acc);
    }
    acc = warp_sum(acc);
    if (lane == 0)
        Y[s] = acc + b2[0];
}

// Gradient of L = (1/B) sum_s (y_s - t_s)^2 accumulated into G (zeroed by the
// caller's stream first), and L into *loss.
__global__ void mlp_grad_kernel(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ T,
                                float *__restrict__ G, float *__restrict__ loss, int B, int D, int H)
{
    __shared__ float sG[kMaxHidden * kMaxIn + 2 * kMaxHidden + 1];
    const int nparam = H * D + 2 * H + 1;
    for (int i = threadIdx.x; i < nparam; i += blockDim.x)
        sG[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const float *W1 = P, *b1 = P + H * D, *w2 = b1 + H;
    float *gW1 = sG, *gb1 = sG + H * D, *gw2 = gb1 + H, *gb2 = gw2 + H;
    if (s < B) {
        const float *x = X + (size_t)s * D;
        float z[kMaxHidden / 32];
        float acc = 0.f;
        for (int u = 0, h = lane; h < H; h += 32, ++u) {
            float v = b1[h];
            for (int i = 0; i < D; ++i)
                v = fmaf(W1[h * D + i], x[i], v);
            z[u] = v;
            acc = fmaf(w2[h], fmaxf(v, 0.f), acc);
        }
        const float y = warp_sum(acc) + P[H * D + 2 * H];
        const float r = y - T[s];
        const float dy = 2.f * r / (float)B;
        if (lane == 0) {
            atomicAdd(gb2, dy);
            atomicAdd(loss, r * r / (float)B);
        }
        for (int u = 0, h = lane; h < H; h += 32, ++u) {
            const float a = fmaxf(z[u], 0.f);
            atomicAdd(gw2 + h, dy * a);
            const float dz = z[u] > 0.f ? dy * w2[h] : 0.f;
            atomicAdd(gb1 + h, dz);
            for (int i = 0; i < D; ++i)
                atomicAdd(gW1 + h * D + i, dz * x[i]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nparam; i += blockDim.x)
        if (sG[i] != 0.f)
            atomicAdd(G + i, sG[i]);
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr * mhat / (sqrt(vhat) + eps) with bias corrections for step t >= 1.
__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, int n, float lr, float beta1, float beta2, float eps, float c1,
                            float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float g = G[i];
    const float m = beta1 * M[i] + (1.f - beta1) * g;
    const float v = beta2 * V[i] + (1.f - beta2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

bool dims_ok(int B, int D, int H) { return B >= 0 && D >= 1 && D <= kMaxIn && H >= 1 && H <= kMaxHidden; }

}  // namespace

extern "C" size_t gf2x_mlp_param_count(int in_dim, int hidden)
{
    return (size_t)hidden * in_dim + 2 * (size_t)hidden + 1;
}

extern "C" gf2x_status gf2x_mlp_forward(const float *params, const float *x, float *y, int batch, int in_dim,
                                        int hidden, gf2x_stream stream)
{
    if (!params || !x || !y || !dims_ok(batch, in_dim, hidden))
        return GF2X_EINVAL;
    if (batch == 0)
        return GF2X_OK;
    const int blocks = (batch + kWarpsPerBlock - 1) / kWarpsPerBlock;
    mlp_forward_kernel<<<blocks, 32 * kWarpsPerBlock, 0, (cudaStream_t)stream>>>(params, x, y, batch, in_dim, hidden);
    return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}

extern "C" gf2x_status gf2x_mlp_grad(const float *params, const float *x, const float *target, float *grad,
                                     float *loss, int batch, int in_dim, int hidden, gf2x_stream stream)
{
    if (!params || !x || !target || !grad || !loss || !dims_ok(batch, in_dim, hidden))
        return GF2X_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = gf2x_mlp_param_count(in_dim, hidden);
    if (cudaMemsetAsync(grad, 0, np * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess)
        return GF2X_ECUDA;
    if (batch == 0)
        return GF2X_OK;
    const int blocks = (batch + kWarpsPerBlock - 1) / kWarpsPerBlock;
    mlp_grad_kernel<<<blocks, 32 * kWarpsPerBlock, 0, s>>>(params, x, target, grad, loss, batch, in_dim, hidden);
    return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}

extern "C" gf2x_status gf2x_mlp_adam(float *params, const float *grad, float *m, float *v, size_t nparams, float lr,
                                     float beta1, float beta2, float eps, int step, gf2x_stream stream)
{
    if (!params || !grad || !m || !v || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
        return GF2X_EINVAL;
    if (nparams == 0)
        return GF2X_OK;
    const float c1 = 1.f - powf(beta1, (float)step);
    const float c2 = 1.f - powf(beta2, (float)step);
    const int threads = 256;
    const int blocks = (int)((nparams + threads - 1) / threads);
    adam_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(params, grad, m, v, (int)nparams, lr, beta1, beta2, eps,
                                                              c1, c2);
    return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}
