// ranker_kernel.cu -- training and scoring of the decimation ranker (the
// learned stand-in for the argmin of Alg. 1) on candidate records.
//
// Model: score = W2 . relu(W1 x + b1) + b2, x = the 8 features of a record,
// W1[64][8], b1[64], W2[64], b2 in one 641-float parameter vector.  With
// `quantize` the forward pass uses the grid-rounded parameters the decoder
// uses (W1, W2 to the 2^-6 grid within [-2, 2], b1 to the 2^-7 grid within [-512, 512]) and the
// gradient passes straight through the rounding to the raw parameters.
// Loss per record: weighted binary cross entropy with logits,
//   l = w_y (softplus(z) - y z),  w_1 = pos_weight, w_0 = 1,
// where y = 1 marks a candidate that is in the sampled fault set.
//
// One thread per record; the 641 gradient sums are reduced per warp with
// shuffles, then per CTA in shared memory, then added to `grad` (FP32
// atomics, so the summation order and the last bits vary between runs).
#include <cuda_runtime.h>

#include <cstdint>

#include "gdg_kernel.cuh"

namespace qd {
namespace rk {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kNP = 641;

__device__ __forceinline__ float grid_round(float x, float scale, float lim) {
  float v = rintf(x * scale);
  v = fminf(fmaxf(v, -lim), lim);
  return v / scale;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
  return v;
}

__global__ void __launch_bounds__(256) ranker_kernel(const float* __restrict__ params, const RankRec* __restrict__ recs,
                                                     const uint8_t* __restrict__ labels, long long n, int quantize,
                                                     float pos_weight, float scale, float* __restrict__ grad,
                                                     float* __restrict__ loss, float* __restrict__ score) {
  __shared__ float P[kNP];
  __shared__ float G[kNP];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < kNP; i += blockDim.x) {
    float v = params[i];
    if (quantize) {
      if (i < 512) v = grid_round(v, 64.0f, 128.0f);
      else if (i < 576) v = grid_round(v, 128.0f, 65536.0f);
      else if (i < 640) v = grid_round(v, 64.0f, 128.0f);
    }
    P[i] = v;
    G[i] = 0.0f;
  }
  __syncthreads();
  const float* W1 = P;
  const float* b1 = P + 512;
  const float* W2 = P + 576;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // every lane of a warp runs the same number of rounds (shuffles below)
  const long long rounds = (n + stride - 1) / stride;
  for (long long r = 0; r < rounds; ++r) {
    const long long i = r * stride + (long long)blockIdx.x * blockDim.x + tid;
    const bool act = i < n;
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = act ? recs[i].x[k] : 0.0f;
    float z = P[640];
    for (int u = 0; u < 64; ++u) {
      float a = b1[u];
#pragma unroll
      for (int k = 0; k < 8; ++k) a += W1[u * 8 + k] * x[k];
      z += W2[u] * fmaxf(a, 0.0f);
    }
    if (act && score) score[i] = z;
    if (!grad && !loss) continue;
    const float y = act ? (float)labels[i] : 0.0f;
    const float wy = y > 0.5f ? pos_weight : 1.0f;
    // softplus(z) - y z, and its derivative sigmoid(z) - y
    const float sp = fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
    if (act && loss) loss[i] = wy * (sp - y * z);
    if (!grad) continue;
    const float sg = z >= 0.0f ? 1.0f / (1.0f + expf(-z)) : expf(z) / (1.0f + expf(z));
    const float dz = act ? wy * (sg - y) * scale : 0.0f;
    for (int u = 0; u < 64; ++u) {
      float a = b1[u];
#pragma unroll
      for (int k = 0; k < 8; ++k) a += W1[u * 8 + k] * x[k];
      const float h = fmaxf(a, 0.0f);
      const float dh = a > 0.0f ? dz * W2[u] : 0.0f;
      const float gw2 = warp_sum(dz * h);
      const float gb1 = warp_sum(dh);
      float gw1[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) gw1[k] = warp_sum(dh * x[k]);
      if (lane == 0) {
        atomicAdd(&G[576 + u], gw2);
        atomicAdd(&G[512 + u], gb1);
#pragma unroll
        for (int k = 0; k < 8; ++k) atomicAdd(&G[u * 8 + k], gw1[k]);
      }
    }
    const float gb2 = warp_sum(dz);
    if (lane == 0) atomicAdd(&G[640], gb2);
  }
  if (!grad) return;
  __syncthreads();
  for (int i = tid; i < kNP; i += blockDim.x)
    if (G[i] != 0.0f) atomicAdd(&grad[i], G[i]);
}

}  // namespace rk

cudaError_t launch_ranker(cudaStream_t st, const float* params, const RankRec* recs, const uint8_t* labels,
                          long long n, int quantize, float pos_weight, float scale, float* grad, float* loss,
                          float* score) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long want = (n + 255) / 256;
  const int grid = (int)(want < 4LL * sms ? want : 4LL * sms);
  rk::ranker_kernel<<<grid, 256, 0, st>>>(params, recs, labels, n, quantize, pos_weight, scale, grad, loss, score);
  return cudaGetLastError();
}

}  // namespace qd
