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
// quantize = 1 (what training and the decoder use) runs on the tensor cores,
// one warp per tile of 16 records:
//   * layer 1: mma.sync m16n8k8 BF16 x BF16 -> FP32 over the 8 features and
//     8 tiles of 8 hidden units, exact (features and grid-rounded weights are
//     BF16 numbers; every partial sum is a multiple of 2^-7 below 2^13);
//     layer 2 in FP32 in the decoder's own fixed order, so the scores equal
//     the decoder's bit for bit;
//   * dL/dW1 = dH^T X: mma.sync m16n8k16 over the 16 records of the tile
//     (units x records times records x features), the operands transposed
//     in registers with movmatrix; dH is split into two BF16 parts
//     (hi = bf16(dh), lo = bf16(dh - hi)), so the products carry ~16
//     significant bits, accumulated in FP32;
//   * dL/db1, dL/dW2, dL/db2 accumulate in FP32 registers.
// quantize = 0 (raw parameters, used to check the rounding's gradient) runs
// one thread per record on the FP32 cores.  Both reduce the 641 gradient
// sums per warp, then per CTA in shared memory, then add them to `grad`
// (FP32 atomics, so the summation order and the last bits vary between
// runs).
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

__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ float bf16_lo_f(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16_hi_f(uint32_t p) { return __uint_as_float(p & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t transpose8x8(uint32_t a) {
  uint32_t d;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}
__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0, float c0, float c1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%9,%10};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0), "f"(c0), "f"(c1), "f"(c0), "f"(c1));
}
__device__ __forceinline__ void mma_k16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                        uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Tensor-core forward / backward on grid-rounded parameters (see the top of
// the file).  Lane l of a warp: g = l / 4 (record g and g + 8 of the tile in
// layer 1), q = l % 4 (features 2q, 2q + 1; hidden units 8t + 2q + c).
__global__ void __launch_bounds__(256) ranker_tc_kernel(const float* __restrict__ params,
                                                        const RankRec* __restrict__ recs,
                                                        const uint8_t* __restrict__ labels, long long n,
                                                        float pos_weight, float scale, float* __restrict__ grad,
                                                        float* __restrict__ loss, float* __restrict__ score) {
  __shared__ float P[kNP];
  __shared__ float G[kNP];
  __shared__ uint32_t Bw1[8 * 32];  // B fragments of W1 for hidden units 8t..8t+7
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = lane >> 2, q = lane & 3;
  for (int i = tid; i < kNP; i += blockDim.x) {
    float v = params[i];
    if (i < 512) v = grid_round(v, 64.0f, 128.0f);
    else if (i < 576) v = grid_round(v, 128.0f, 65536.0f);
    else if (i < 640) v = grid_round(v, 64.0f, 128.0f);
    P[i] = v;
    G[i] = 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < 256; i += blockDim.x) {
    const int t = i >> 5, l = i & 31, u = 8 * t + (l >> 2), k = 2 * (l & 3);
    Bw1[i] = bf16x2_rn(P[u * 8 + k], P[u * 8 + k + 1]);  // exact: the 2^-6 grid within [-2, 2]
  }
  __syncthreads();
  const float* b1 = P + 512;
  const float* W2 = P + 576;
  const float b2 = P[640];
  float gw1[4][4] = {};  // dL/dW1: M-tile m = units 16m.., lane: (unit 16m + g (+8), features 2q, 2q + 1)
  float gb1[16] = {}, gw2[16] = {};  // units 8t + 2q + c at index 2t + c
  float gb2 = 0.0f;
  const long long n_tiles = (n + 15) / 16;
  const long long wid = ((long long)blockIdx.x * blockDim.x + tid) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long tile = wid; tile < n_tiles; tile += nw) {
    const long long r0 = tile * 16 + g, r1 = r0 + 8;
    const bool v0 = r0 < n, v1 = r1 < n;
    float x00 = 0.0f, x01 = 0.0f, x10 = 0.0f, x11 = 0.0f;
    if (v0) {
      const float2 x = *(const float2*)&recs[r0].x[2 * q];
      x00 = x.x;
      x01 = x.y;
    }
    if (v1) {
      const float2 x = *(const float2*)&recs[r1].x[2 * q];
      x10 = x.x;
      x11 = x.y;
    }
    const uint32_t a0 = bf16x2_rn(x00, x01), a1 = bf16x2_rn(x10, x11);  // features are BF16 numbers
    // ---- layer 1 (exact) and layer 2 in the decoder's order ----
    float acc[8][4];
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int u = 8 * t + 2 * q;
      mma_k8(acc[t], a0, a1, Bw1[32 * t + lane], b1[u], b1[u + 1]);
      s0 = __fadd_rn(s0, __fmul_rn(W2[u], fmaxf(acc[t][0], 0.0f)));
      s0 = __fadd_rn(s0, __fmul_rn(W2[u + 1], fmaxf(acc[t][1], 0.0f)));
      s1 = __fadd_rn(s1, __fmul_rn(W2[u], fmaxf(acc[t][2], 0.0f)));
      s1 = __fadd_rn(s1, __fmul_rn(W2[u + 1], fmaxf(acc[t][3], 0.0f)));
    }
    float z[2];
    {
      const int qb = lane & ~3;
      float p0[4], p1[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        p0[i] = __shfl_sync(FULL, s0, qb + i);
        p1[i] = __shfl_sync(FULL, s1, qb + i);
      }
      z[0] = __fadd_rn(__fadd_rn(__fadd_rn(p0[0], p0[1]), __fadd_rn(p0[2], p0[3])), b2);
      z[1] = __fadd_rn(__fadd_rn(__fadd_rn(p1[0], p1[1]), __fadd_rn(p1[2], p1[3])), b2);
    }
    if (score && q == 0) {
      if (v0) score[r0] = z[0];
      if (v1) score[r1] = z[1];
    }
    if (!grad && !loss) continue;
    // ---- loss and dL/dz (records r0, r1; every lane of the quad) ----
    float dz[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool act = h ? v1 : v0;
      const long long r = h ? r1 : r0;
      const float y = act ? (float)labels[r] : 0.0f;
      const float wy = y > 0.5f ? pos_weight : 1.0f;
      const float zz = z[h];
      if (act && loss && q == 0) loss[r] = wy * (fmaxf(zz, 0.0f) + log1pf(expf(-fabsf(zz))) - y * zz);
      const float sg = zz >= 0.0f ? 1.0f / (1.0f + expf(-zz)) : expf(zz) / (1.0f + expf(zz));
      dz[h] = act ? wy * (sg - y) * scale : 0.0f;
    }
    if (!grad) continue;
    if (q == 0) gb2 += dz[0] + dz[1];
    // ---- dH, dL/db1, dL/dW2; dH^T in BF16 hi / lo parts, transposed ----
    uint32_t ah[8][2], al[8][2];  // [t][half]: (unit 8t + g, records 8 half + 2q, + 1) after the transpose
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int u = 8 * t + 2 * q;
      float dh[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float a = acc[t][e];
        dh[e] = a > 0.0f ? dz[e >> 1] * W2[u + (e & 1)] : 0.0f;
        gw2[2 * t + (e & 1)] += dz[e >> 1] * fmaxf(a, 0.0f);
      }
      gb1[2 * t] += dh[0] + dh[2];
      gb1[2 * t + 1] += dh[1] + dh[3];
      const uint32_t h0 = bf16x2_rn(dh[0], dh[1]), h1 = bf16x2_rn(dh[2], dh[3]);
      const uint32_t l0 = bf16x2_rn(dh[0] - bf16_lo_f(h0), dh[1] - bf16_hi_f(h0));
      const uint32_t l1 = bf16x2_rn(dh[2] - bf16_lo_f(h1), dh[3] - bf16_hi_f(h1));
      ah[t][0] = transpose8x8(h0);
      ah[t][1] = transpose8x8(h1);
      al[t][0] = transpose8x8(l0);
      al[t][1] = transpose8x8(l1);
    }
    // X of the tile as B (records x features): (records 2q, 2q + 1 | +8, feature g)
    const uint32_t xb0 = transpose8x8(a0), xb1 = transpose8x8(a1);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      mma_k16(gw1[m], ah[2 * m][0], ah[2 * m + 1][0], ah[2 * m][1], ah[2 * m + 1][1], xb0, xb1);
      mma_k16(gw1[m], al[2 * m][0], al[2 * m + 1][0], al[2 * m][1], al[2 * m + 1][1], xb0, xb1);
    }
  }
  if (!grad) return;
  // ---- reduce over the warp, then the CTA, then add to grad ----
#pragma unroll
  for (int i = 0; i < 16; ++i) {  // lanes with the same q hold the same units
    float a = gb1[i], b = gw2[i];
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
      a += __shfl_xor_sync(FULL, a, off);
      b += __shfl_xor_sync(FULL, b, off);
    }
    if (g == 0) {
      const int u = 8 * (i >> 1) + 2 * q + (i & 1);
      atomicAdd(&G[512 + u], a);
      atomicAdd(&G[576 + u], b);
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    atomicAdd(&G[(16 * m + g) * 8 + 2 * q], gw1[m][0]);
    atomicAdd(&G[(16 * m + g) * 8 + 2 * q + 1], gw1[m][1]);
    atomicAdd(&G[(16 * m + g + 8) * 8 + 2 * q], gw1[m][2]);
    atomicAdd(&G[(16 * m + g + 8) * 8 + 2 * q + 1], gw1[m][3]);
  }
  gb2 = warp_sum(gb2);
  if (lane == 0) atomicAdd(&G[640], gb2);
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
  if (quantize) {  // tensor cores: 16 records per warp
    const long long want = (n + 127) / 128;
    const int grid = (int)(want < 4LL * sms ? want : 4LL * sms);
    rk::ranker_tc_kernel<<<grid, 256, 0, st>>>(params, recs, labels, n, pos_weight, scale, grad, loss, score);
    return cudaGetLastError();
  }
  const long long want = (n + 255) / 256;
  const int grid = (int)(want < 4LL * sms ? want : 4LL * sms);
  rk::ranker_kernel<<<grid, 256, 0, st>>>(params, recs, labels, n, quantize, pos_weight, scale, grad, loss, score);
  return cudaGetLastError();
}

}  // namespace qd
