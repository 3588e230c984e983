// learn_kernel.cu -- training kernels of the learned weighted min-sum.
//
// There is no counterpart in the paper: the fixed normalisation alpha of
// Eq. (1) becomes a weight w[t][e] per edge and iteration, trained by
// gradient descent on window samples.
//
// Forward (one sample = one window syndrome), T unrolled flooding iterations
// on the full window with explicit per-edge messages, t = 1..T:
//   c2v[e]  = (-1)^{s_j} * w[t][e] * min_{e' != e} |v2c[e']| * prod_{e' != e} sign(v2c[e'])
//   post[i] = Lambda_i + sum_{e in M(i)} c2v[e]          (ascending check order)
//   v2c[e]  = clip(post[i] - c2v[e], +-clip)
// starting from v2c = Lambda.  Loss: soft-syndrome BCE at t = T,
//   P(check j odd) = (1 - prod_{i in N(j)} tanh(post_i / 2)) / 2,
//   loss = mean_j BCE(P_j, s_j),
// since 1 - 2 sigma(-x) = tanh(x / 2).
// Backward: the adjoint of the unrolled iterations, recomputed segment by
// segment from checkpoints of v2c every `ckpt` iterations.  A min-sum check
// sends each edge the magnitude of one other edge (the smallest, or the second
// smallest for the edge holding the smallest), so its gradient flows to at
// most two inputs; derivatives of sign() and of a saturated clip are zero.
// FP32 throughout; tanhf / logf are CUDA's.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>

#include "gdg_kernel.cuh"

namespace qd {

namespace lrn {

__device__ __forceinline__ float clipf(float x, float c) { return x > c ? c : (x < -c ? -c : x); }

struct CheckMins {
  float m1, m2;
  int e1, e2;
  uint32_t neg;
};

// two smallest |v| over the check's edges and their edge ids, sign parity
__device__ __forceinline__ CheckMins check_mins(const WmsGraph& G, const float* v, int j) {
  CheckMins c{CUDART_INF_F, CUDART_INF_F, -1, -1, 0u};
  for (int q = G.row_ptr[j]; q < G.row_ptr[j + 1]; ++q) {
    const int e = (int)(G.row_ent[q] & 0xFFFFu);
    const float x = v[e];
    const float a = fabsf(x);
    if (a < c.m1) {
      c.m2 = c.m1;
      c.e2 = c.e1;
      c.m1 = a;
      c.e1 = e;
    } else if (a < c.m2) {
      c.m2 = a;
      c.e2 = e;
    }
    c.neg ^= (x < 0.0f);
  }
  return c;
}

struct Smem {
  float *v2c, *c2v, *gv, *post, *gpost, *tmp;
  uint32_t* sb;
};

// one flooding iteration t (1-based) of weighted min-sum; v2c -> c2v, post, v2c
__device__ void wms_iteration(const WmsGraph& G, const float* w, const Smem& S, int t) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const float* wt = w + (size_t)(t - 1) * G.ne;
  for (int j = tid; j < G.nr; j += NT) {
    const CheckMins c = check_mins(G, S.v2c, j);
    const uint32_t sj = (S.sb[j >> 5] >> (j & 31)) & 1u;
    for (int q = G.row_ptr[j]; q < G.row_ptr[j + 1]; ++q) {
      const int e = (int)(G.row_ent[q] & 0xFFFFu);
      const float m = (e == c.e1) ? c.m2 : c.m1;
      const uint32_t sg = c.neg ^ (S.v2c[e] < 0.0f) ^ sj;
      const float mag = __fmul_rn(wt[e], m);
      S.c2v[e] = sg ? -mag : mag;
    }
  }
  __syncthreads();
  for (int i = tid; i < G.nc; i += NT) {
    float p = G.llr[i];
    for (int e = G.col_ptr[i]; e < G.col_ptr[i + 1]; ++e) p = __fadd_rn(p, S.c2v[e]);
    S.post[i] = p;
    for (int e = G.col_ptr[i]; e < G.col_ptr[i + 1]; ++e) S.v2c[e] = clipf(__fsub_rn(p, S.c2v[e]), G.clip);
  }
  __syncthreads();
}

// soft-syndrome BCE of the posteriors in S.post; writes dLoss/dpost to S.gpost
// (scaled by 1/nr) and returns the loss (thread 0)
__device__ float soft_syndrome_loss(const WmsGraph& G, const Smem& S, bool want_grad) {
  const int tid = threadIdx.x, NT = blockDim.x;
  __shared__ float red[32];
  float lsum = 0.0f;
  // per check: product of tanh(post/2) over its variables; per-edge exclusive products in tmp
  for (int j = tid; j < G.nr; j += NT) {
    const int qb = G.row_ptr[j], qe = G.row_ptr[j + 1];
    float prod = 1.0f;
    for (int q = qb; q < qe; ++q) {
      const int i = (int)(G.row_ent[q] >> 16);
      const int e = (int)(G.row_ent[q] & 0xFFFFu);
      S.tmp[e] = prod;  // prefix product (exclusive)
      prod *= tanhf(0.5f * S.post[i]);
    }
    const uint32_t sj = (S.sb[j >> 5] >> (j & 31)) & 1u;
    float P = 0.5f * (1.0f - prod);
    const float eps = 1e-7f;
    const bool clamped = P < eps || P > 1.0f - eps;
    P = fminf(fmaxf(P, eps), 1.0f - eps);
    lsum += sj ? -logf(P) : -logf(1.0f - P);
    if (want_grad) {
      // dL/dprod = dL/dP * dP/dprod, with dP/dprod = -1/2
      const float dP = clamped ? 0.0f : (sj ? -1.0f / P : 1.0f / (1.0f - P)) / (float)G.nr;
      const float dprod = -0.5f * dP;
      float suf = 1.0f;
      for (int q = qe - 1; q >= qb; --q) {
        const int i = (int)(G.row_ent[q] >> 16);
        const int e = (int)(G.row_ent[q] & 0xFFFFu);
        const float th = tanhf(0.5f * S.post[i]);
        S.tmp[e] = dprod * S.tmp[e] * suf * 0.5f * (1.0f - th * th);  // contribution to dL/dpost_i
        suf *= th;
      }
    }
  }
  __syncthreads();
  if (want_grad)
    for (int i = tid; i < G.nc; i += NT) {
      float g = 0.0f;
      for (int e = G.col_ptr[i]; e < G.col_ptr[i + 1]; ++e) g += S.tmp[e];
      S.gpost[i] = g;
    }
  // block sum of the loss
  for (int off = 16; off; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if ((tid & 31) == 0) red[tid >> 5] = lsum;
  __syncthreads();
  float tot = 0.0f;
  if (tid == 0)
    for (int x = 0; x < (NT >> 5); ++x) tot += red[x];
  __syncthreads();
  return tot / (float)G.nr;
}

__global__ void __launch_bounds__(256) wms_kernel(WmsGraph G, const float* __restrict__ w,
                                                  const uint32_t* __restrict__ synd, long long n,
                                                  int backward, float grad_scale, float* __restrict__ grad_w,
                                                  float* __restrict__ loss_out, float* __restrict__ post_out,
                                                  float* __restrict__ scratch, size_t scratch_per_cta,
                                                  int* __restrict__ work) {
  extern __shared__ __align__(16) char smem[];
  const int tid = threadIdx.x, NT = blockDim.x;
  Smem S;
  S.v2c = (float*)smem;
  S.c2v = S.v2c + G.ne;
  S.gv = S.c2v + G.ne;
  S.tmp = S.gv + G.ne;
  S.post = S.tmp + G.ne;
  S.gpost = S.post + G.nc;
  S.sb = (uint32_t*)(S.gpost + G.nc);
  __shared__ long long sh_sample;
  float* ck = scratch + (size_t)blockIdx.x * scratch_per_cta;  // checkpoints [nseg][ne]
  const int nseg = (G.T + G.ckpt - 1) / G.ckpt;
  float* segbuf = ck + (size_t)nseg * G.ne;  // inputs of a segment's iterations [ckpt][ne]
  while (true) {
    __syncthreads();
    if (tid == 0) sh_sample = atomicAdd(work, 1);
    __syncthreads();
    const long long s = sh_sample;
    if (s >= n) break;
    for (int x = tid; x < G.rw; x += NT) S.sb[x] = synd[(size_t)s * G.rw + x];
    for (int i = tid; i < G.nc; i += NT)
      for (int e = G.col_ptr[i]; e < G.col_ptr[i + 1]; ++e) S.v2c[e] = G.llr[i];  // t = 0
    __syncthreads();
    // ---- forward with checkpoints ----
    for (int t = 1; t <= G.T; ++t) {
      if (backward && (t - 1) % G.ckpt == 0) {
        float* dst = ck + (size_t)((t - 1) / G.ckpt) * G.ne;
        for (int e = tid; e < G.ne; e += NT) dst[e] = S.v2c[e];
      }
      wms_iteration(G, w, S, t);
    }
    const float L = soft_syndrome_loss(G, S, backward != 0);
    if (tid == 0 && loss_out) loss_out[s] = L;
    if (post_out)
      for (int i = tid; i < G.nc; i += NT) post_out[(size_t)s * G.nc + i] = S.post[i];
    if (!backward) continue;
    // ---- adjoint, segment by segment ----
    for (int e = tid; e < G.ne; e += NT) S.gv[e] = 0.0f;  // v2c^(T) does not enter the loss
    __syncthreads();
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int t0 = seg * G.ckpt, t1 = min(G.T, t0 + G.ckpt);
      // recompute the segment, keeping each iteration's input messages
      for (int e = tid; e < G.ne; e += NT) S.v2c[e] = ck[(size_t)seg * G.ne + e];
      __syncthreads();
      for (int t = t0 + 1; t <= t1; ++t) {
        float* dst = segbuf + (size_t)(t - t0 - 1) * G.ne;
        for (int e = tid; e < G.ne; e += NT) dst[e] = S.v2c[e];
        __syncthreads();
        if (t < t1) wms_iteration(G, w, S, t);
      }
      for (int t = t1; t > t0; --t) {
        const float* vin = segbuf + (size_t)(t - t0 - 1) * G.ne;  // v2c^(t-1)
        const float* wt = w + (size_t)(t - 1) * G.ne;
        // recompute c2v^(t), post^(t) from vin
        for (int e = tid; e < G.ne; e += NT) S.v2c[e] = vin[e];
        __syncthreads();
        for (int j = tid; j < G.nr; j += NT) {
          const CheckMins c = check_mins(G, S.v2c, j);
          const uint32_t sj = (S.sb[j >> 5] >> (j & 31)) & 1u;
          for (int q = G.row_ptr[j]; q < G.row_ptr[j + 1]; ++q) {
            const int e = (int)(G.row_ent[q] & 0xFFFFu);
            const float m = (e == c.e1) ? c.m2 : c.m1;
            const uint32_t sg = c.neg ^ (S.v2c[e] < 0.0f) ^ sj;
            const float mag = __fmul_rn(wt[e], m);
            S.c2v[e] = sg ? -mag : mag;
          }
        }
        __syncthreads();
        // VN adjoint: v2c^(t)[e] = clip(post - c2v[e]), post = Lambda + sum c2v
        for (int i = tid; i < G.nc; i += NT) {
          float p = G.llr[i];
          for (int e = G.col_ptr[i]; e < G.col_ptr[i + 1]; ++e) p = __fadd_rn(p, S.c2v[e]);
          float gp = (t == G.T) ? S.gpost[i] : 0.0f;
          for (int e = G.col_ptr[i]; e < G.col_ptr[i + 1]; ++e) {
            const float x = __fsub_rn(p, S.c2v[e]);
            if (x > -G.clip && x < G.clip) gp += S.gv[e];
          }
          for (int e = G.col_ptr[i]; e < G.col_ptr[i + 1]; ++e) {
            const float x = __fsub_rn(p, S.c2v[e]);
            const float pass = (x > -G.clip && x < G.clip) ? S.gv[e] : 0.0f;
            S.tmp[e] = gp - pass;  // dL/dc2v[e]
          }
        }
        __syncthreads();
        // CN adjoint: weight gradient and routing to the argmin inputs
        for (int j = tid; j < G.nr; j += NT) {
          const CheckMins c = check_mins(G, S.v2c, j);
          const uint32_t sj = (S.sb[j >> 5] >> (j & 31)) & 1u;
          float g1 = 0.0f, g2 = 0.0f;  // into |v2c[e1]| and |v2c[e2]|
          for (int q = G.row_ptr[j]; q < G.row_ptr[j + 1]; ++q) {
            const int e = (int)(G.row_ent[q] & 0xFFFFu);
            const bool own = (e == c.e1);
            const float m = own ? c.m2 : c.m1;
            const uint32_t sg = c.neg ^ (S.v2c[e] < 0.0f) ^ sj;
            const float sgn = sg ? -1.0f : 1.0f;
            const float gc = S.tmp[e];
            atomicAdd(&grad_w[(size_t)(t - 1) * G.ne + e], grad_scale * gc * sgn * m);
            const float gm = gc * sgn * wt[e];
            if (own) g2 += gm;
            else g1 += gm;
          }
          for (int q = G.row_ptr[j]; q < G.row_ptr[j + 1]; ++q) {
            const int e = (int)(G.row_ent[q] & 0xFFFFu);
            float g = 0.0f;
            if (e == c.e1) g = g1 * (S.v2c[e] < 0.0f ? -1.0f : 1.0f);
            else if (e == c.e2) g = g2 * (S.v2c[e] < 0.0f ? -1.0f : 1.0f);
            S.gv[e] = g;  // dL/dv2c^(t-1)[e]
          }
        }
        __syncthreads();
      }
    }
  }
}

// window-local shots: every window column fires with its prior; the syndrome
// is H_win e over the window's rows (Philox counter word 3 = 1 + window)
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Window-local samples: every window column fires with its prior (Philox
// word 3 = domain).  Outputs (each optional): the window syndrome [n][rw];
// the same bits placed at rows row0.. of a whole-shot detector vector
// [n][det_words] (zeros elsewhere); the fired columns [n][cw].
__global__ void wms_sample_kernel(WmsGraph G, const uint32_t* __restrict__ thr, unsigned long long seed,
                                  unsigned long long off, long long n, uint32_t domain,
                                  uint32_t* __restrict__ synd, uint32_t* __restrict__ det, int det_words,
                                  int row0, uint32_t* __restrict__ fault, int cw) {
  extern __shared__ uint32_t srow[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long s = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  uint32_t* row = srow + (size_t)wib * G.rw;
  for (int x = lane; x < G.rw; x += 32) row[x] = 0;
  __syncwarp();
  if (s < n) {
    const unsigned long long shot = off + (unsigned long long)s;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int g = lane; g < (G.nc + 3) / 4; g += 32) {
      const uint4 u = philox(make_uint4((uint32_t)g, (uint32_t)shot, (uint32_t)(shot >> 32), domain), key);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int c = 4 * g + r;
        if (c < G.nc && uu[r] < thr[c]) {
          for (int e = G.col_ptr[c]; e < G.col_ptr[c + 1]; ++e) {
            const int j = G.col_rows[e];
            atomicXor(&row[j >> 5], 1u << (j & 31));
          }
          if (fault) atomicOr(&fault[(size_t)s * cw + (c >> 5)], 1u << (c & 31));
        }
      }
    }
  }
  __syncwarp();
  if (s < n) {
    if (synd)
      for (int x = lane; x < G.rw; x += 32) synd[(size_t)s * G.rw + x] = row[x];
    if (det)
      for (int x = lane; x < det_words; x += 32) {
        // detector bits 32x .. 32x + 31 = window rows 32x - row0 ..
        const int b = 32 * x - row0;
        uint32_t v = 0;
        if (b > -32 && b < G.nr) {
          const int wq = b >= 0 ? (b >> 5) : -1, sh = b & 31;
          const uint32_t lo = (wq >= 0 && wq < G.rw) ? row[wq] : 0u;
          const uint32_t hi = (wq + 1 >= 0 && wq + 1 < G.rw) ? row[wq + 1] : 0u;
          v = sh ? ((lo >> sh) | (hi << (32 - sh))) : lo;
        }
        det[(size_t)s * det_words + x] = v;
      }
  }
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace lrn

size_t wms_smem_bytes(int ne, int nc, int rw) { return sizeof(float) * (4 * (size_t)ne + 2 * (size_t)nc) + 4 * (size_t)rw; }

size_t wms_scratch_per_cta(int ne, int T, int ckpt) {
  const int nseg = (T + ckpt - 1) / ckpt;
  return (size_t)(nseg + ckpt) * ne;  // floats
}

cudaError_t wms_set_smem(size_t bytes) {
  return cudaFuncSetAttribute(lrn::wms_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t wms_occupancy(size_t smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, lrn::wms_kernel, 256, smem);
}

cudaError_t launch_wms(cudaStream_t st, int grid, size_t smem, const WmsGraph& G, const float* w, const uint32_t* synd,
                       long long n, int backward, float grad_scale, float* grad_w, float* loss, float* post,
                       float* scratch, size_t scratch_per_cta, int* work) {
  lrn::wms_kernel<<<grid, 256, smem, st>>>(G, w, synd, n, backward, grad_scale, grad_w, loss, post, scratch,
                                           scratch_per_cta, work);
  return cudaGetLastError();
}

cudaError_t launch_wms_sample(cudaStream_t st, const WmsGraph& G, const uint32_t* thr, unsigned long long seed,
                              unsigned long long off, long long n, unsigned domain, uint32_t* synd, uint32_t* det,
                              int det_words, int row0, uint32_t* fault, int cw) {
  if (n <= 0) return cudaSuccess;
  if (fault) {
    const cudaError_t e = cudaMemsetAsync(fault, 0, sizeof(uint32_t) * (size_t)n * cw, st);
    if (e != cudaSuccess) return e;
  }
  const int wpb = 8;
  lrn::wms_sample_kernel<<<(unsigned)((n + wpb - 1) / wpb), 32 * wpb, sizeof(uint32_t) * wpb * G.rw, st>>>(
      G, thr, seed, off, n, domain, synd, det, det_words, row0, fault, cw);
  return cudaGetLastError();
}

cudaError_t launch_adam(cudaStream_t st, float* w, const float* g, float* m, float* v, long long n, float lr,
                        float b1, float b2, float eps, int step) {
  if (n <= 0) return cudaSuccess;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  lrn::adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace qd
