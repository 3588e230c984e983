// gdg_kernel.cu -- the window decoder, sampler, commit and evaluation kernels.
//
// decode (one persistent launch per window step; CTA = one shot at a time):
//   a1  window syndrome: bits [row0, row0 + n_rows) of the shot's detectors
//   a2  pre-BP: n_pre flooding min-sum iterations on the full window
//       (Eq. (1)-(4)), whole CTA; check node j by one warp, variable node i
//       by one thread; early stop when H e = s (Sec. II-A)
//   a3  ranking key ((h0+h1)+h2)+h3 of the last four posteriors, bitonic sort
//       of (key, column) ascending, first 2w' columns kept (Sec. III); the
//       shortened matrix is rebuilt in shared memory
//   a4-a7 GDG: warp w runs decision paths w, w+NW, ... (Alg. 2 on the 2^k
//       tree): BP steps of iters_per_step iterations, SELECT-VN (Alg. 1) with
//       aggressive decimation (Alg. 3), guess value by the path id, peeling
//   a8  minimum path metric Eq. (5) over converged paths, ties to the lowest id
// Every wait is a __syncthreads/__syncwarp of this CTA; nothing spins.
#include <cuda_runtime.h>

#include <math_constants.h>

#include <cfloat>
#include <cstdint>

#include "gdg_kernel.cuh"

namespace qd {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;
enum { BR_CONVERGED = 0, BR_MAXDEPTH = 1, BR_CONTRADICTION = 2, BR_NOCAND = 3, BR_INTERNAL = 4 };

__device__ __forceinline__ float clipf(float x, float c) { return x > c ? c : (x < -c ? -c : x); }

// mu_{j->i} from the check's compressed state (see gdg_kernel.cuh).
__device__ __forceinline__ float c2v_msg(float alpha, float clip, float m1, float m2, uint16_t am,
                                         uint8_t cfl, int e, uint8_t sg) {
  float m = ((uint16_t)e == am) ? m2 : m1;
  if (cfl & 2) m = clip;  // single active VN: minimum over the empty set = clip
  float mag = __fmul_rn(alpha, m);
  return (((cfl & 1u) ^ sg) != 0) ? -mag : mag;
}

__device__ __forceinline__ uint32_t bit_of(const uint32_t* w, int j) { return (w[j >> 5] >> (j & 31)) & 1u; }

// order-preserving map of a float to uint32 (-0 and +0 equal)
__device__ __forceinline__ uint32_t ordkey(float f) {
  if (f == 0.0f) f = 0.0f;
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ void warp_min2(float& m1, float& m2, int& am) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    float x1 = __shfl_xor_sync(FULL, m1, off);
    float x2 = __shfl_xor_sync(FULL, m2, off);
    int xa = __shfl_xor_sync(FULL, am, off);
    if (x1 < m1 || (x1 == m1 && xa < am)) {
      m2 = fminf(m1, x2);
      m1 = x1;
      am = xa;
    } else {
      m2 = fminf(m2, x1);
    }
  }
}

// lexicographic (value, index) minimum over the warp
__device__ __forceinline__ void warp_argmin(float& v, int& k) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    float xv = __shfl_xor_sync(FULL, v, off);
    int xk = __shfl_xor_sync(FULL, k, off);
    if (xv < v || (xv == v && xk < k)) {
      v = xv;
      k = xk;
    }
  }
}

// Exclusive scan of a[0..n) in place, by one warp; returns the total.
__device__ int warp_scan_excl(int* a, int n, int lane) {
  int chunk = (n + 31) / 32;
  int beg = lane * chunk, end = min(n, beg + chunk);
  int s = 0;
  for (int i = beg; i < end; ++i) s += a[i];
  int incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int y = __shfl_up_sync(FULL, incl, off);
    if (lane >= off) incl += y;
  }
  int run = incl - s;
  for (int i = beg; i < end; ++i) {
    int v = a[i];
    a[i] = run;
    run += v;
  }
  return __shfl_sync(FULL, incl, 31);
}

struct ShortG {
  int nr, ns, rw;
  const uint16_t *colptr, *colrows, *rowptr, *rowedges, *edgecol;
  const float* llr;
  const uint8_t* vdeg;
  const uint32_t* sbits;
};

struct BrPtr {
  float *post, *acc;
  uint8_t *hfl, *sign, *cfl;
  int8_t* status;
  float *min1, *min2;
  uint16_t* amin;
  int* deg;
  uint32_t *sp, *par, *unsat;
};

__device__ __forceinline__ void decimate_atomic(const ShortG& G, const BrPtr& B, int k, int v) {
  B.status[k] = (int8_t)v;
  for (int e = G.colptr[k]; e < G.colptr[k + 1]; ++e) {
    int j = G.colrows[e];
    atomicSub(&B.deg[j], 1);
    if (v) atomicXor(&B.sp[j >> 5], 1u << (j & 31));
  }
}

// Peeling (Sec. IV): repeatedly fix the lone active VN of a degree-one check
// to the check's current syndrome; a check left with no active VN and
// syndrome 1 is a contradiction.  One check at a time, always the lowest-index
// degree-one check, after testing every check for a contradiction (this order
// also fixes the partial state of a path killed by a contradiction).
// Returns #peeled or -1 (contradiction), -2 on an inconsistent degree count
// (internal error).
__device__ int peel(const ShortG& G, const BrPtr& B, int lane) {
  int npeel = 0;
  for (int guard = 0; guard <= G.ns + 1; ++guard) {
    bool contra = false;
    int cand = 0x7fffffff;
    for (int j = lane; j < G.nr; j += 32) {
      int d = B.deg[j];
      if (d == 0) {
        if (bit_of(B.sp, j)) contra = true;
      } else if (d == 1 && cand == 0x7fffffff) {
        cand = j;
      }
    }
    if (__any_sync(FULL, contra)) return -1;
    const int j = (int)__reduce_min_sync(FULL, (unsigned)cand);
    if (j == 0x7fffffff) return npeel;
    int found = -1;
    for (int q = G.rowptr[j] + lane; q < G.rowptr[j + 1]; q += 32) {
      int i = G.edgecol[G.rowedges[q]];
      if (B.status[i] == -1) found = i;
    }
    unsigned fm = __ballot_sync(FULL, found >= 0);
    if (!fm) return -2;
    int i = __shfl_sync(FULL, found, __ffs(fm) - 1);
    int v = (int)bit_of(B.sp, j);
    __syncwarp();
    if (lane == 0) {
      B.status[i] = (int8_t)v;
      for (int e = G.colptr[i]; e < G.colptr[i + 1]; ++e) {
        int r = G.colrows[e];
        B.deg[r] -= 1;
        if (v) B.sp[r >> 5] ^= 1u << (r & 31);
      }
    }
    __syncwarp();
    ++npeel;
  }
  return -2;
}

// One decision path of Alg. 2 on the shortened window, run by one warp.
__device__ void run_branch(const KParams& P, const ShortG& G, const BrPtr& B, int id, int lane,
                           int* out_status, double* out_pm, uint32_t* out_ebits, BranchTrace* btr,
                           StepTrace* st, int dmx, int8_t* fstat, long long* edge_visits) {
  const int nr = G.nr, ns = G.ns, rw = G.rw;
  const bool mainb = (id == 0);
  const int dmax = mainb ? P.dmax_main : P.dmax_other;
  const float PA = mainb ? P.pa_main : P.pa_other;
  float PB = mainb ? P.pb_main : P.pb_other;
  for (int k = lane; k < ns; k += 32) B.status[k] = -1;
  for (int j = lane; j < nr; j += 32) B.deg[j] = G.rowptr[j + 1] - G.rowptr[j];
  for (int x = lane; x < rw; x += 32) B.sp[x] = G.sbits[x];
  if (st)
    for (int q = lane; q < dmx; q += 32) st[q] = StepTrace{-2, -1, 0, 0, 0};
  __syncwarp();
  int status = BR_MAXDEPTH, depth = 0, iters = 0;
  long long visits = 0;  // active edges touched by the check-node passes
  double pm = CUDART_INF;
  bool first = true;
  if (P.peel_init) {
    int np = peel(G, B, lane);
    if (np < 0) {
      status = np == -1 ? BR_CONTRADICTION : BR_INTERNAL;
      goto done;
    }
  }
  for (int D = 1; D <= dmax; ++D) {
    depth = D;
    for (int it = 1; it <= P.ips; ++it) {
      uint32_t* par = B.par + (iters & 1) * rw;
      for (int x = lane; x < rw; x += 32) par[x] = 0;
      // ---- check-node update, Eq. (1), over active VNs ----
      for (int j = lane; j < nr; j += 32) {
        const int d = B.deg[j];
        if (d == 0) continue;
        const float om1 = B.min1[j], om2 = B.min2[j];
        const uint16_t oam = B.amin[j];
        const uint8_t ocfl = B.cfl[j];
        float m1 = FLT_MAX * 2.0f, m2 = FLT_MAX * 2.0f;
        int am = 0xFFFF;
        unsigned neg = 0;
        const int qe = G.rowptr[j + 1];
        for (int q = G.rowptr[j]; q < qe; ++q) {
          const int e = G.rowedges[q];
          const int i = G.edgecol[e];
          if (B.status[i] != -1) continue;  // stale message of a decimated VN
          ++visits;
          float v = first ? G.llr[i]
                          : clipf(__fsub_rn(B.post[i], c2v_msg(P.alpha, P.clip, om1, om2, oam, ocfl,
                                                              e, B.sign[e])),
                                  P.clip);
          float a = fabsf(v);
          if (a < m1) {
            m2 = m1;
            m1 = a;
            am = e;
          } else if (a < m2) {
            m2 = a;
          }
          unsigned s = v < 0.0f;
          neg ^= s;
          B.sign[e] = (uint8_t)s;
        }
        B.min1[j] = m1;
        B.min2[j] = m2;
        B.amin[j] = (uint16_t)am;
        B.cfl[j] = (uint8_t)((neg ^ bit_of(B.sp, j)) | ((d == 1) << 1));
      }
      __syncwarp();
      // ---- variable-node update, Eq. (2)-(3); history of Sec. IV-A ----
      const bool hist = it > P.ips - 4;
      const bool hist0 = it == P.ips - 3;
      for (int k = lane; k < ns; k += 32) {
        if (B.status[k] != -1) continue;
        float p = G.llr[k];
        const int ee = G.colptr[k + 1];
        for (int e = G.colptr[k]; e < ee; ++e) {
          const int j = G.colrows[e];
          p = __fadd_rn(p, c2v_msg(P.alpha, P.clip, B.min1[j], B.min2[j], B.amin[j], B.cfl[j], e,
                                   B.sign[e]));
        }
        B.post[k] = p;
        if (hist) {
          uint8_t f = (uint8_t)((p <= 0.0f) | ((p < PA) << 1) | ((p > P.pc) << 2) | ((p > P.pd) << 3));
          if (hist0) {
            B.acc[k] = p;
            B.hfl[k] = f;
          } else {
            B.acc[k] = __fadd_rn(B.acc[k], p);
            B.hfl[k] &= f;
          }
        }
        if (p <= 0.0f)
          for (int e = G.colptr[k]; e < ee; ++e) {
            const int j = G.colrows[e];
            atomicXor(&par[j >> 5], 1u << (j & 31));
          }
      }
      __syncwarp();
      ++iters;
      first = false;
      bool ok = true;
      for (int x = lane; x < rw; x += 32) ok &= (par[x] == B.sp[x]);
      if (__all_sync(FULL, ok)) {
        status = BR_CONVERGED;
        double s = 0.0;
        for (int k = lane; k < ns; k += 32) {
          int st8 = B.status[k];
          bool one = st8 == 1 || (st8 == -1 && B.post[k] <= 0.0f);
          if (one) s += (double)G.llr[k];
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
        pm = s;
        goto done;
      }
    }
    if (D == dmax) break;  // no decimation after the last BP step
    {
      // ---- SELECT-VN (Alg. 1) with AGG-DEC (Alg. 3) ----
      const uint32_t* lastpar = B.par + ((iters - 1) & 1) * rw;
      if (!P.low_err)
        for (int x = lane; x < rw; x += 32) B.unsat[x] = lastpar[x] ^ B.sp[x];
      __syncwarp();
      const float PBd = (D == 1) ? P.pb_d1 : PB;
      float bL = CUDART_INF_F, tL = CUDART_INF_F;
      int bk = 0x7fffffff, tk = 0x7fffffff, nagg = 0;
      for (int k = lane; k < ns; k += 32) {
        if (B.status[k] != -1 || G.vdeg[k] <= 2) continue;
        const float L = B.acc[k];
        const uint8_t fl = B.hfl[k];
        if (!P.low_err) {
          int nus = 0;
          for (int e = G.colptr[k]; e < G.colptr[k + 1]; ++e) nus += bit_of(B.unsat, G.colrows[e]);
          int bdec = -1;
          if ((fl & 2) && L < PBd) bdec = 1;
          else if (((fl & 4) && D <= P.pc_max_depth) || ((fl & 8) && nus >= P.n_unsat_min)) bdec = 0;
          if (bdec >= 0) {
            decimate_atomic(G, B, k, bdec);
            ++nagg;
            continue;
          }
        }
        if (L < bL) {
          bL = L;
          bk = k;
        }
        if ((fl & 1) && L < tL) {
          tL = L;
          tk = k;
        }
      }
      warp_argmin(bL, bk);
      warp_argmin(tL, tk);
#pragma unroll
      for (int off = 16; off; off >>= 1) nagg += __shfl_xor_sync(FULL, nagg, off);
      __syncwarp();
      int g, f;
      if (tk != 0x7fffffff) {
        g = tk;
        f = 1;
      } else if (bk != 0x7fffffff) {
        g = bk;
        f = bL <= 0.0f ? 1 : 0;
      } else {
        if (st && lane == 0) st[D - 1] = StepTrace{-1, -1, 0, (int16_t)nagg, 0};
        status = BR_NOCAND;
        goto done;
      }
      int v = f;
      if (D <= P.k) v = ((id >> (P.k - D)) & 1) ? 1 - f : f;  // b + (-1)^b f
      if (lane == 0) {
        B.status[g] = (int8_t)v;
        for (int e = G.colptr[g]; e < G.colptr[g + 1]; ++e) {
          int r = G.colrows[e];
          B.deg[r] -= 1;
          if (v) B.sp[r >> 5] ^= 1u << (r & 31);
        }
      }
      __syncwarp();
      int np = peel(G, B, lane);
      if (st && lane == 0) st[D - 1] = StepTrace{(int16_t)g, (int8_t)v, 0, (int16_t)nagg, (int16_t)(np < 0 ? -1 : np)};
      if (np < 0) {
        status = np == -1 ? BR_CONTRADICTION : BR_INTERNAL;
        goto done;
      }
    }
  }
done:
  __syncwarp();
  for (int base = 0; base < ns; base += 32) {
    int k = base + lane;
    bool one = false;
    if (k < ns) {
      int s8 = B.status[k];
      one = s8 == 1 || (s8 == -1 && B.post[k] <= 0.0f);
      if (fstat) fstat[k] = (int8_t)s8;
    }
    unsigned m = __ballot_sync(FULL, one);
    if (lane == 0) out_ebits[base >> 5] = m;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) visits += __shfl_xor_sync(FULL, visits, off);
  if (lane == 0) {
    *out_status = status;
    *out_pm = status == BR_CONVERGED ? pm : CUDART_INF;
    if (btr) *btr = BranchTrace{status, depth, iters, 0, status == BR_CONVERGED ? pm : CUDART_INF};
    atomicAdd((unsigned long long*)edge_visits, (unsigned long long)visits);
  }
  __syncwarp();
}

// Trace layout of one shot: int32 head[4]; BranchTrace[nb]; StepTrace[nb][dmx];
// int8 final_status[nb][ns_max]; uint16 short columns[ns_max].
__host__ __device__ inline size_t trace_off_br() { return 16; }
__host__ __device__ inline size_t trace_off_st(int nb) { return 16 + sizeof(BranchTrace) * nb; }
__host__ __device__ inline size_t trace_off_fs(int nb, int dmx) {
  return trace_off_st(nb) + sizeof(StepTrace) * (size_t)nb * dmx;
}
__host__ __device__ inline size_t trace_off_sel(int nb, int dmx, int nsm) {
  return (trace_off_fs(nb, dmx) + (size_t)nb * nsm + 1) & ~(size_t)1;
}
__host__ __device__ inline size_t trace_bytes(int nb, int dmx, int nsm) {
  return (trace_off_sel(nb, dmx, nsm) + 2 * (size_t)nsm + 15) & ~(size_t)15;
}

__global__ void __launch_bounds__(512, 1)
    decode_window_kernel(KParams P, WinDev W, Layout L, const uint32_t* __restrict__ det,
                         int det_words, long long n_shots, uint32_t* __restrict__ corr, int corr_words,
                         int32_t* __restrict__ status_out, char* __restrict__ trace, size_t tr_bytes,
                         int dmx, int ns_max, int* __restrict__ work, long long* __restrict__ counters) {
  extern __shared__ __align__(16) char sm[];
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
  const int nr = W.n_rows, nc = W.n_cols;
  uint32_t* sbits = (uint32_t*)(sm + L.sbits);
  uint32_t* cbits = (uint32_t*)(sm + L.cbits);
  uint16_t* sel = (uint16_t*)(sm + L.sel);
  int* misc = (int*)(sm + L.misc);
  char* U = sm + L.U;
  float* post = (float*)(U + L.p_post);
  float* key = (float*)(U + L.p_key);
  float* min1 = (float*)(U + L.p_min1);
  float* min2 = (float*)(U + L.p_min2);
  uint16_t* amin = (uint16_t*)(U + L.p_amin);
  uint8_t* cfl = (uint8_t*)(U + L.p_cfl);
  uint8_t* sign = (uint8_t*)(U + L.p_sign);
  uint32_t* parb = (uint32_t*)(U + L.p_par);
  unsigned long long* sortb = (unsigned long long*)(U + L.p_sort);

  while (true) {
    __syncthreads();
    if (tid == 0) misc[0] = atomicAdd(work, 1);
    __syncthreads();
    const long long shot = misc[0];
    if (shot >= n_shots) break;
    char* tr = trace ? trace + (size_t)shot * tr_bytes : nullptr;

    // ---- a1: window syndrome ----
    const uint32_t* dp = det + (size_t)shot * det_words;
    for (int x = tid; x < L.rw; x += NT) {
      int b0 = W.row0 + 32 * x;
      uint32_t lo = dp[b0 >> 5];
      uint32_t hi = ((b0 >> 5) + 1 < det_words) ? dp[(b0 >> 5) + 1] : 0u;
      int sh = b0 & 31;
      uint32_t v = sh ? ((lo >> sh) | (hi << (32 - sh))) : lo;
      int rem = nr - 32 * x;
      if (rem < 32) v &= (1u << rem) - 1u;
      sbits[x] = v;
    }
    for (int x = tid; x < L.cw; x += NT) cbits[x] = 0;
    __syncthreads();

    // ---- a2: pre-BP on the full window ----
    bool conv = false;
    int t = 0;
    const int tk0 = P.n_pre - 3 > 1 ? P.n_pre - 3 : 1;
    if (P.n_pre == 0) {
      // decision from the priors alone; key = 4 Lambda
      uint32_t* pb = parb;
      for (int x = tid; x < L.rw; x += NT) pb[x] = 0;
      __syncthreads();
      for (int i = tid; i < nc; i += NT) {
        float li = W.llr[i];
        post[i] = li;
        key[i] = __fadd_rn(__fadd_rn(__fadd_rn(li, li), li), li);
        if (li <= 0.0f)
          for (int e = W.col_ptr[i]; e < W.col_ptr[i + 1]; ++e) {
            int j = W.col_rows[e];
            atomicXor(&pb[j >> 5], 1u << (j & 31));
          }
      }
      __syncthreads();
      bool ok = true;
      for (int x = 0; x < L.rw; ++x) ok &= (pb[x] == sbits[x]);
      conv = ok;
    }
    for (t = 1; t <= P.n_pre; ++t) {
      uint32_t* pb = parb + (t & 1) * L.rw;
      for (int x = tid; x < L.rw; x += NT) pb[x] = 0;
      for (int j = warp; j < nr; j += NW) {
        const int beg = W.row_ptr[j], end = W.row_ptr[j + 1];
        const float om1 = min1[j], om2 = min2[j];
        const uint16_t oam = amin[j];
        const uint8_t ocfl = cfl[j];
        float m1 = FLT_MAX * 2.0f, m2 = FLT_MAX * 2.0f;
        int am = 0xFFFF;
        unsigned neg = 0;
        for (int q = beg + lane; q < end; q += 32) {
          const int e = W.row_edges[q];
          const int i = W.edge_col[e];
          float v = (t == 1) ? W.llr[i]
                             : clipf(__fsub_rn(post[i], c2v_msg(P.alpha, P.clip, om1, om2, oam, ocfl,
                                                               e, sign[e])),
                                     P.clip);
          float a = fabsf(v);
          if (a < m1) {
            m2 = m1;
            m1 = a;
            am = e;
          } else if (a < m2) {
            m2 = a;
          }
          unsigned s = v < 0.0f;
          neg ^= s;
          sign[e] = (uint8_t)s;
        }
        warp_min2(m1, m2, am);
        neg = __reduce_xor_sync(FULL, neg);
        __syncwarp();
        if (lane == 0) {
          min1[j] = m1;
          min2[j] = m2;
          amin[j] = (uint16_t)am;
          cfl[j] = (uint8_t)((neg ^ bit_of(sbits, j)) | ((end - beg == 1) << 1));
        }
      }
      __syncthreads();
      const bool kacc = t >= tk0;
      for (int i = tid; i < nc; i += NT) {
        float p = W.llr[i];
        const int eb = W.col_ptr[i], ee = W.col_ptr[i + 1];
        for (int e = eb; e < ee; ++e) {
          const int j = W.col_rows[e];
          p = __fadd_rn(p, c2v_msg(P.alpha, P.clip, min1[j], min2[j], amin[j], cfl[j], e, sign[e]));
        }
        post[i] = p;
        if (kacc) {
          float kv;
          if (t == tk0) {
            if (P.n_pre < 4) {
              float li = W.llr[i], s = li;
              for (int r = 1; r < 4 - P.n_pre; ++r) s = __fadd_rn(s, li);
              kv = __fadd_rn(s, p);
            } else {
              kv = p;
            }
          } else {
            kv = __fadd_rn(key[i], p);
          }
          key[i] = kv;
        }
        if (p <= 0.0f)
          for (int e = eb; e < ee; ++e) {
            const int j = W.col_rows[e];
            atomicXor(&pb[j >> 5], 1u << (j & 31));
          }
      }
      __syncthreads();
      bool ok = true;
      for (int x = 0; x < L.rw; ++x) ok &= (pb[x] == sbits[x]);
      if (ok) {
        conv = true;
        break;
      }
    }
    const int t_run = conv ? (P.n_pre == 0 ? 0 : t) : P.n_pre;
    if (tid == 0) atomicAdd((unsigned long long*)&counters[0], (unsigned long long)t_run * W.n_edges);

    int winner = -1, n_short = 0;
    if (conv) {
      for (int base = warp * 32; base < nc; base += NT) {
        int i = base + lane;
        bool one = i < nc && post[i] <= 0.0f;
        unsigned m = __ballot_sync(FULL, one);
        if (lane == 0) cbits[base >> 5] = m;
      }
      if (tid == 0) atomicAdd((unsigned long long*)&counters[2], 1ull);
    } else {
      // ---- a3: rank by the four-iteration sum, keep the first n_short ----
      n_short = W.n_short;
      for (int i = tid; i < L.sortn; i += NT)
        sortb[i] = i < nc ? (((unsigned long long)ordkey(key[i]) << 32) | (unsigned)i) : ~0ull;
      __syncthreads();
      for (int kk = 2; kk <= L.sortn; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
          for (int i = tid; i < L.sortn; i += NT) {
            int ixj = i ^ jj;
            if (ixj > i) {
              unsigned long long a = sortb[i], b = sortb[ixj];
              bool up = (i & kk) == 0;
              if ((a > b) == up) {
                sortb[i] = b;
                sortb[ixj] = a;
              }
            }
          }
          __syncthreads();
        }
      for (int k = tid; k < n_short; k += NT) sel[k] = (uint16_t)(sortb[k] & 0xFFFFu);
      __syncthreads();
      // ---- shortened matrix in shared memory ----
      uint16_t* scp = (uint16_t*)(sm + L.s_colptr);
      uint16_t* scr = (uint16_t*)(sm + L.s_colrows);
      uint16_t* srp = (uint16_t*)(sm + L.s_rowptr);
      uint16_t* sre = (uint16_t*)(sm + L.s_rowedges);
      uint16_t* sec = (uint16_t*)(sm + L.s_edgecol);
      float* sllr = (float*)(sm + L.s_llr);
      uint8_t* svd = (uint8_t*)(sm + L.s_vdeg);
      int* rc = (int*)(sm + L.rowcnt);
      int* tmp = (int*)sortb;  // sort buffer is free now
      for (int k = tid; k < n_short; k += NT) {
        int c = sel[k];
        int d = W.col_ptr[c + 1] - W.col_ptr[c];
        tmp[k] = d;
        sllr[k] = W.llr[c];
        svd[k] = (uint8_t)d;
      }
      for (int j = tid; j <= nr; j += NT) rc[j] = 0;
      __syncthreads();
      if (warp == 0) {
        int tot = warp_scan_excl(tmp, n_short, lane);
        if (lane == 0) tmp[n_short] = tot;
      }
      __syncthreads();
      for (int k = tid; k <= n_short; k += NT) scp[k] = (uint16_t)tmp[k];
      for (int k = tid; k < n_short; k += NT) {
        int c = sel[k], o = tmp[k];
        for (int e = W.col_ptr[c]; e < W.col_ptr[c + 1]; ++e, ++o) {
          int r = W.col_rows[e];
          scr[o] = (uint16_t)r;
          sec[o] = (uint16_t)k;
          atomicAdd(&rc[r], 1);
        }
      }
      __syncthreads();
      if (warp == 0) {
        int tot = warp_scan_excl(rc, nr, lane);
        if (lane == 0) rc[nr] = tot;
      }
      __syncthreads();
      for (int j = tid; j <= nr; j += NT) srp[j] = (uint16_t)rc[j];
      __syncthreads();
      const int es = scp[n_short];
      for (int e = tid; e < es; e += NT) {
        int r = scr[e];
        int pos = atomicAdd(&rc[r], 1);
        sre[pos] = (uint16_t)e;
      }
      __syncthreads();
      // ---- a4-a7: GDG, one decision path per warp ----
      ShortG G{nr, n_short, L.rw, scp, scr, srp, sre, sec, sllr, svd, sbits};
      int* res_status = (int*)(sm + L.res_status);
      double* res_pm = (double*)(sm + L.res_pm);
      uint32_t* res_e = (uint32_t*)(sm + L.res_ebits);
      char* slot = U + (size_t)warp * L.b_size;
      BrPtr B{(float*)(slot + L.b_post),    (float*)(slot + L.b_acc),    (uint8_t*)(slot + L.b_hfl),
              (uint8_t*)(slot + L.b_sign),  (uint8_t*)(slot + L.b_cfl),  (int8_t*)(slot + L.b_status),
              (float*)(slot + L.b_min1),    (float*)(slot + L.b_min2),   (uint16_t*)(slot + L.b_amin),
              (int*)(slot + L.b_deg),       (uint32_t*)(slot + L.b_sp),  (uint32_t*)(slot + L.b_par),
              (uint32_t*)(slot + L.b_unsat)};
      long long* gdg_it = (long long*)(sm + L.misc + 16);
      if (tid == 0) *gdg_it = 0;
      __syncthreads();
      for (int id = warp; id < P.nb; id += NW) {
        BranchTrace* btr = tr ? (BranchTrace*)(tr + trace_off_br()) + id : nullptr;
        StepTrace* st = tr ? (StepTrace*)(tr + trace_off_st(P.nb)) + (size_t)id * dmx : nullptr;
        int8_t* fs = tr ? (int8_t*)(tr + trace_off_fs(P.nb, dmx)) + (size_t)id * ns_max : nullptr;
        run_branch(P, G, B, id, lane, &res_status[id], &res_pm[id], res_e + (size_t)id * L.sw, btr, st,
                   dmx, fs, gdg_it);
      }
      __syncthreads();
      // ---- a8: least path metric, ties to the lowest id ----
      if (tid == 0) {
        int best = -1;
        double bp = CUDART_INF;
        for (int id = 0; id < P.nb; ++id)
          if (res_status[id] == BR_CONVERGED && res_pm[id] < bp) {
            bp = res_pm[id];
            best = id;
          }
        misc[1] = best;
        atomicAdd((unsigned long long*)&counters[1], (unsigned long long)(*gdg_it));
        atomicAdd((unsigned long long*)&counters[3], 1ull);
      }
      __syncthreads();
      winner = misc[1];
      const uint32_t* eb = res_e + (size_t)(winner >= 0 ? winner : 0) * L.sw;
      for (int k = tid; k < n_short; k += NT)
        if ((eb[k >> 5] >> (k & 31)) & 1u) atomicOr(&cbits[sel[k] >> 5], 1u << (sel[k] & 31));
      if (tr)
        for (int k = tid; k < n_short; k += NT) ((uint16_t*)(tr + trace_off_sel(P.nb, dmx, ns_max)))[k] = sel[k];
    }
    __syncthreads();
    uint32_t* co = corr + (size_t)shot * corr_words;
    for (int x = tid; x < corr_words; x += NT) co[x] = x < L.cw ? cbits[x] : 0u;
    if (tid == 0) {
      if (status_out) status_out[shot] = conv ? -1 : (winner >= 0 ? winner : -2);
      if (tr) {
        int32_t* h = (int32_t*)tr;
        h[0] = conv ? 1 : 0;
        h[1] = conv ? -1 : winner;
        h[2] = n_short;
        h[3] = t_run;
      }
    }
  }
}

// ---- Philox4x32-10 (Salmon et al., SC'11) ----
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// One warp per shot; fired columns XOR their detectors into a warp-private
// shared-memory row.
__global__ void sample_kernel(int n_cols, const uint32_t* __restrict__ thr, const int* __restrict__ cptr,
                              const int* __restrict__ cdet, const uint32_t* __restrict__ cobs, int det_words,
                              unsigned long long seed, unsigned long long off, long long n,
                              uint32_t* __restrict__ det, uint32_t* __restrict__ obs) {
  extern __shared__ uint32_t srow[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long s = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  uint32_t* row = srow + (size_t)wib * det_words;
  for (int x = lane; x < det_words; x += 32) row[x] = 0;
  __syncwarp();
  uint32_t ob = 0;
  if (s < n) {
    const unsigned long long shot = off + (unsigned long long)s;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int ng = (n_cols + 3) >> 2;
    for (int g = lane; g < ng; g += 32) {
      uint4 u = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)shot, (uint32_t)(shot >> 32), 0u), key);
      uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int c = 4 * g + r;
        if (c < n_cols && uu[r] < thr[c]) {
          for (int e = cptr[c]; e < cptr[c + 1]; ++e) {
            int d = cdet[e];
            atomicXor(&row[d >> 5], 1u << (d & 31));
          }
          ob ^= cobs[c];
        }
      }
    }
  }
  __syncwarp();
  ob = __reduce_xor_sync(FULL, ob);
  if (s < n) {
    for (int x = lane; x < det_words; x += 32) det[(size_t)s * det_words + x] = row[x];
    if (lane == 0) obs[s] = ob;
  }
}

// Commit (Eq. (10)) + residue test (Eq. (11)); one thread per shot.
__global__ void commit_kernel(int n_commit, const int* __restrict__ cptr, const int* __restrict__ cdet,
                              const uint32_t* __restrict__ cobs, int corr_words,
                              const uint32_t* __restrict__ corr, long long n, uint32_t* __restrict__ det,
                              int det_words, uint32_t* __restrict__ obs_pred, uint32_t* __restrict__ resid,
                              int res_b0, int res_b1) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t* c = corr + (size_t)s * corr_words;
  uint32_t* d = det + (size_t)s * det_words;
  uint32_t ob = 0;
  const int nw = (n_commit + 31) >> 5;
  for (int x = 0; x < nw; ++x) {
    uint32_t m = c[x];
    int rem = n_commit - 32 * x;
    if (rem < 32) m &= (1u << rem) - 1u;
    while (m) {
      int b = __ffs(m) - 1;
      m &= m - 1;
      int col = 32 * x + b;
      for (int e = cptr[col]; e < cptr[col + 1]; ++e) {
        int q = cdet[e];
        d[q >> 5] ^= 1u << (q & 31);
      }
      ob ^= cobs[col];
    }
  }
  obs_pred[s] ^= ob;
  uint32_t bad = 0;
  for (int q = res_b0; q < res_b1;) {
    int wq = q >> 5, lo = q & 31;
    int hiq = min(res_b1, (wq + 1) * 32);
    uint32_t m = d[wq] >> lo;
    int nb = hiq - q;
    if (nb < 32) m &= (1u << nb) - 1u;
    bad |= m;
    q = hiq;
  }
  if (bad) resid[s] |= 1u;
}

__global__ void evaluate_kernel(const uint32_t* __restrict__ pred, const uint32_t* __restrict__ obs,
                                const uint32_t* __restrict__ resid, long long n, uint32_t* __restrict__ fail,
                                long long* __restrict__ n_fail) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t f = 0;
  if (s < n) {
    f = (resid[s] & 1u) | ((pred[s] != obs[s]) ? 2u : 0u);
    if (fail) fail[s] = f;
  }
  unsigned m = __ballot_sync(FULL, f != 0);
  if (n_fail && (threadIdx.x & 31) == 0 && m) atomicAdd((unsigned long long*)n_fail, (unsigned long long)__popc(m));
}

}  // namespace dev
}  // namespace qd

// ---------------------------------------------------------------------------
// Host-side launch wrappers (declared in qdec_internal.h).
namespace qd {

size_t trace_bytes_per_shot(int nb, int dmx, int ns_max) { return dev::trace_bytes(nb, dmx, ns_max); }

cudaError_t set_decode_smem(size_t bytes) {
  return cudaFuncSetAttribute(dev::decode_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

cudaError_t decode_occupancy(int threads, size_t smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dev::decode_window_kernel, threads, smem);
}

cudaError_t launch_decode(int grid, int threads, size_t smem, cudaStream_t st, const KParams& P,
                          const WinDev& W, const Layout& L, const uint32_t* det, int det_words,
                          long long n, uint32_t* corr, int corr_words, int32_t* status, char* trace,
                          size_t tr_bytes, int dmx, int ns_max, int* work, long long* counters) {
  dev::decode_window_kernel<<<grid, threads, smem, st>>>(P, W, L, det, det_words, n, corr, corr_words,
                                                         status, trace, tr_bytes, dmx, ns_max, work,
                                                         counters);
  return cudaGetLastError();
}

cudaError_t launch_sample(cudaStream_t st, int n_cols, const uint32_t* thr, const int* cptr,
                          const int* cdet, const uint32_t* cobs, int det_words,
                          unsigned long long seed, unsigned long long off, long long n, uint32_t* det,
                          uint32_t* obs) {
  if (n <= 0) return cudaSuccess;
  const int wpb = 8;
  long long blocks = (n + wpb - 1) / wpb;
  dev::sample_kernel<<<(unsigned)blocks, 32 * wpb, sizeof(uint32_t) * wpb * det_words, st>>>(
      n_cols, thr, cptr, cdet, cobs, det_words, seed, off, n, det, obs);
  return cudaGetLastError();
}

cudaError_t launch_commit(cudaStream_t st, int n_commit, const int* cptr, const int* cdet,
                          const uint32_t* cobs, int corr_words, const uint32_t* corr, long long n,
                          uint32_t* det, int det_words, uint32_t* obs_pred, uint32_t* resid, int b0,
                          int b1) {
  if (n <= 0) return cudaSuccess;
  const int tpb = 128;
  dev::commit_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(
      n_commit, cptr, cdet, cobs, corr_words, corr, n, det, det_words, obs_pred, resid, b0, b1);
  return cudaGetLastError();
}

cudaError_t launch_evaluate(cudaStream_t st, const uint32_t* pred, const uint32_t* obs,
                            const uint32_t* resid, long long n, uint32_t* fail, long long* n_fail) {
  if (n <= 0) return cudaSuccess;
  const int tpb = 256;
  dev::evaluate_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(pred, obs, resid, n, fail, n_fail);
  return cudaGetLastError();
}

}  // namespace qd
