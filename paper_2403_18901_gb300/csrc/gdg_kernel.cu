// gdg_kernel.cu -- the window decoder, sampler, commit and evaluation kernels.
//
// decode, per shot:
//   a1  window syndrome: bits [row0, row0 + n_rows) of the shot's detectors
//   a2  pre-BP: n_pre flooding min-sum iterations on the full window
//       (Eq. (1)-(4)); a check node by one lane (shot mode) or a lane group
//       (path mode), a variable node by one thread; early stop when H e = s
//       (Sec. II-A), tested inside the next check pass
//   a3  ranking key ((h0+h1)+h2)+h3 of the last four posteriors, bitonic sort
//       of (key, column) ascending, first 2w' columns kept (Sec. III); the
//       shortened matrix is rebuilt in shared memory with its checks and
//       columns numbered in processing order (descending degree)
//   a4-a7 GDG decision paths (Alg. 2 on the 2^k tree and the side branches of
//       Fig. 2): BP steps of iters_per_step iterations, SELECT-VN (Alg. 1)
//       with aggressive decimation (Alg. 3), guess value by the path id,
//       peeling
//   a8  minimum path metric Eq. (5) over converged paths, ties to the lowest id;
//       without a converged path, path 0 or (fallback rules) the estimate with
//       the fewest unsatisfied (committed, then all) checks
//   (message reuse between windows, optional) the output path's final
//       posteriors kept per window column; the next window's pre-BP starts
//       its first VN->CN messages from them
//
// Two launch shapes run the same path code:
//   shot mode (throughput): persistent CTAs of up to 8 warps take shots from
//     a work counter; after the CTA-wide pre-BP the warps take decision paths
//     from a shared-memory queue in a host-planned order, one warp per path;
//     paths resume from snapshots of the prefixes they share with earlier
//     paths, and at every step boundary a warp parks its path for a waiting
//     one with more steps left (snapshots in a per-CTA pool in global memory;
//     see ForkCtx);
//   path mode (latency, small batches): one CTA per (shot, path); the path
//     CTAs of a shot form a thread-block cluster that splits the pre-BP over
//     distributed shared memory, each CTA then ranks, shortens and runs its
//     one path with all its threads, stores the result in global scratch,
//     and the last CTA of the shot to arrive (atomic counter, no waiting)
//     picks the winner.
// Every wait is a CTA, warp or cluster barrier, except the bulk-copy
// mbarrier, whose wait is bounded; the path scheduler never waits (a path
// whose snapshot is not ready starts from an earlier one or from the root).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cfloat>
#include <cstdint>

#include "gdg_kernel.cuh"
#include "qdec_internal.h"

namespace qd {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;
enum { BR_CONVERGED = 0, BR_MAXDEPTH = 1, BR_CONTRADICTION = 2, BR_NOCAND = 3, BR_INTERNAL = 4 };
constexpr int kNone = 0x7fffffff;

// |x| bounded by c by min / max: for finite x the comparisons' result; a NaN
// x (only a dead entry of a decision path's check pass) gives +c, so its sign
// bit is 0 and needs no mask there
__device__ __forceinline__ float clipf(float x, float c) { return fmaxf(fminf(x, c), -c); }

// mu_{j->i} from the check's compressed state (see gdg_kernel.cuh).
__device__ __forceinline__ float c2v_msg(float alpha, float clip, const CNState& c, int e, uint32_t sg) {
  float m = ((c.ac & 0xFFFFu) == (uint32_t)e) ? c.m2 : c.m1;
  if (c.ac & (2u << 16)) m = clip;  // single active VN: minimum over the empty set = clip
  const float mag = __fmul_rn(alpha, m);
  return ((((c.ac >> 16) & 1u) ^ sg) != 0) ? -mag : mag;
}

// Check state as stored.  With learned weights the magnitudes stay unscaled
// (each edge applies its own weight); for the plain decoder they are stored
// already multiplied by alpha (alpha * clip for a single active input), the
// same FP32 products c2v_msg forms, with the parity as their sign, so a
// message is one select and the edge's own sign.
// `rows` (the check's CSR range, begin | end << 16) rides along in the
// record's last word, so the check pass loads it with the state.
template <bool LW>
__device__ __forceinline__ CNState cn_store(float alpha, float clip, float m1, float m2, int am, uint32_t par,
                                            bool single, uint32_t rows) {
  if (LW) return CNState{m1, m2, (uint32_t)am | (par << 16) | ((uint32_t)single << 17), rows};
  const float s1 = __fmul_rn(alpha, single ? clip : m1);
  const float s2 = single ? s1 : __fmul_rn(alpha, m2);
  // the sign parity rides in the sign bits of the two (non-negative) magnitudes
  return CNState{par ? -s1 : s1, par ? -s2 : s2, (uint32_t)am, rows};
}

template <bool LW>
__device__ __forceinline__ float c2v(float w, float clip, const CNState& c, int e, uint32_t sg) {
  if (LW) return c2v_msg(w, clip, c, e, sg);
  const float m = (c.ac == (uint32_t)e) ? c.m2 : c.m1;  // signed by the parity already
  return sg ? -m : m;
}

__device__ __forceinline__ uint32_t bit_of(const uint32_t* w, int j) { return (w[j >> 5] >> (j & 31)) & 1u; }

// ---- bulk asynchronous copies global -> shared (TMA, cp.async.bulk) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// A CTA's staging state: its mbarrier (one arrival + transaction bytes per
// phase), the parity of the phase in flight, a shared flag that turns the
// bulk path off after a wait ran out, and the counter such events go to.
struct Stager {
  uint64_t* bar;
  int* off;
  long long* err;
  unsigned phase;
};

__device__ __forceinline__ Stager stager_init(char* where, long long* err) {
  Stager st{(uint64_t*)where, (int*)(where + 8), err, 0u};
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(st.bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *st.off = 0;
  }
  __syncthreads();
  return st;
}

struct StagePiece {
  void* dst;
  const void* src;
  unsigned bytes;
};

// Copies the pieces into shared memory, all threads calling: one bulk copy
// per piece issued by thread 0, completion tracked on the mbarrier, every
// thread waiting with a bound of ~2^31 cycles.  Pieces that are not 16-byte
// aligned in address and size, an empty list, or a wait that ran out (counted
// in *err; the bulk path then stays off for this CTA) use plain loads.
__device__ void stage_pieces(Stager& st, const StagePiece* pc, int n) {
  bool aligned = true;
  unsigned tot = 0;
  for (int i = 0; i < n; ++i) {
    aligned = aligned && (((smem_u32(pc[i].dst) | (unsigned)(uintptr_t)pc[i].src | pc[i].bytes) & 15u) == 0u);
    tot += pc[i].bytes;
  }
  __syncthreads();  // every earlier access to these bytes has finished
  if (aligned && tot > 0 && !*st.off) {
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(st.bar)), "r"(tot)
                   : "memory");
      for (int i = 0; i < n; ++i)
        if (pc[i].bytes)
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                           smem_u32(pc[i].dst)),
                       "l"(pc[i].src), "r"(pc[i].bytes), "r"(smem_u32(st.bar))
                       : "memory");
    }
    unsigned ok = 0;
    const long long t0 = clock64();
    while (!ok && clock64() - t0 < (1ll << 31)) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                   : "=r"(ok)
                   : "r"(smem_u32(st.bar)), "r"(st.phase)
                   : "memory");
    }
    st.phase ^= 1u;
    if (__syncthreads_and(ok != 0)) return;
    if (threadIdx.x == 0) {
      *st.off = 1;
      atomicAdd((unsigned long long*)st.err, 1ull);
    }
  }
  for (int i = 0; i < n; ++i) {
    const uint16_t* s16 = (const uint16_t*)pc[i].src;
    uint16_t* d16 = (uint16_t*)pc[i].dst;
    for (unsigned x = threadIdx.x; x < pc[i].bytes / 2; x += blockDim.x) d16[x] = s16[x];
  }
  __syncthreads();
}

// Multiplier of Eq. (1) at iteration t >= 1 for full-window edge ef: alpha, or
// the learned weight w[min(t, T)][ef].
__device__ __forceinline__ float edge_weight(const float* wts, int wT, int wE, float alpha, int t, int ef) {
  if (!wts) return alpha;
  const int row = t < 1 ? 0 : (t < wT ? t : wT) - 1;  // never a row before the first
  return wts[(size_t)row * wE + ef];
}

// order-preserving map of a float to uint32 (-0 and +0 equal)
__device__ __forceinline__ uint32_t ordkey(float f) {
  if (f == 0.0f) f = 0.0f;
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ void warp_min2(float& m1, float& m2, int& am) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const float x1 = __shfl_xor_sync(FULL, m1, off);
    const float x2 = __shfl_xor_sync(FULL, m2, off);
    const int xa = __shfl_xor_sync(FULL, am, off);
    if (x1 < m1 || (x1 == m1 && xa < am)) {
      m2 = fminf(m1, x2);
      m1 = x1;
      am = xa;
    } else {
      m2 = fminf(m2, x1);
    }
  }
}

// (min1, min2, argmin) and sign parity over aligned groups of tpc lanes
// (tpc a power of two <= 32); every lane of a group ends with the result.
__device__ __forceinline__ void group_min2(float& m1, float& m2, int& am, uint32_t& neg, int tpc) {
  for (int off = tpc >> 1; off; off >>= 1) {
    const float x1 = __shfl_xor_sync(FULL, m1, off);
    const float x2 = __shfl_xor_sync(FULL, m2, off);
    const int xa = __shfl_xor_sync(FULL, am, off);
    neg ^= __shfl_xor_sync(FULL, neg, off);
    if (x1 < m1 || (x1 == m1 && xa < am)) {
      m2 = fminf(m1, x2);
      m1 = x1;
      am = xa;
    } else {
      m2 = fminf(m2, x1);
    }
  }
}

__host__ __device__ inline int lanes_per_check(int threads, int n_checks) {
  int t = 1;
  while (t < 8 && 2 * t * n_checks <= threads) t <<= 1;
  return t;
}

// Lanes per check of a decision path run by a whole CTA: the most (<= 8) that
// keep the check pass within two rounds of threads / lanes checks.  Checks
// come in descending degree, so the first round holds the heavy ones, whose
// edges the extra lanes split (measured on [[144]] (3,1) windows, 216 checks,
// 512 threads: 1.18 / 1.02 / 1.19 ms per window with 2 / 4 / 8 lanes).
__host__ __device__ inline int path_lanes_per_check(int threads, int n_checks) {
  int t = 1;
  while (t < 8 && 2 * (threads / (2 * t)) >= n_checks) t <<= 1;
  return t;
}

// lexicographic (value, index) minimum over the warp
__device__ __forceinline__ void warp_argmin(float& v, int& k) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const float xv = __shfl_xor_sync(FULL, v, off);
    const int xk = __shfl_xor_sync(FULL, k, off);
    if (xv < v || (xv == v && xk < k)) {
      v = xv;
      k = xk;
    }
  }
}

// Exclusive scan of a[0..n) in place, by one warp; returns the total.
__device__ int warp_scan_excl(int* a, int n, int lane) {
  const int chunk = (n + 31) / 32;
  const int beg = lane * chunk, end = min(n, beg + chunk);
  int s = 0;
  for (int i = beg; i < end; ++i) s += a[i];
  int incl = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, off);
    if (lane >= off) incl += y;
  }
  int run = incl - s;
  for (int i = beg; i < end; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
  return __shfl_sync(FULL, incl, 31);
}

// ---- cooperative groups of threads that run one decision path ----
struct WarpGrp {  // one warp
  int rank;
  static constexpr int size = 32;
  static constexpr bool kWarp = true;
  __device__ void sync() const { __syncwarp(); }
  __device__ bool all(bool p) const { return __all_sync(FULL, p); }
  __device__ bool any(bool p) const { return __any_sync(FULL, p); }
  __device__ unsigned min_u(unsigned v) const { return __reduce_min_sync(FULL, v); }
  __device__ int sum_i(int v) const { return (int)__reduce_add_sync(FULL, (unsigned)v); }
  __device__ long long sum_ll(long long v) const {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
  }
  __device__ double sum_d(double v) const {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
  }
  __device__ void argmin(float& v, int& k) const { warp_argmin(v, k); }
  // SELECT-VN's reductions in one: two lexicographic argmins and a count;
  // every lane's shared-memory writes are visible after it
  __device__ void select_reduce(float& bv, int& bk, float& tv, int& tk, int& n) const {
    warp_argmin(bv, bk);
    warp_argmin(tv, tk);
    n = (int)__reduce_add_sync(FULL, (unsigned)n);
    __syncwarp();
  }
};

struct CtaGrp {  // the whole CTA; every member must call every primitive
  int rank, size;
  static constexpr bool kWarp = false;
  char* red;  // >= 32 * 16 bytes of shared memory
  __device__ void sync() const { __syncthreads(); }
  __device__ bool all(bool p) const { return __syncthreads_and(p) != 0; }
  __device__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
  __device__ unsigned min_u(unsigned v) const {
    v = __reduce_min_sync(FULL, v);
    unsigned* r = (unsigned*)red;
    __syncthreads();
    if ((rank & 31) == 0) r[rank >> 5] = v;
    __syncthreads();
    unsigned m = r[0];
    for (int i = 1; i < (size >> 5); ++i) m = min(m, r[i]);
    return m;
  }
  __device__ int sum_i(int v) const {
    v = (int)__reduce_add_sync(FULL, (unsigned)v);
    int* r = (int*)red;
    __syncthreads();
    if ((rank & 31) == 0) r[rank >> 5] = v;
    __syncthreads();
    int s = 0;
    for (int i = 0; i < (size >> 5); ++i) s += r[i];
    return s;
  }
  __device__ long long sum_ll(long long v) const {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    long long* r = (long long*)red;
    __syncthreads();
    if ((rank & 31) == 0) r[rank >> 5] = v;
    __syncthreads();
    long long s = 0;
    for (int i = 0; i < (size >> 5); ++i) s += r[i];
    return s;
  }
  __device__ double sum_d(double v) const {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    double* r = (double*)red;
    __syncthreads();
    if ((rank & 31) == 0) r[rank >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (size >> 5); ++i) s += r[i];
    return s;
  }
  __device__ void argmin(float& v, int& k) const {
    warp_argmin(v, k);
    float* rv = (float*)red;
    int* rk = (int*)(red + 4 * 32);
    __syncthreads();
    if ((rank & 31) == 0) {
      rv[rank >> 5] = v;
      rk[rank >> 5] = k;
    }
    __syncthreads();
    v = rv[0];
    k = rk[0];
    for (int i = 1; i < (size >> 5); ++i)
      if (rv[i] < v || (rv[i] == v && rk[i] < k)) {
        v = rv[i];
        k = rk[i];
      }
  }
  // SELECT-VN's reductions in one exchange (two barriers instead of seven):
  // two lexicographic argmins and a count, for at most 16 warps (the
  // path-mode CTA); every thread's shared-memory writes are visible after it
  __device__ void select_reduce(float& bv, int& bk, float& tv, int& tk, int& n) const {
    warp_argmin(bv, bk);
    warp_argmin(tv, tk);
    n = (int)__reduce_add_sync(FULL, (unsigned)n);
    float* r_bv = (float*)red;
    int* r_bk = (int*)(red + 64);
    float* r_tv = (float*)(red + 128);
    int* r_tk = (int*)(red + 192);
    int* r_n = (int*)(red + 256);
    __syncthreads();
    if ((rank & 31) == 0) {
      const int w = rank >> 5;
      r_bv[w] = bv;
      r_bk[w] = bk;
      r_tv[w] = tv;
      r_tk[w] = tk;
      r_n[w] = n;
    }
    __syncthreads();
    bv = r_bv[0];
    bk = r_bk[0];
    tv = r_tv[0];
    tk = r_tk[0];
    n = r_n[0];
    for (int i = 1; i < (size >> 5); ++i) {
      if (r_bv[i] < bv || (r_bv[i] == bv && r_bk[i] < bk)) {
        bv = r_bv[i];
        bk = r_bk[i];
      }
      if (r_tv[i] < tv || (r_tv[i] == tv && r_tk[i] < tk)) {
        tv = r_tv[i];
        tk = r_tk[i];
      }
      n += r_n[i];
    }
  }
};

struct ShortG {
  int nr, ns, rw;
  const uint16_t *colptr, *colrows, *rowptr;
  const uint32_t* rowent;  // CSR entry: edge id | (short column << 16)
  const float* llr;
  const uint8_t* vdeg;
  const uint32_t* sbits;
  const uint16_t* efull;  // short edge -> full-window edge (learned weights)
  const float* wts;
  int wT, wE;
  int rpb;  // window rows per block (block of a column = its first row / rpb)
  const uint16_t* sel;    // short column -> window column
  // Checks and short columns are numbered by descending degree (ties by
  // window row / rank); these map a label back to the window row and to the
  // ranked column, whose order decides every tie.
  const uint16_t* cperm;
  const uint16_t* vperm;
  int ncr;  // window rows [0, ncr) are the ones the window commits
};

struct Slot {
  float *post, *acc;
  uint8_t *hfl, *sign;
  int8_t* status;
  CNState* cns;
  int* deg;
  uint32_t *sp, *unsat;
  int8_t* hq;  // ranker only: the last four posteriors as round(2 clamp(x, 63.5)), oldest first
};

__device__ __forceinline__ Slot make_slot(char* base, const Layout& L) {
  return Slot{(float*)(base + L.b_post),   (float*)(base + L.b_acc),     (uint8_t*)(base + L.b_hfl),
              (uint8_t*)(base + L.b_sign), (int8_t*)(base + L.b_status), (CNState*)(base + L.b_cns),
              (int*)(base + L.b_deg),      (uint32_t*)(base + L.b_sp),
              (uint32_t*)(base + L.b_unsat), (int8_t*)(base + L.b_hq)};
}

// Posterior of a decimated VN: a NaN, so the check-node pass recognises a
// stale edge from the posterior it loads anyway.
__device__ __forceinline__ float stale() { return __int_as_float(0x7fffffff); }

__device__ __forceinline__ void decimate_atomic(const ShortG& G, const Slot& B, int k, int v) {
  B.status[k] = (int8_t)v;
  B.post[k] = stale();
  for (int e = G.colptr[k]; e < G.colptr[k + 1]; ++e) {
    const int j = G.colrows[e];
    atomicSub(&B.deg[j], 1);
    if (v) atomicXor(&B.sp[j >> 5], 1u << (j & 31));
  }
}

__device__ __forceinline__ void decimate_one(const ShortG& G, const Slot& B, int k, int v) {
  B.status[k] = (int8_t)v;
  B.post[k] = stale();
  for (int e = G.colptr[k]; e < G.colptr[k + 1]; ++e) {
    const int r = G.colrows[e];
    B.deg[r] -= 1;
    if (v) B.sp[r >> 5] ^= 1u << (r & 31);
  }
}

// Peeling (Sec. IV): repeatedly fix the lone active VN of a degree-one check
// to the check's current syndrome; a check left with no active VN and
// syndrome 1 is a contradiction.  One check at a time, always the lowest-index
// degree-one check, after testing every check for a contradiction (this order
// also fixes the partial state of a path killed by a contradiction).
// Returns #peeled, -1 (contradiction) or -2 (inconsistent degree count).
template <class Grp>
__device__ int peel(const ShortG& G, const Slot& B, const Grp& g) {
  int npeel = 0;
  for (int guard = 0; guard <= G.ns + 1; ++guard) {
    bool contra = false;
    int cand = kNone;  // (window row << 16) | label of the lowest degree-one check
    for (int j = g.rank; j < G.nr; j += g.size) {
      const int d = B.deg[j];
      if (d == 0) {
        if (bit_of(B.sp, j)) contra = true;
      } else if (d == 1) {
        cand = min(cand, ((int)G.cperm[j] << 16) | j);
      }
    }
    if (g.any(contra)) return -1;
    const int jc = (int)g.min_u((unsigned)cand);
    if (jc == kNone) return npeel;
    const int j = jc & 0xFFFF;
    int found = kNone;
    for (int q = G.rowptr[j] + g.rank; q < G.rowptr[j + 1]; q += g.size) {
      const int i = (int)(G.rowent[q] >> 16);
      if (B.status[i] == -1) found = i;
    }
    const int i = (int)g.min_u((unsigned)found);
    if (i == kNone) return -2;
    const int v = (int)bit_of(B.sp, j);
    g.sync();
    if (g.rank == 0) decimate_one(G, B, i, v);
    g.sync();
    ++npeel;
  }
  return -2;
}

// ---- learned decimation ranker (replaces the argmin of Alg. 1) ----
// score = W2 . relu(W1 x + b1) + b2 over the candidate features
//   x = (L/4, h0, h1, h2, h3 on the 1/2 grid clamped to +-63.5, #unsatisfied
//        neighbour checks (<= 127), static degree, block of the first
//        detector (<= 255)).
// With W1 on the 2^-6 grid in [-2, 2] and b1 on the 2^-7 grid in [-512, 512] every layer-1
// partial sum is a multiple of 2^-7 below 2^13: the BF16 tensor-core product
// with FP32 accumulation is exact, in any order.  Layer 2 runs in FP32 in one
// fixed order per candidate: s_q = sum over t = 0..7, c = 0..1 of
// W2[u] h[u], u = 8t + 2q + c (lane q of the quad that holds those units in
// the MMA accumulator layout), score = ((s_0 + s_1) + (s_2 + s_3)) + b2.

__device__ __forceinline__ float qfeat(float x) {
  return (float)__float2int_rn(2.0f * fminf(fmaxf(x, -63.5f), 63.5f)) * 0.5f;
}
__device__ __forceinline__ int8_t qhist(float x) { return (int8_t)__float2int_rn(2.0f * fminf(fmaxf(x, -63.5f), 63.5f)); }

// two BF16-exact floats as a packed pair (low half = first)
__device__ __forceinline__ uint32_t bf16x2_exact(float lo, float hi) {
  return (__float_as_uint(lo) >> 16) | (__float_as_uint(hi) & 0xFFFF0000u);
}

// D = A B + C, m16n8k8, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void mma_m16n8k8_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0, float c0,
                                                 float c1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%9,%10};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0), "f"(c0), "f"(c1), "f"(c0), "f"(c1));
}

__device__ __forceinline__ bool ranker_candidate(const ShortG& G, const Slot& B, int k) {
  return k < G.ns && B.status[k] == -1 && G.vdeg[k] > 2;
}

// Features 2 tig and 2 tig + 1 of short column k (zero for a non-candidate).
__device__ __forceinline__ uint32_t ranker_pair(const ShortG& G, const Slot& B, int k, bool cand, int tig) {
  if (!cand) return 0u;
  float lo, hi;
  const uint32_t h4 = *(const uint32_t*)(B.hq + 4 * k);
  const float hv0 = (float)(int8_t)(h4 & 0xFF) * 0.5f, hv1 = (float)(int8_t)((h4 >> 8) & 0xFF) * 0.5f;
  const float hv2 = (float)(int8_t)((h4 >> 16) & 0xFF) * 0.5f, hv3 = (float)(int8_t)(h4 >> 24) * 0.5f;
  if (tig == 0) {
    lo = qfeat(__fmul_rn(B.acc[k], 0.25f));
    hi = hv0;
  } else if (tig == 1) {
    lo = hv1;
    hi = hv2;
  } else if (tig == 2) {
    int nus = 0;
    for (int e = G.colptr[k]; e < G.colptr[k + 1]; ++e) nus += bit_of(B.unsat, G.colrows[e]);
    lo = hv3;
    hi = (float)min(nus, 127);
  } else {
    lo = (float)G.vdeg[k];
    hi = (float)min(G.cperm[G.colrows[G.colptr[k]]] / G.rpb, 255);
  }
  return bf16x2_exact(lo, hi);
}

// Highest score over the candidates (ties to the lowest ranked column), as
// (-score, (ranked column << 16) | label) for the group's lexicographic
// argmin.  Each warp of the group scores tiles of 16 consecutive labels;
// every lane of the group calls.
template <class Grp>
__device__ void ranker_select(const KParams& P, const ShortG& G, const Slot& B, const Grp& g, float& nv, int& nk) {
  const int lane = g.rank & 31, wid = g.rank >> 5, nw = g.size >> 5;
  const int gi = lane >> 2, tig = lane & 3, qb = lane & ~3;
  const float* b1 = P.rkq + 512;
  const float* w2 = P.rkq + 576;
  const float b2 = P.rkq[640];
  nv = CUDART_INF_F;
  nk = kNone;
  for (int t0 = 16 * wid; t0 < G.ns; t0 += 16 * nw) {
    const int r0 = t0 + gi, r1 = r0 + 8;
    const bool c0 = ranker_candidate(G, B, r0), c1 = ranker_candidate(G, B, r1);
    const uint32_t a0 = ranker_pair(G, B, r0, c0, tig), a1 = ranker_pair(G, B, r1, c1, tig);
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int u = 8 * t + 2 * tig;
      float d[4];
      mma_m16n8k8_bf16(d, a0, a1, P.rkb[32 * t + lane], b1[u], b1[u + 1]);
      const float wa = w2[u], wb = w2[u + 1];
      s0 = __fadd_rn(s0, __fmul_rn(wa, d[0] > 0.0f ? d[0] : 0.0f));
      s0 = __fadd_rn(s0, __fmul_rn(wb, d[1] > 0.0f ? d[1] : 0.0f));
      s1 = __fadd_rn(s1, __fmul_rn(wa, d[2] > 0.0f ? d[2] : 0.0f));
      s1 = __fadd_rn(s1, __fmul_rn(wb, d[3] > 0.0f ? d[3] : 0.0f));
    }
    float q[4], p[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      q[i] = __shfl_sync(FULL, s0, qb + i);
      p[i] = __shfl_sync(FULL, s1, qb + i);
    }
    const float sc0 = __fadd_rn(__fadd_rn(__fadd_rn(q[0], q[1]), __fadd_rn(q[2], q[3])), b2);
    const float sc1 = __fadd_rn(__fadd_rn(__fadd_rn(p[0], p[1]), __fadd_rn(p[2], p[3])), b2);
    // ties to the lowest ranked column: (column << 16) | label
    if (c0) {
      const int pk = ((int)G.vperm[r0] << 16) | r0;
      if (-sc0 < nv || (-sc0 == nv && pk < nk)) {
        nv = -sc0;
        nk = pk;
      }
    }
    if (c1) {
      const int pk = ((int)G.vperm[r1] << 16) | r1;
      if (-sc1 < nv || (-sc1 == nv && pk < nk)) {
        nv = -sc1;
        nk = pk;
      }
    }
  }
  g.argmin(nv, nk);
}

// Records of every candidate of this step (path 0 only), in any order.
template <class Grp>
__device__ void dump_candidates(const KParams& P, const ShortG& G, const Slot& B, const Grp& g, long long shot, int D,
                                int gsel) {
  for (int k = g.rank; k < G.ns; k += g.size) {
    if (!ranker_candidate(G, B, k)) continue;
    const uint32_t h4 = *(const uint32_t*)(B.hq + 4 * k);
    int nus = 0;
    for (int e = G.colptr[k]; e < G.colptr[k + 1]; ++e) nus += bit_of(B.unsat, G.colrows[e]);
    const float L = B.acc[k];
    const int pos = atomicAdd(P.dump_n, 1);
    if (pos >= P.dump_cap) continue;
    RankRec r;
    r.x[0] = qfeat(__fmul_rn(L, 0.25f));
    r.x[1] = (float)(int8_t)(h4 & 0xFF) * 0.5f;
    r.x[2] = (float)(int8_t)((h4 >> 8) & 0xFF) * 0.5f;
    r.x[3] = (float)(int8_t)((h4 >> 16) & 0xFF) * 0.5f;
    r.x[4] = (float)(int8_t)(h4 >> 24) * 0.5f;
    r.x[5] = (float)min(nus, 127);
    r.x[6] = (float)G.vdeg[k];
    r.x[7] = (float)min(G.cperm[G.colrows[G.colptr[k]]] / G.rpb, 255);
    r.shot = (int32_t)shot;
    r.wcol = G.sel[G.vperm[k]];
    r.depth = (int16_t)D;
    r.path = 0;
    r.flags = (L <= 0.0f ? 1 : 0) | (k == gsel ? 2 : 0);
    P.dump[pos] = r;
  }
}

// Eq. (5): the summed priors of the path's estimate (decimated values and the
// hard decisions of the active VNs), in FP64 (exact: every prior lies in
// (2^-15, 16), so every partial sum is exact in any order).
template <class Grp>
__device__ double path_metric(const ShortG& G, const Slot& B, const Grp& g) {
  double s = 0.0;
  for (int k = g.rank; k < G.ns; k += g.size) {
    const int st8 = B.status[k];
    if (st8 == 1 || (st8 == -1 && B.post[k] <= 0.0f)) s += (double)G.llr[k];
  }
  return g.sum_d(s);
}

// H e = s for the current decisions (Eq. (4), decimated VNs through s'):
// writes every check's unsatisfied bit to B.unsat and returns whether any is
// unsatisfied.  Checks in natural order, one per lane.
template <class Grp>
__device__ bool parity_pass(const ShortG& G, const Slot& B, const Grp& g) {
  bool any = false;
  for (int base = 0; base < G.nr; base += g.size) {
    const int j = base + g.rank;
    bool u = false;
    if (j < G.nr) {
      uint32_t hp = bit_of(B.sp, j);
      for (int q = G.rowptr[j]; q < G.rowptr[j + 1]; ++q) hp ^= B.post[G.rowent[q] >> 16] <= 0.0f;  // NaN: decimated
      u = hp != 0u;
    }
    const unsigned m = __ballot_sync(FULL, u);
    const int w0 = base + (g.rank & ~31);
    if ((g.rank & 31) == 0 && w0 < G.nr) B.unsat[w0 >> 5] = m;
    any |= u;
  }
  return g.any(any);
}

struct PathOut {
  int* status;
  double* pm;
  uint32_t* ebits;
  BranchTrace* btr;
  StepTrace* st;
  int8_t* fstat;
  long long* visits;  // accumulates active edge visits, the path's shared prefix included
  long long* exec;    // accumulates the active edge visits this launch executed (nullable)
  long long shot;
  float* keep;        // message reuse: this path's final values by label (nullable)
};

// Shot mode's shared path prefixes.  Paths that made the same decisions at
// depths 1..D-1 are in the same state after the BP of step D (that BP does
// not depend on the path: both P_A flags of Alg. 3 are kept), so a path can
// resume there from a snapshot another path left instead of recomputing the
// prefix from the root.  A snapshot is a 32-byte header (depth, iterations,
// iterations since the messages were initialised, the `first` flag, the
// producing path, the prefix's edge visits) and a copy of the slot.
//
// Preemption (sched): the paths of a shot outnumber the warps, and the main
// branch is the longest, so a fixed assignment leaves warps idle at the end
// of the shot.  At every step boundary a warp compares the steps its path
// has left with those of the waiting paths -- parked paths, and queued paths
// whose planned snapshot is ready -- and when one has more than one step
// more, it parks its own path (a snapshot of the same form in the path's own
// buffer) and switches to it: longest remaining work first.  Path states
// (sched words): 0 queued, 1 running, 2 | D << 8 parked after the BP of
// step D, 3 done.
struct ForkCtx {
  const char* src;       // snapshot to resume from (nullptr: from the root)
  const int16_t* chain;  // this path's snapshot node by depth (index D - 1), -1: none; nullptr: no snapshots
  int* flags;            // per node: 0 free, 1 being written, 2 ready
  char* pool;            // this CTA's snapshots, `stride` bytes apart: nodes, then one per path
  unsigned stride;
  char* slot;            // this warp's slot and its size
  unsigned slot_bytes;
  const StepTrace* st0;  // the shot's step records (path p at st0 + p * dmx), or nullptr
  unsigned* sched;       // per path state word (nullptr: no preemption)
  const int16_t* fnode;  // per path: its planned snapshot node (-1: none) and that node's depth
  const int16_t* fdep;
  int n_nodes;
};
constexpr unsigned kSnapHeader = kSnapHeaderBytes;
enum { PS_QUEUED = 0, PS_RUNNING = 1, PS_PARKED = 2, PS_DONE = 3 };

// Snapshot of a path's state after the BP of step D (all lanes of the group).
template <class Grp>
__device__ void write_snapshot(char* dst, const ForkCtx& F, const Grp& g, int D, int iters, int tw, bool first,
                               int producer, long long vs) {
  if (g.rank == 0) {
    int* h = (int*)dst;
    __stcg(h, D);
    __stcg(h + 1, iters);
    __stcg(h + 2, tw);
    __stcg(h + 3, first ? 1 : 0);
    __stcg(h + 4, producer);
    __stcg((long long*)(dst + 24), vs);
  }
  const uint4* s4 = (const uint4*)F.slot;
  uint4* d4 = (uint4*)(dst + kSnapHeader);
  for (unsigned x = g.rank; x < F.slot_bytes / 16u; x += g.size) __stcg(d4 + x, s4[x]);
  __threadfence();  // the snapshot and this path's decision records before its flag
  g.sync();
}

// Check-node update of Eq. (1) over the active VNs of one decision path, TPC
// lanes per check (a template parameter, so that the loops and the group
// reduction are unrolled for it); checks in label order (descending static
// degree): the lanes of a round loop alike.  Each check also takes the parity
// of its active VNs' hard decisions (Eq. (4)) from the posteriors it reads:
// for it >= 2 this pass is the convergence test H e = s of the previous
// iteration (Sec. II-A).  Returns whether this lane saw an unsatisfied check.
template <bool LW, int TPC, int FM>
__device__ __forceinline__ bool check_pass_fm(const KParams& P, const ShortG& G, const Slot& B, int R, int S,
                                              bool first_rt, int tw, long long& visits) {
  // FM: 0 the first-iteration flag at run time, 1 / 2 fixed true / false
  const bool first = FM == 0 ? first_rt : FM == 1;
  const int nr = G.nr, sub = R & (TPC - 1);
  const int nr_rounds = (nr + S / TPC - 1) / (S / TPC) * (S / TPC);
  bool unsat = false;
  int nvis = 0;  // this pass's active edge visits (added to the 64-bit count once)
  for (int j0 = R / TPC; j0 < nr_rounds; j0 += S / TPC) {
    const int j = j0 < nr ? j0 : nr - 1;
    const int d = j0 < nr ? B.deg[j] : 0;
    if (TPC == 1 && d == 0) {  // no shuffle partner waits for this lane
      if (j0 < nr) unsat |= bit_of(B.sp, j) != 0u;
      continue;
    }
    const CNState oc = B.cns[j];
    float m1 = CUDART_INF_F, m2 = CUDART_INF_F;
    int am = 0xFFFF;
    uint32_t neg = 0, hp = 0;
    // one row entry; the (min1, min2) pair and so every message do not
    // depend on the order in which a check sees its inputs
    // (no branch: a NaN input -- the stale message of a decimated VN, or no
    // entry -- takes part with magnitude +inf and writes nothing)
    auto take = [&](uint32_t ent, float pv, uint32_t sg) {
      const bool live = pv == pv;
      hp ^= pv <= 0.0f;  // false for NaN
      const int e = (int)(ent & 0xFFFFu);
      // the previous iteration's multiplier, only when there was one (tw >= 1)
      const float wprev = (LW && !first) ? edge_weight(G.wts, G.wT, G.wE, P.alpha, tw, G.efull[e]) : P.alpha;
      const float v = first ? pv : clipf(__fsub_rn(pv, c2v<LW>(wprev, P.clip, oc, e, sg)), P.clip);
      const float a = live ? fabsf(v) : CUDART_INF_F;
      am = a < m1 ? e : am;
      m2 = fminf(m2, fmaxf(m1, a));
      m1 = fminf(m1, a);
      const uint32_t sgn = v < 0.0f;  // false for a NaN input: clipf gives +clip, the first pass NaN
      neg ^= sgn;
      if (live) B.sign[e] = (uint8_t)sgn;
    };
    if (sub == 0) nvis += d;  // the row's active entries (B.deg counts the active VNs of a check)
    const int qe = d ? (int)(oc.pad >> 16) : 0;
    for (int q = (d ? (int)(oc.pad & 0xFFFFu) : 0) + 2 * sub; q < qe; q += 2 * TPC) {
      const bool two = q + 1 < qe;
      const uint32_t e0 = G.rowent[q], e1 = two ? G.rowent[q + 1] : e0;
      const float p0 = B.post[e0 >> 16], p1 = two ? B.post[e1 >> 16] : stale();
      const uint32_t s0 = B.sign[e0 & 0xFFFFu], s1 = B.sign[e1 & 0xFFFFu];
      take(e0, p0, s0);
      take(e1, p1, s1);
    }
    if (TPC > 1) {
      group_min2(m1, m2, am, neg, TPC);
      for (int off = TPC >> 1; off; off >>= 1) hp ^= __shfl_xor_sync(FULL, hp, off);
    }
    if (sub == 0 && j0 < nr) unsat |= (hp ^ bit_of(B.sp, j)) != 0u;
    if (sub == 0 && d > 0)
      B.cns[j] = cn_store<LW>(P.alpha, P.clip, m1, m2, am, neg ^ bit_of(B.sp, j), d == 1, oc.pad);
  }
  visits += nvis;
  return unsat;
}

// One-warp paths (TPC 1) run a copy specialised for the first iteration after
// the messages were (re)initialised and one for the others.
template <bool LW, int TPC>
__device__ __forceinline__ bool check_pass(const KParams& P, const ShortG& G, const Slot& B, int R, int S, bool first,
                                           int tw, long long& visits) {
  if (TPC == 1)
    return first ? check_pass_fm<LW, TPC, 1>(P, G, B, R, S, true, tw, visits)
                 : check_pass_fm<LW, TPC, 2>(P, G, B, R, S, false, tw, visits);
  return check_pass_fm<LW, TPC, 0>(P, G, B, R, S, first, tw, visits);
}

// One decision path of Alg. 2 on the shortened window, run by group g.
// LW: learned per-edge weights instead of alpha (compiled separately so the
// plain decoder carries no weight lookups).
// Returns -1 when the path is finished, or (preemption) the path this group
// switches to after parking this one; *claimed is the state word it took.
template <bool LW, class Grp>
__device__ int run_path(const KParams& P, const ShortG& G, const Slot& B, int id, const Grp& g,
                        const PathOut& out, int dmx, const ForkCtx& F, unsigned* claimed = nullptr) {
  const int nr = G.nr, ns = G.ns, R = g.rank, S = g.size;
  // one lane per check for a warp; small lane groups per check for a CTA
  const int tpc = Grp::kWarp ? 1 : path_lanes_per_check(S, nr);
  // Fig. 2: main branch (id 0), tree branches, side branches (split > 0),
  // which keep the main-branch thresholds up to and including their split
  const int split = path_split(P, id);
  const int d_reinit = path_reinit(P, id, split);
  const int dmax = path_dmax(P, id, split);
  auto main_rules = [&](int D) { return id == 0 || (split && D <= split); };
  int status = BR_MAXDEPTH, depth = 0, iters = 0;
  int tw = 0;  // iterations since the messages were (re)initialised (learned weights)
  long long visits = 0, inherited = 0;  // executed here / the resumed prefix's (lane 0)
  double pm = CUDART_INF;
  bool first = true;
  int D0 = 1;  // first depth of this run: resumed runs start at its SELECT-VN
  if (F.src) {
    // resume from a snapshot taken after the BP of step D0 by a path with the
    // same decisions at depths 1..D0-1
    const int* h = (const int*)F.src;
    D0 = __ldcg(h);
    iters = __ldcg(h + 1);
    tw = __ldcg(h + 2);
    first = __ldcg(h + 3) != 0;
    const int producer = __ldcg(h + 4);
    if (R == 0) inherited = __ldcg((const long long*)(F.src + 24));
    const uint4* s4 = (const uint4*)(F.src + kSnapHeader);
    uint4* d4 = (uint4*)F.slot;
    for (unsigned x = R; x < F.slot_bytes / 16u; x += S) d4[x] = __ldcg(s4 + x);
    // a path resumed from its own parking snapshot keeps its records
    if (out.st && producer != id) {  // the decision records of the shared prefix are the producer's
      const StepTrace* ps = F.st0 + (size_t)producer * dmx;
      for (int q = R; q < dmx; q += S) {
        StepTrace r{-2, -1, 0, 0, 0};
        if (q < D0 - 1) {
          const uint2 v = __ldcg((const uint2*)(ps + q));
          memcpy(&r, &v, sizeof(r));
        }
        out.st[q] = r;
      }
    }
    g.sync();
  } else {
    for (int k = R; k < ns; k += S) {
      B.status[k] = -1;
      B.post[k] = G.llr[k];  // t = 0: mu_{i->j} = Lambda_i (Sec. II-A)
    }
    for (int j = R; j < nr; j += S) {
      B.deg[j] = G.rowptr[j + 1] - G.rowptr[j];
      B.cns[j].pad = (uint32_t)G.rowptr[j] | ((uint32_t)G.rowptr[j + 1] << 16);
    }
    for (int base = 0; base < nr; base += S) {  // the window syndrome by check label
      const int j = base + R;
      const unsigned m = __ballot_sync(FULL, j < nr && bit_of(G.sbits, G.cperm[j]));
      if ((R & 31) == 0 && base + R < nr) B.sp[(base + R) >> 5] = m;
    }
    if (out.st)
      for (int q = R; q < dmx; q += S) out.st[q] = StepTrace{-2, -1, 0, 0, 0};
    g.sync();
    if (P.peel_init) {
      const int np = peel(G, B, g);
      if (np < 0) {
        status = np == -1 ? BR_CONTRADICTION : BR_INTERNAL;
        goto done;
      }
    }
  }
  for (int D = D0; D <= dmax; ++D) {
    depth = D;
    if (!(F.src && D == D0)) {  // (a resumed run's snapshot holds its first step's BP)
    const int ips = (D == 1 && P.ips1 > 0) ? P.ips1 : P.ips;  // the first step may have its own length
    for (int it = 1; it <= ips; ++it) {
      // ---- check-node update, Eq. (1), and the previous iteration's H e = s ----
      bool unsat;
      if constexpr (Grp::kWarp) {
        unsat = check_pass<LW, 1>(P, G, B, R, S, first, tw, visits);
      } else {
        if (tpc == 8) unsat = check_pass<LW, 8>(P, G, B, R, S, first, tw, visits);
        else if (tpc == 4) unsat = check_pass<LW, 4>(P, G, B, R, S, first, tw, visits);
        else if (tpc == 2) unsat = check_pass<LW, 2>(P, G, B, R, S, first, tw, visits);
        else unsat = check_pass<LW, 1>(P, G, B, R, S, first, tw, visits);
      }
      if (!g.any(unsat) && it >= 2) {  // the previous iteration's decisions satisfy H e = s
        status = BR_CONVERGED;
        pm = path_metric(G, B, g);
        goto done;
      }
      // ---- variable-node update, Eq. (2)-(3); history of Sec. IV-A ----
      const bool hist = it > ips - 4;
      const bool hist0 = it == ips - 3;
      // variables in label order (descending degree): the lanes of a round loop alike
      for (int k = R; k < ns; k += S) {
        // (a decimated column runs the loop too, without a branch, and stores nothing)
        const bool act = B.status[k] == -1;
        float p = G.llr[k];
        const int eb = G.colptr[k], ee = G.colptr[k + 1];
        auto msg = [&](int e) {
          const float wt = LW ? edge_weight(G.wts, G.wT, G.wE, P.alpha, tw + 1, G.efull[e]) : P.alpha;
          return c2v<LW>(wt, P.clip, B.cns[G.colrows[e]], e, B.sign[e]);
        };
        // ascending check order (Eq. (2)); most short columns have degree 1 or 2
        int e = eb;
        for (; e + 1 < ee; e += 2) {
          const float c0 = msg(e), c1 = msg(e + 1);
          p = __fadd_rn(p, c0);
          p = __fadd_rn(p, c1);
        }
        if (e < ee) p = __fadd_rn(p, msg(e));
        if (!act) continue;
        B.post[k] = p;
        if (hist) {
          if (P.rkq || P.dump) B.hq[4 * k + (it - (ips - 3))] = qhist(p);
          // both P_A tests of Alg. 3 (main branch: bit 1, other branches: bit 4),
          // so that the step's BP does not depend on the path
          const uint8_t f = (uint8_t)((p <= 0.0f) | ((p < P.pa_main) << 1) | ((p > P.pc) << 2) | ((p > P.pd) << 3) |
                                      ((p < P.pa_other) << 4));
          if (hist0) {
            B.acc[k] = p;
            B.hfl[k] = f;
          } else {
            B.acc[k] = __fadd_rn(B.acc[k], p);
            B.hfl[k] &= f;
          }
        }
      }
      g.sync();
      ++iters;
      ++tw;
      first = false;
    }
    // the step's last iteration: its own convergence test, which also leaves
    // the unsatisfied-check words for Alg. 3 and the ranker
    if (!parity_pass(G, B, g)) {
      status = BR_CONVERGED;
      pm = path_metric(G, B, g);
      goto done;
    }
    // a snapshot here for paths queued later that share the decisions so far
    // (the first path to get here writes it)
    if (F.chain && F.chain[D - 1] >= 0) {
      const int n = F.chain[D - 1];
      int won = 0;
      if (R == 0) won = atomicCAS(&F.flags[n], 0, 1) == 0;
      if (g.any(won != 0)) {
        write_snapshot(F.pool + (size_t)n * F.stride, F, g, D, iters, tw, first, id, g.sum_ll(visits + inherited));
        if (R == 0) atomicExch(&F.flags[n], 2);
      }
    }
    }
    // preemption point: switch to a waiting path with more steps left (not
    // right where this run resumed)
    if (F.sched && D < dmax && !(F.src && D == D0)) {
      int c = -1;
      unsigned cw = 0;
      if (R == 0) {
        int best = dmax - D + 2;  // more than one step more than this path's dmax - D + 1
        for (int p = 0; p < P.nb; ++p) {
          const unsigned w = *(volatile unsigned*)&F.sched[p];
          int at = 0;
          if ((w & 3u) == PS_PARKED) at = (int)(w >> 8);
          else if (w == PS_QUEUED && F.fnode[p] >= 0 && *(volatile int*)&F.flags[F.fnode[p]] == 2) at = F.fdep[p];
          if (!at) continue;
          const int rem = path_dmax(P, p, path_split(P, p)) - at + 1;
          if (rem > best) {
            best = rem;
            c = p;
            cw = w;
          }
        }
        if (c >= 0 && atomicCAS(&F.sched[c], cw, (unsigned)PS_RUNNING) != cw) c = -1;
      }
      const unsigned cu = g.min_u(R == 0 && c >= 0 ? (unsigned)c : 0xFFFFFFFFu);  // lane 0's choice
      c = cu == 0xFFFFFFFFu ? -1 : (int)cu;
      if (c >= 0) {
        const unsigned cw0 = g.min_u(R == 0 ? cw : 0xFFFFFFFFu);
        if (claimed) *claimed = cw0;
        // park: this path resumes from its own snapshot after the BP of step D
        const long long own = g.sum_ll(visits);
        write_snapshot(F.pool + (size_t)(F.n_nodes + id) * F.stride, F, g, D, iters, tw, first, id,
                       g.sum_ll(visits + inherited));
        if (R == 0) {
          atomicExch(&F.sched[id], (unsigned)PS_PARKED | ((unsigned)D << 8));
          if (out.exec) atomicAdd((unsigned long long*)out.exec, (unsigned long long)own);
        }
        g.sync();
        return c;
      }
    }
    if (D == dmax) break;  // no decimation after the last BP step
    {
      // ---- SELECT-VN (Alg. 1) with AGG-DEC (Alg. 3) ----
      const float PBd = (D == 1) ? P.pb_d1 : (main_rules(D) ? P.pb_main : P.pb_other);
      const uint8_t pa_bit = main_rules(D) ? 2 : 16;
      // bk, tk: (ranked column << 16) | label, so that ties go to the lowest
      // ranked column (the oracle's index order) whatever the label order
      float bL = CUDART_INF_F, tL = CUDART_INF_F;
      int bk = kNone, tk = kNone, nagg = 0;
      for (int k = R; k < ns; k += S) {
        if (B.status[k] != -1 || G.vdeg[k] <= 2) continue;
        const float L = B.acc[k];
        const uint8_t fl = B.hfl[k];
        if (!P.low_err) {
          int nus = 0;
          for (int e = G.colptr[k]; e < G.colptr[k + 1]; ++e) nus += bit_of(B.unsat, G.colrows[e]);
          int bdec = -1;
          if ((fl & pa_bit) && L < PBd) bdec = 1;
          else if (((fl & 4) && D <= P.pc_max_depth) || ((fl & 8) && nus >= P.n_unsat_min)) bdec = 0;
          if (bdec >= 0) {
            decimate_atomic(G, B, k, bdec);
            ++nagg;
            continue;
          }
        }
        if (P.rkq) continue;
        const int pk = ((int)G.vperm[k] << 16) | k;
        if (L < bL || (L == bL && pk < bk)) {
          bL = L;
          bk = pk;
        }
        if ((fl & 1) && (L < tL || (L == tL && pk < tk))) {
          tL = L;
          tk = pk;
        }
      }
      if (P.rkq) {
        g.sync();  // the aggressive decisions are visible
        ranker_select(P, G, B, g, bL, bk);
        if (bk != kNone) bL = B.acc[bk & 0xFFFF];  // f keeps the rule of Alg. 1: [L <= 0]
        nagg = g.sum_i(nagg);
        g.sync();
      } else {
        g.select_reduce(bL, bk, tL, tk, nagg);
      }
      int gsel, f;
      if (tk != kNone) {
        gsel = tk & 0xFFFF;
        f = 1;
      } else if (bk != kNone) {
        gsel = bk & 0xFFFF;
        f = bL <= 0.0f ? 1 : 0;
      } else {
        if (out.st && R == 0) out.st[D - 1] = StepTrace{-1, -1, 0, (int16_t)nagg, 0};
        status = BR_NOCAND;
        goto done;
      }
      if (P.dump && id == 0) {
        dump_candidates(P, G, B, g, out.shot, D, gsel);
        g.sync();
      }
      int v = f;
      if (split) {
        if (D == split) v = 1 - f;  // the one contrary decision of a side branch
      } else if (D <= P.k) {
        v = ((id >> (P.k - D)) & 1) ? 1 - f : f;  // b + (-1)^b f
      }
      if (R == 0) decimate_one(G, B, gsel, v);
      g.sync();
      const int np = peel(G, B, g);
      if (out.st && R == 0)
        out.st[D - 1] = StepTrace{(int16_t)G.vperm[gsel], (int8_t)v, 0, (int16_t)nagg, (int16_t)(np < 0 ? -1 : np)};
      if (np < 0) {
        status = np == -1 ? BR_CONTRADICTION : BR_INTERNAL;
        goto done;
      }
      if (D == d_reinit) {  // mu_{i->j} = Lambda_i again: the next pass reads the priors
        for (int k = R; k < ns; k += S)
          if (B.status[k] == -1) B.post[k] = G.llr[k];
        tw = 0;
        first = true;
        g.sync();
      }
    }
  }
done:
  // the estimate by ranked column (bit vperm[k] for label k)
  for (int x = R; x < (ns + 31) >> 5; x += S) out.ebits[x] = 0u;
  g.sync();
  for (int k = R; k < ns; k += S) {
    const int s8 = B.status[k];
    const int kr = G.vperm[k];
    if (s8 == 1 || (s8 == -1 && B.post[k] <= 0.0f)) atomicOr(&out.ebits[kr >> 5], 1u << (kr & 31));
    if (out.fstat) out.fstat[kr] = (int8_t)s8;
  }
  // The fallback key of a path that did not converge (the window's output
  // when no path converges is the least key, ties to the lowest id): rule 1
  // counts the unsatisfied checks of its estimate, rule 2 those among the
  // committed rows first (key = committed * (nr + 1) + all).  It takes the
  // place of the path metric, which only a converged path has.
  double fkey = CUDART_INF;
  if (status != BR_CONVERGED && P.fallback) {
    parity_pass(G, B, g);
    g.sync();
    long long nu = 0;
    for (int j = R; j < G.nr; j += S)
      if (bit_of(B.unsat, j)) nu += (P.fallback == 2 && G.cperm[j] < G.ncr) ? (long long)G.nr + 2 : 1;
    fkey = (double)g.sum_ll(nu);
  }
  // message reuse: what this path would leave the next window if it is the
  // window's output path (converged, path 0, or any path under a fallback
  // rule): the final posterior of each active column, +-clip for a decimated one
  if (out.keep && (status == BR_CONVERGED || id == 0 || P.fallback))
    for (int k = R; k < ns; k += S) {
      const int s8 = B.status[k];
      out.keep[k] = s8 == -1 ? B.post[k] : (s8 ? -P.clip : P.clip);
    }
  visits = g.sum_ll(visits);
  if (R == 0) {
    *out.status = status;
    *out.pm = status == BR_CONVERGED ? pm : fkey;
    if (out.btr) *out.btr = BranchTrace{status, depth, iters, 0, status == BR_CONVERGED ? pm : CUDART_INF};
    atomicAdd((unsigned long long*)out.visits, (unsigned long long)(visits + inherited));
    if (out.exec) atomicAdd((unsigned long long*)out.exec, (unsigned long long)visits);
    if (F.sched) atomicExch(&F.sched[id], (unsigned)PS_DONE);
  }
  g.sync();
  return -1;
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

struct DecodeArgs {
  KParams P;
  WinDev W;
  Layout L;
  const uint32_t* det;
  int det_words;
  long long n_shots;
  uint32_t* corr;
  int corr_words;
  int32_t* status_out;
  char* trace;
  size_t tr_bytes;
  int dmx, ns_max;
  int* work;            // shot mode: work counter
  long long* counters;  // [0] pre-BP edge-iterations, [1] GDG edge visits, [2] pre-BP converged,
                        // [3] GDG windows, [4] bulk staging waits that ran out
  char* path_res;       // path mode: results [shot][path]
  int* arrive;          // path mode: per-shot arrival counters (0 between launches)
  int sw_max;
  // windows too large for shared memory: the union region (pre-BP scratch and
  // path slots) of CTA b lives at uglob + b * ubytes in global memory
  // (L2-resident at these sizes) instead of after the persistent part
  char* uglob;
  size_t ubytes;
  // path mode: CTAs per shot (the paths, then idle CTAs up to a whole number
  // of clusters, which only help with the pre-BP)
  int cps;
  // executed GDG edge visits (nullable; counters[1] counts every path's
  // whole run, resumed prefixes included)
  long long* exec;
  ForkDev F;  // shot mode: snapshots of shared path prefixes
  // message reuse between windows (nullptr: off): keep[shot * keep_ld + c]
  // what the output path of this window ends with for window column c (NaN:
  // nothing), read by the next window through prev[c] (this window's column
  // -> the previous window's, -1: none; nullptr for the first window);
  // kpath[(slot * nb + path) * ns_max + label] each candidate path's values
  // (slot: the CTA in shot mode, the shot in path mode)
  float* keep;
  int keep_ld;
  const int16_t* prev;
  float* kpath;
};

// UG (a template parameter, so that shared-memory kernels keep shared-memory
// instructions for every union access): the region lives in global memory.
template <bool UG>
__device__ __forceinline__ char* union_base(const DecodeArgs& A, char* sm) {
  if (UG) return A.uglob + (size_t)blockIdx.x * A.ubytes;
  return sm + A.L.U;
}

// One window step of several decoders in one launch (kernel parameter).
struct BatchArgs {
  int n_seg;
  unsigned q_off;  // shared-memory offset of the launch's own work slot
  int* work;
  long long seg_end[kMaxBatch];  // cumulative shot counts
  DecodeArgs seg[kMaxBatch];
};

// Commit (Eq. (10)) + residue test (Eq. (11)) of one decoder's window.
struct CommitArgs {
  int n_commit;
  const int *cptr, *cdet;
  const uint32_t* cobs;
  int corr_words;
  const uint32_t* corr;
  long long n;
  uint32_t* det;
  int det_words;
  uint32_t *obs_pred, *resid;
  int b0, b1;
};
struct CommitBatch {
  int n_seg;
  long long seg_end[kMaxBatch];
  CommitArgs seg[kMaxBatch];
};

// ---- ascending sort of n = 2^m 64-bit keys in shared memory (all threads) ----
// A bitonic network.  Every stage of stride < 256 runs in registers: a warp
// holds a segment of 256 keys, lane L the keys L + 32 r (r < 8), so strides
// 32..128 pair two registers of a lane and strides 1..16 two lanes (shuffles).
// Strides >= 256 pass through shared memory, up to three stages per pass.
// Keys that differ sort the same under any correct network.
__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long v, int m) {
  const unsigned lo = __shfl_xor_sync(FULL, (unsigned)v, m), hi = __shfl_xor_sync(FULL, (unsigned)(v >> 32), m);
  return ((unsigned long long)hi << 32) | lo;
}

// stride 32 RJ: registers r and r | RJ of a lane
template <int RJ>
__device__ __forceinline__ void reg_stage(unsigned long long (&v)[8], int base, int lane, int kk) {
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if (!(r & RJ)) {
      const bool up = ((base + 32 * r + lane) & kk) == 0;
      const unsigned long long a = v[r], b = v[r | RJ];
      const bool sw = (a > b) == up;
      v[r] = sw ? b : a;
      v[r | RJ] = sw ? a : b;
    }
}

// the stages of block size kk with strides j0 >= j >= 1 (j0 < 256) of one
// register segment whose first key has global index base
__device__ __forceinline__ void seg_stages(unsigned long long (&v)[8], int base, int lane, int kk, int j0) {
  for (int j = j0; j > 0; j >>= 1) {
    if (j == 128) {
      reg_stage<4>(v, base, lane, kk);
    } else if (j == 64) {
      reg_stage<2>(v, base, lane, kk);
    } else if (j == 32) {
      reg_stage<1>(v, base, lane, kk);
    } else {
      const bool low = (lane & j) == 0;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const unsigned long long o = shfl_u64(v[r], j);
        const bool up = ((base + 32 * r + lane) & kk) == 0;
        const bool keep_min = low == up;
        v[r] = keep_min ? (o < v[r] ? o : v[r]) : (o > v[r] ? o : v[r]);
      }
    }
  }
}

// M stages of strides j, j/2, ..., j/2^(M-1) (all >= 256) through shared memory
template <int M>
__device__ __forceinline__ void smem_stages(unsigned long long* s, int n, int kk, int j) {
  const int b1 = __ffs(j) - 1;
  for (int g = threadIdx.x; g < (n >> M); g += blockDim.x) {
    int base = g;
#pragma unroll
    for (int q = M - 1; q >= 0; --q) {  // zero bits at b1-M+1 .. b1, lowest first
      const int b = b1 - q;
      base = ((base >> b) << (b + 1)) | (base & ((1 << b) - 1));
    }
    const bool up = (base & kk) == 0;
    unsigned long long v[1 << M];
#pragma unroll
    for (int t = 0; t < (1 << M); ++t) {
      int off = 0;
#pragma unroll
      for (int l = 0; l < M; ++l) off += ((t >> l) & 1) * (j >> (M - 1 - l));
      v[t] = s[base + off];
    }
#pragma unroll
    for (int l = M - 1; l >= 0; --l)  // bit l of t <-> stride j >> (M - 1 - l), largest first
#pragma unroll
      for (int t = 0; t < (1 << M); ++t)
        if (!((t >> l) & 1)) {
          const unsigned long long a = v[t], b = v[t | (1 << l)];
          const bool sw = (a > b) == up;
          v[t] = sw ? b : a;
          v[t | (1 << l)] = sw ? a : b;
        }
#pragma unroll
    for (int t = 0; t < (1 << M); ++t) {
      int off = 0;
#pragma unroll
      for (int l = 0; l < M; ++l) off += ((t >> l) & 1) * (j >> (M - 1 - l));
      s[base + off] = v[t];
    }
  }
}

// Call with every thread; s holds n keys (n a power of two); returns after a barrier.
__device__ void block_sort_u64(unsigned long long* s, int n) {
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = NT >> 5;
  if (n < 256) {  // tiny windows: the plain network
    for (int kk = 2; kk <= n; kk <<= 1)
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int i = tid; i < n; i += NT) {
          const int ixj = i ^ jj;
          if (ixj > i) {
            const unsigned long long a = s[i], b = s[ixj];
            if ((a > b) == ((i & kk) == 0)) {
              s[i] = b;
              s[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    return;
  }
  // every block size up to 256 inside the segments
  for (int sg = warp; sg < (n >> 8); sg += nw) {
    const int base = sg << 8;
    unsigned long long v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = s[base + 32 * r + lane];
    for (int kk = 2; kk <= 256; kk <<= 1) seg_stages(v, base, lane, kk, kk >> 1);
#pragma unroll
    for (int r = 0; r < 8; ++r) s[base + 32 * r + lane] = v[r];
  }
  __syncthreads();
  for (int kk = 512; kk <= n; kk <<= 1) {
    int j = kk >> 1;
    for (; j >= 256 * 4; j >>= 3) {  // three stages, all of stride >= 256
      smem_stages<3>(s, n, kk, j);
      __syncthreads();
    }
    if (j >= 512) {
      smem_stages<2>(s, n, kk, j);
      __syncthreads();
    } else if (j == 256) {
      smem_stages<1>(s, n, kk, j);
      __syncthreads();
    }
    for (int sg = warp; sg < (n >> 8); sg += nw) {
      const int base = sg << 8;
      unsigned long long v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = s[base + 32 * r + lane];
      seg_stages(v, base, lane, kk, 128);
#pragma unroll
      for (int r = 0; r < 8; ++r) s[base + 32 * r + lane] = v[r];
    }
    __syncthreads();
  }
}

// ---- thread-block clusters: distributed shared memory ----
__device__ __forceinline__ unsigned cl_size() {
  unsigned n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; orders the shared-memory writes
// before it with the reads (local or remote) after it
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the address of `p` (a shared-memory location of this CTA) in CTA `rank`
__device__ __forceinline__ unsigned cl_map(const void* p, unsigned rank) {
  unsigned a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
  return a;
}
__device__ __forceinline__ float cl_ld_f32(unsigned a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t cl_ld_u32(unsigned a) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t cl_ld_u8(unsigned a) {
  uint16_t v;
  asm volatile("ld.shared::cluster.u8 %0, [%1];" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void cl_st_f32(unsigned a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void cl_st_u32(unsigned a, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ CNState cl_ld_cns(unsigned a) {
  CNState c;
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=f"(c.m1), "=f"(c.m2), "=r"(c.ac), "=r"(c.pad)
               : "r"(a));
  return c;
}

// a2 split over the CTAs of a cluster (path mode, one cluster per shot): CTA
// r owns the r-th slice of the checks and of the variables, runs the check
// pass of Eq. (1) for its checks and the variable pass of Eq. (2)-(3) for its
// variables.  A remote load costs a round trip of ~1200 cycles (a cluster
// barrier ~470), so values travel the cheap way: each CTA pushes its
// posteriors (and ranking keys) and its "unsatisfied" flag into every CTA's
// shared memory before the barrier that ends the pass, and the check pass
// reads them locally; the variable pass requests a variable's check states
// and signs from their owners in one round trip.  Two cluster barriers per
// iteration separate the passes, so every value read was written in the pass
// before, and after the last one no CTA touches another's shared memory.
// The arithmetic of every message and posterior is that of the single-CTA
// loop; at the end every CTA holds the whole posterior and key.  Returns t as
// the loop leaves it; conv and t_conv as in the caller.
template <bool LW>
__device__ int prebp_cluster(const DecodeArgs& A, const WinDev& W, const WinDev& Wg, char* sm, char* U,
                             const uint32_t* sbits, bool& conv, int& t_conv) {
  const KParams& P = A.P;
  const Layout& L = A.L;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31;
  const int nr = W.n_rows, nc = W.n_cols;
  const unsigned C = cl_size(), r = cl_rank();
  float* post = (float*)(U + L.p_post);
  float* key = (float*)(U + L.p_key);
  CNState* cns = (CNState*)(U + L.p_cns);
  uint8_t* sign = (uint8_t*)(U + L.p_sign);
  // flags[8 * parity + c]: CTA c found an unsatisfied check (in the reduction
  // scratch of the path phase, idle until the pre-BP ends)
  int* flags = (int*)(sm + L.red);
  // slices; the owner of check j is floor(j / sc) = umulhi(j, ceil(2^32 / sc)), exact for j, sc < 2^16
  const int sc = (nr + (int)C - 1) / (int)C, sv = (nc + (int)C - 1) / (int)C;
  const unsigned mc = (unsigned)((0x100000000ull + sc - 1) / sc);
  const int jb = min(nr, (int)r * sc), je = min(nr, jb + sc);
  const int ib = min(nc, (int)r * sv), ie = min(nc, ib + sv);
  const int tpc = lanes_per_check(NT, max(1, je - jb)), sub = tid & (tpc - 1);
  const int nrr = (je - jb + NT / tpc - 1) / (NT / tpc) * (NT / tpc);
  const int tk0 = P.n_pre - 3 > 1 ? P.n_pre - 3 : 1;
  int t;
  for (t = 1; t <= P.n_pre; ++t) {
    bool unsat = false;
    for (int j0 = tid / tpc; j0 < nrr; j0 += NT / tpc) {
      const bool real = jb + j0 < je;
      const int j = real ? jb + j0 : je - 1;
      const int beg = Wg.row_ptr[j], end = real ? Wg.row_ptr[j + 1] : beg;
      const CNState oc = cns[j];
      float m1 = CUDART_INF_F, m2 = CUDART_INF_F;
      int am = 0xFFFF;
      uint32_t neg = 0, hp = 0;
      for (int q = beg + 4 * sub; q < end; q += 4 * tpc) {
        uint32_t ent[4];
        float pv[4];
        uint32_t sg[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ent[u] = (q + u < end) ? Wg.row_ent[q + u] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned i = ent[u] >> 16, e = ent[u] & 0xFFFFu;
          pv[u] = 0.0f;
          sg[u] = 0u;
          if (q + u < end) {
            pv[u] = post[i];  // t = 1: the first VN->CN message (the prior, or the value kept for the column)
            sg[u] = sign[e];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (q + u >= end) break;
          const int e = (int)(ent[u] & 0xFFFFu);
          hp ^= pv[u] <= 0.0f;
          const float wprev = (LW && t > 1) ? edge_weight(W.wts, W.wT, W.n_edges, P.alpha, t - 1, e) : P.alpha;
          const float v = (t == 1) ? pv[u] : clipf(__fsub_rn(pv[u], c2v<LW>(wprev, P.clip, oc, e, sg[u])), P.clip);
          const float a = fabsf(v);
          am = a < m1 ? e : am;
          m2 = fminf(m2, fmaxf(m1, a));
          m1 = fminf(m1, a);
          const uint32_t sgn = v < 0.0f;
          neg ^= sgn;
          sign[e] = (uint8_t)sgn;
        }
      }
      if (tpc > 1) {
        group_min2(m1, m2, am, neg, tpc);
        for (int off = tpc >> 1; off; off >>= 1) hp ^= __shfl_xor_sync(FULL, hp, off);
      }
      if (sub == 0 && real) {
        cns[j] = cn_store<LW>(P.alpha, P.clip, m1, m2, am, neg ^ bit_of(sbits, j), end - beg == 1, 0u);
        unsat |= (hp ^ bit_of(sbits, j)) != 0u;
      }
    }
    const int lu = __syncthreads_or(unsat);
    if (tid < (int)C) cl_st_u32(cl_map(&flags[8 * (t & 1) + (int)r], (unsigned)tid), (uint32_t)lu);
    cl_sync();  // check states, signs and flags of pass t
    const bool any = __any_sync(FULL, lane < (int)C && flags[8 * (t & 1) + lane] != 0);
    if (!any && t >= 2) {  // iteration t-1 satisfies H e = s in every slice
      conv = true;
      t_conv = t - 1;
      break;
    }
    const bool kacc = t >= tk0;
    for (int i = ib + tid; i < ie; i += NT) {
      float p = Wg.llr[i];
      const int eb = Wg.col_ptr[i], ee = Wg.col_ptr[i + 1];
      // up to six messages requested at once (the column degree of these
      // windows), then added in ascending check order (Eq. (2))
      for (int e0 = eb; e0 < ee; e0 += 6) {
        CNState c[6];
        uint32_t sg[6];
#pragma unroll
        for (int u = 0; u < 6; ++u)
          if (e0 + u < ee) {
            const unsigned j = Wg.col_rows[e0 + u], o = __umulhi(j, mc);
            c[u] = cl_ld_cns(cl_map(&cns[j], o));
            sg[u] = cl_ld_u8(cl_map(&sign[e0 + u], o));
          }
#pragma unroll
        for (int u = 0; u < 6; ++u)
          if (e0 + u < ee) {
            const float wt = LW ? edge_weight(W.wts, W.wT, W.n_edges, P.alpha, t, e0 + u) : P.alpha;
            p = __fadd_rn(p, c2v<LW>(wt, P.clip, c[u], e0 + u, sg[u]));
          }
      }
      post[i] = p;
      for (unsigned c = 0; c < C; ++c)  // every CTA reads the whole posterior in its check pass
        if (c != r) cl_st_f32(cl_map(&post[i], c), p);
      if (kacc) {
        float kv;
        if (t == tk0) {
          if (P.n_pre < 4) {
            const float li = Wg.llr[i];
            float s = li;
            for (int q = 1; q < 4 - P.n_pre; ++q) s = __fadd_rn(s, li);
            kv = __fadd_rn(s, p);
          } else {
            kv = p;
          }
        } else {
          kv = __fadd_rn(key[i], p);
        }
        key[i] = kv;
        for (unsigned c = 0; c < C; ++c)
          if (c != r) cl_st_f32(cl_map(&key[i], c), kv);
      }
    }
    cl_sync();  // posteriors (and keys) of pass t, in every CTA
  }
  // every CTA holds the whole posterior and key: the last variable pass
  // pushed them before the barrier that ended the loop, and no CTA touches
  // another's shared memory after it
  return t;
}

// a1 + a2 (+ a3 when not converged): the shared prefix of both launch shapes.
// Returns true when the pre-BP converged (cbits then hold its decision).
template <bool LW, bool WIDE, bool UG>
__device__ bool window_prefix(const DecodeArgs& A, const WinDev& W, char* sm, long long shot, int* t_run_out,
                              Stager& stg) {
  const KParams& P = A.P;
  const Layout& L = A.L;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nr = W.n_rows, nc = W.n_cols;
  uint32_t* sbits = (uint32_t*)(sm + L.sbits);
  uint32_t* cbits = (uint32_t*)(sm + L.cbits);
  uint16_t* sel = (uint16_t*)(sm + L.sel);
  char* U = union_base<UG>(A, sm);
  float* post = (float*)(U + L.p_post);
  float* key = (float*)(U + L.p_key);
  CNState* cns = (CNState*)(U + L.p_cns);
  uint8_t* sign = (uint8_t*)(U + L.p_sign);
  uint32_t* parb = (uint32_t*)(U + L.p_par);
  unsigned long long* sortb = (unsigned long long*)(U + L.p_sort);

  // ---- a1: window syndrome ----
  const uint32_t* dp = A.det + (size_t)shot * A.det_words;
  for (int x = tid; x < L.rw; x += NT) {
    const int b0 = W.row0 + 32 * x;
    const uint32_t lo = dp[b0 >> 5];
    const uint32_t hi = ((b0 >> 5) + 1 < A.det_words) ? dp[(b0 >> 5) + 1] : 0u;
    const int sh = b0 & 31;
    uint32_t v = sh ? ((lo >> sh) | (hi << (32 - sh))) : lo;
    const int rem = nr - 32 * x;
    if (rem < 32) v &= (1u << rem) - 1u;
    sbits[x] = v;
  }
  for (int x = tid; x < L.cw; x += NT) cbits[x] = 0;
  __syncthreads();

  // the window graph in shared memory for the pre-BP loop when the union
  // region has room (shot mode); the ranking and shortening below read W
  WinDev Wg = W;
  if (L.pre_stage) {
    uint16_t* cp = (uint16_t*)(U + L.q_colptr);
    uint16_t* cr = (uint16_t*)(U + L.q_colrows);
    uint16_t* rp = (uint16_t*)(U + L.q_rowptr);
    uint32_t* re = (uint32_t*)(U + L.q_rowent);
    float* ll = (float*)(U + L.q_llr);
    uint16_t* vp = (uint16_t*)(U + L.q_vperm);
    const StagePiece pc[6] = {{cp, W.col_ptr, al16(2u * (nc + 1))},       {cr, W.col_rows, al16(2u * W.n_edges)},
                              {rp, W.row_ptr, al16(2u * (nr + 1))},       {re, W.row_ent, al16(4u * W.n_edges)},
                              {ll, W.llr, al16(4u * nc)},                 {vp, W.vperm, al16(2u * nc)}};
    stage_pieces(stg, pc, 6);
    Wg.col_ptr = cp;
    Wg.col_rows = cr;
    Wg.row_ptr = rp;
    Wg.row_ent = re;
    Wg.llr = ll;
    Wg.vperm = vp;
  }

  // ---- a2: pre-BP on the full window ----
  const int tpc_pre = WIDE ? lanes_per_check(NT, nr) : 1, sub_pre = tid & (tpc_pre - 1);
  const int nr_rounds = (nr + NT / tpc_pre - 1) / (NT / tpc_pre) * (NT / tpc_pre);
  bool conv = false;
  int t = 0;
  const int tk0 = P.n_pre - 3 > 1 ? P.n_pre - 3 : 1;
  if (P.n_pre == 0) {
    uint32_t* pb = parb;
    for (int x = tid; x < L.rw; x += NT) pb[x] = 0;
    __syncthreads();
    for (int i = tid; i < nc; i += NT) {
      const float li = Wg.llr[i];
      post[i] = li;
      key[i] = __fadd_rn(__fadd_rn(__fadd_rn(li, li), li), li);
      if (li <= 0.0f)
        for (int e = Wg.col_ptr[i]; e < Wg.col_ptr[i + 1]; ++e) {
          const int j = Wg.col_rows[e];
          atomicXor(&pb[j >> 5], 1u << (j & 31));
        }
    }
    __syncthreads();
    bool ok = true;
    for (int x = 0; x < L.rw; ++x) ok &= (pb[x] == sbits[x]);
    conv = ok;
  }
  if (P.n_pre > 0) {
    // the first VN->CN messages of the pre-BP: the prior, or (message reuse)
    // what the previous window's output path kept for the same DEM column
    const float* kept = (A.keep && A.prev) ? A.keep + (size_t)shot * A.keep_ld : nullptr;
    for (int i = tid; i < nc; i += NT) {
      float v = Wg.llr[i];
      if (kept) {
        const int pc = A.prev[i];
        if (pc >= 0) {
          const float x = kept[pc];
          if (x == x) v = x;
        }
      }
      post[i] = v;
    }
    __syncthreads();
  }
  int t_conv = 0;
  if (WIDE && !UG && P.n_pre > 0 && cl_size() > 1 && nr >= 2 * (int)cl_size() && nc >= 2 * (int)cl_size()) {
    t = prebp_cluster<LW>(A, W, Wg, sm, U, sbits, conv, t_conv);
  } else {
  for (t = 1; t <= P.n_pre; ++t) {
    // check nodes; each check also takes the parity of the hard decisions it
    // reads, so for t >= 2 the pass is the convergence test of iteration t-1
    bool unsat = false;
    for (int j0 = tid / tpc_pre; j0 < nr_rounds; j0 += NT / tpc_pre) {
      const int j = j0 < nr ? j0 : nr - 1;
      const int beg = Wg.row_ptr[j], end = j0 < nr ? Wg.row_ptr[j + 1] : beg;
      const CNState oc = cns[j];
      float m1 = CUDART_INF_F, m2 = CUDART_INF_F;
      int am = 0xFFFF;
      uint32_t neg = 0, hp = 0;
      for (int q = beg + 4 * sub_pre; q < end; q += 4 * tpc_pre) {
        uint32_t ent[4];
        float pv[4];
        uint32_t sg[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ent[u] = (q + u < end) ? Wg.row_ent[q + u] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = (int)(ent[u] >> 16), e = (int)(ent[u] & 0xFFFFu);
          pv[u] = post[i];  // t = 1: the first VN->CN message (the prior, or the value kept for the column)
          sg[u] = sign[e];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (q + u >= end) break;
          const int e = (int)(ent[u] & 0xFFFFu);
          hp ^= pv[u] <= 0.0f;
          const float wprev = (LW && t > 1) ? edge_weight(W.wts, W.wT, W.n_edges, P.alpha, t - 1, e) : P.alpha;
          const float v = (t == 1) ? pv[u] : clipf(__fsub_rn(pv[u], c2v<LW>(wprev, P.clip, oc, e, sg[u])), P.clip);
          const float a = fabsf(v);
          am = a < m1 ? e : am;
          m2 = fminf(m2, fmaxf(m1, a));
          m1 = fminf(m1, a);
          const uint32_t sgn = v < 0.0f;
          neg ^= sgn;
          sign[e] = (uint8_t)sgn;
        }
      }
      if (tpc_pre > 1) {
        group_min2(m1, m2, am, neg, tpc_pre);
        for (int off = tpc_pre >> 1; off; off >>= 1) hp ^= __shfl_xor_sync(FULL, hp, off);
      }
      if (sub_pre == 0 && j0 < nr) {
        cns[j] = cn_store<LW>(P.alpha, P.clip, m1, m2, am, neg ^ bit_of(sbits, j), end - beg == 1, 0u);
        unsat |= (hp ^ bit_of(sbits, j)) != 0u;
      }
    }
    if (!__syncthreads_or(unsat) && t >= 2) {  // iteration t-1 satisfies H e = s
      conv = true;
      t_conv = t - 1;
      break;
    }
    const bool kacc = t >= tk0;
    for (int i0 = tid; i0 < nc; i0 += NT) {
      const int i = Wg.vperm[i0];  // descending degree: the lanes of a round loop alike
      float p = Wg.llr[i];
      const int eb = Wg.col_ptr[i], ee = Wg.col_ptr[i + 1];
      // up to six messages requested at once, then added in ascending check
      // order (Eq. (2))
      for (int e0 = eb; e0 < ee; e0 += 6) {
        CNState c[6];
        uint32_t sg[6];
#pragma unroll
        for (int u = 0; u < 6; ++u)
          if (e0 + u < ee) {
            c[u] = cns[Wg.col_rows[e0 + u]];
            sg[u] = sign[e0 + u];
          }
#pragma unroll
        for (int u = 0; u < 6; ++u)
          if (e0 + u < ee) {
            const float wt = LW ? edge_weight(W.wts, W.wT, W.n_edges, P.alpha, t, e0 + u) : P.alpha;
            p = __fadd_rn(p, c2v<LW>(wt, P.clip, c[u], e0 + u, sg[u]));
          }
      }
      post[i] = p;
      if (kacc) {
        float kv;
        if (t == tk0) {
          if (P.n_pre < 4) {
            const float li = Wg.llr[i];
            float s = li;
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
    }
    __syncthreads();
  }
  }
  if (!conv && P.n_pre > 0) {  // the convergence test of the last iteration
    bool unsat = false;
    for (int j = tid; j < nr; j += NT) {
      uint32_t hp = bit_of(sbits, j);
      for (int q = Wg.row_ptr[j]; q < Wg.row_ptr[j + 1]; ++q) hp ^= post[Wg.row_ent[q] >> 16] <= 0.0f;
      unsat |= hp != 0u;
    }
    if (!__syncthreads_or(unsat)) {
      conv = true;
      t_conv = P.n_pre;
    }
  }
  if (conv && P.n_pre > 0) t = t_conv;
  *t_run_out = conv ? (P.n_pre == 0 ? 0 : t) : P.n_pre;
  if (conv) {
    for (int base = warp * 32; base < nc; base += NT) {
      const int i = base + lane;
      const bool one = i < nc && post[i] <= 0.0f;
      const unsigned m = __ballot_sync(FULL, one);
      if (lane == 0) cbits[base >> 5] = m;
    }
    __syncthreads();
    return true;
  }

  // ---- a3: rank by the four-iteration sum, keep the first n_short ----
  const int n_short = W.n_short;
  for (int i = tid; i < L.sortn; i += NT)
    sortb[i] = i < nc ? (((unsigned long long)ordkey(key[i]) << 32) | (unsigned)i) : ~0ull;
  __syncthreads();
  block_sort_u64(sortb, L.sortn);
  for (int k = tid; k < n_short; k += NT) sel[k] = (uint16_t)(sortb[k] & 0xFFFFu);
  __syncthreads();
  // ---- shortened matrix in shared memory, numbered in processing order ----
  // Columns and checks get labels by descending degree (ties by rank / row),
  // so the lanes of a round loop alike and touch neighbouring words; vperm
  // and cperm map a label back to the ranked column and the window row, which
  // decide every tie.  A column's checks stay in ascending window row (the
  // order of the sum of Eq. (2)).
  uint16_t* scp = (uint16_t*)(sm + L.s_colptr);
  uint16_t* scr = (uint16_t*)(sm + L.s_colrows);
  uint16_t* srp = (uint16_t*)(sm + L.s_rowptr);
  uint32_t* sre = (uint32_t*)(sm + L.s_rowent);
  float* sllr = (float*)(sm + L.s_llr);
  uint8_t* svd = (uint8_t*)(sm + L.s_vdeg);
  uint16_t* sef = (uint16_t*)(sm + L.s_efull);
  uint16_t* cperm = (uint16_t*)(sm + L.s_cperm);
  uint16_t* vperm = (uint16_t*)(sm + L.s_vperm);
  int* rc = (int*)(sm + L.rowcnt);
  int* tmp = (int*)sortb;  // the sort buffer is free now
  for (int k = tid; k < n_short; k += NT) {
    const int c = sel[k];
    tmp[k] = W.col_ptr[c + 1] - W.col_ptr[c];
  }
  for (int j = tid; j <= nr; j += NT) rc[j] = 0;
  __syncthreads();
  for (int k = tid; k < n_short; k += NT) {  // rows of the shortened matrix
    const int c = sel[k];
    for (int e = W.col_ptr[c]; e < W.col_ptr[c + 1]; ++e) atomicAdd(&rc[W.col_rows[e]], 1);
  }
  for (int k = tid; k < n_short; k += NT) {  // rank by counting; no sort needed at these sizes
    const int dk = tmp[k];
    int r = 0;
    for (int i = 0; i < n_short; ++i) {
      const int di = tmp[i];
      r += (di > dk) || (di == dk && i < k);
    }
    vperm[r] = (uint16_t)k;
  }
  __syncthreads();
  uint16_t* cinv = srp;  // window row -> label, until the row pointers are built
  for (int j = tid; j < nr; j += NT) {
    const int dj = rc[j];
    int r = 0;
    for (int i = 0; i < nr; ++i) {
      const int di = rc[i];
      r += (di > dj) || (di == dj && i < j);
    }
    cperm[r] = (uint16_t)j;
    cinv[j] = (uint16_t)r;
  }
  for (int k = tid; k < n_short; k += NT) {
    const int kr = vperm[k];
    svd[k] = (uint8_t)tmp[kr];
    sllr[k] = W.llr[sel[kr]];
  }
  __syncthreads();
  for (int k = tid; k < n_short; k += NT) tmp[k] = svd[k];
  __syncthreads();
  if (warp == 0) {
    const int tot = warp_scan_excl(tmp, n_short, lane);
    if (lane == 0) tmp[n_short] = tot;
  }
  __syncthreads();
  for (int k = tid; k <= n_short; k += NT) scp[k] = (uint16_t)tmp[k];
  for (int k = tid; k < n_short; k += NT) {
    const int c = sel[vperm[k]];
    int o = tmp[k];
    for (int e = W.col_ptr[c]; e < W.col_ptr[c + 1]; ++e, ++o) {
      scr[o] = cinv[W.col_rows[e]];
      if (LW) sef[o] = (uint16_t)e;  // the shortened edge keeps its full-window edge's weights
    }
  }
  for (int j = tid; j <= nr; j += NT) rc[j] = 0;
  __syncthreads();
  for (int k = tid; k < n_short; k += NT)
    for (int e = scp[k]; e < scp[k + 1]; ++e) atomicAdd(&rc[scr[e]], 1);
  __syncthreads();
  if (warp == 0) {
    const int tot = warp_scan_excl(rc, nr, lane);
    if (lane == 0) rc[nr] = tot;
  }
  __syncthreads();
  for (int j = tid; j <= nr; j += NT) srp[j] = (uint16_t)rc[j];
  __syncthreads();
  for (int k = tid; k < n_short; k += NT)
    for (int e = scp[k]; e < scp[k + 1]; ++e) {
      const int pos = atomicAdd(&rc[scr[e]], 1);
      sre[pos] = (uint32_t)e | ((uint32_t)k << 16);
    }
  __syncthreads();
  return false;
}

__device__ __forceinline__ ShortG short_graph(char* sm, const Layout& L, const WinDev& W, int ns) {
  return ShortG{W.n_rows, ns, L.rw,
                (const uint16_t*)(sm + L.s_colptr), (const uint16_t*)(sm + L.s_colrows),
                (const uint16_t*)(sm + L.s_rowptr), (const uint32_t*)(sm + L.s_rowent),
                (const float*)(sm + L.s_llr),       (const uint8_t*)(sm + L.s_vdeg),
                (const uint32_t*)(sm + L.sbits),    (const uint16_t*)(sm + L.s_efull),
                W.wts, W.wT, W.n_edges, W.rows_per_block, (const uint16_t*)(sm + L.sel),
                (const uint16_t*)(sm + L.s_cperm), (const uint16_t*)(sm + L.s_vperm), W.n_commit_rows};
}

__device__ __forceinline__ PathOut trace_out(const DecodeArgs& A, char* tr, int id, long long shot) {
  PathOut o{};
  if (tr) {
    o.btr = (BranchTrace*)(tr + trace_off_br()) + id;
    o.st = (StepTrace*)(tr + trace_off_st(A.P.nb)) + (size_t)id * A.dmx;
    o.fstat = (int8_t*)(tr + trace_off_fs(A.P.nb, A.dmx)) + (size_t)id * A.ns_max;
  }
  o.visits = &A.counters[1];
  o.exec = A.exec;
  o.shot = shot;
  return o;
}

// The output path of a window in which no path converged: path 0, or under a
// fallback rule the least fallback key (stored in the path-metric slot of an
// unconverged path), ties to the lowest id.
__device__ __forceinline__ int fallback_path(const KParams& P, const double* pm) {
  int fb = 0;
  if (P.fallback)
    for (int id = 1; id < P.nb; ++id)
      if (pm[id] < pm[fb]) fb = id;
  return fb;
}

__device__ void write_outputs(const DecodeArgs& A, char* sm, long long shot, bool conv, int winner,
                              int n_short, int t_run, char* tr) {
  const Layout& L = A.L;
  const int tid = threadIdx.x, NT = blockDim.x;
  const uint32_t* cbits = (const uint32_t*)(sm + L.cbits);
  uint32_t* co = A.corr + (size_t)shot * A.corr_words;
  for (int x = tid; x < A.corr_words; x += NT) co[x] = x < L.cw ? cbits[x] : 0u;
  if (tr && !conv)
    for (int k = tid; k < n_short; k += NT)
      ((uint16_t*)(tr + trace_off_sel(A.P.nb, A.dmx, A.ns_max)))[k] = ((const uint16_t*)(sm + L.sel))[k];
  if (tid == 0) {
    if (A.status_out) A.status_out[shot] = conv ? -1 : (winner >= 0 ? winner : -2);
    if (tr) {
      int32_t* h = (int32_t*)tr;
      h[0] = conv ? 1 : 0;
      h[1] = conv ? -1 : winner;
      h[2] = conv ? 0 : n_short;
      h[3] = t_run;
    }
    atomicAdd((unsigned long long*)&A.counters[0], (unsigned long long)t_run * A.W.n_edges);
    atomicAdd((unsigned long long*)&A.counters[conv ? 2 : 3], 1ull);
  }
}

// Message reuse: the values this window leaves the next one, per window
// column (all threads of the CTA).  kp = the output path's values by label;
// kp = nullptr: the pre-BP converged, and its posterior `post` (still in the
// union region's pre-BP scratch) is kept for every column.
__device__ void keep_for_next(const DecodeArgs& A, char* sm, long long shot, const float* kp, int n_short,
                              const float* post = nullptr) {
  const int tid = threadIdx.x, NT = blockDim.x, nc = A.W.n_cols;
  float* out = A.keep + (size_t)shot * A.keep_ld;
  if (!kp) {
    for (int c = tid; c < nc; c += NT) out[c] = post[c];
    return;
  }
  const uint16_t* sel = (const uint16_t*)(sm + A.L.sel);
  const uint16_t* vperm = (const uint16_t*)(sm + A.L.s_vperm);
  for (int c = tid; c < nc; c += NT) out[c] = CUDART_NAN_F;
  __syncthreads();
  for (int k = tid; k < n_short; k += NT) out[sel[vperm[k]]] = __ldcg(kp + k);
}

// ---- shot mode: persistent CTAs of up to 8 warps, one warp per decision path ----
// One shot of one window by the whole CTA (every thread calls).  misc[2], the
// decision-path queue, must be 0 on entry.
template <bool LW, bool UG>
__device__ void shot_body(const DecodeArgs& A, long long shot, char* sm, Stager& stg) {
  const Layout& L = A.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int* misc = (int*)(sm + L.misc);
  int* res_status = (int*)(sm + L.res_status);
  double* res_pm = (double*)(sm + L.res_pm);
  uint32_t* res_e = (uint32_t*)(sm + L.res_ebits);
  uint32_t* cbits = (uint32_t*)(sm + L.cbits);
  const uint16_t* sel = (const uint16_t*)(sm + L.sel);
  char* tr = A.trace ? A.trace + (size_t)shot * A.tr_bytes : nullptr;
  int t_run = 0;
  const bool conv = window_prefix<LW, false, UG>(A, A.W, sm, shot, &t_run, stg);
  int winner = -1;
  const int n_short = conv ? 0 : A.W.n_short;
  if (!conv) {
    // warps beyond the layout's path slots (batched launches) sit out the paths
    if (warp < L.nslots) {
      const ShortG G = short_graph(sm, L, A.W, n_short);
      char* slot = union_base<UG>(A, sm) + (size_t)warp * L.b_size;
      const Slot B = make_slot(slot, L);
      const WarpGrp g{lane};
      // snapshots of shared prefixes, when planned and this CTA has a pool
      // shared prefixes and preemption, when planned and this CTA has a pool
      const bool fork = A.F.pool && (int)blockIdx.x < A.F.pool_ctas;
      const int nb = A.P.nb;
      ForkCtx F{};
      F.flags = (int*)(sm + L.red);
      F.pool = fork ? A.F.pool + (size_t)blockIdx.x * A.F.cta_bytes : nullptr;
      F.stride = kSnapHeader + L.b_size;
      F.slot = slot;
      F.slot_bytes = L.b_size;
      F.st0 = tr ? (const StepTrace*)(tr + trace_off_st(nb)) : nullptr;
      F.sched = (fork && A.F.sched) ? (unsigned*)(sm + L.red) + kMaxForkNodes : nullptr;
      F.fnode = A.F.fnode;
      F.fdep = A.F.fdep;
      F.n_nodes = A.F.n_nodes;
      int next = -1;  // the path taken at a preemption point
      unsigned next_w = 0;
      while (true) {
        int id = -1;
        unsigned w0 = PS_QUEUED;  // the taken path's state word: queued or parked after step D
        if (next >= 0) {
          id = next;
          w0 = next_w;
          next = -1;
        } else {
          while (true) {  // the next queued path that no preemption took
            int pos = 0;
            if (lane == 0) pos = atomicAdd(&misc[2], 1);
            pos = __shfl_sync(FULL, pos, 0);
            if (pos >= nb) break;
            const int cand = fork ? (int)A.F.order[pos] : path_at(A.P, pos);
            int ok = 1;
            if (F.sched && lane == 0) ok = atomicCAS(&F.sched[cand], (unsigned)PS_QUEUED, (unsigned)PS_RUNNING) == PS_QUEUED;
            if (__shfl_sync(FULL, ok, 0)) {
              id = cand;
              break;
            }
          }
          if (id < 0 && F.sched) {  // a parked path, the one with the most steps left
            int c = -1;
            unsigned cw = 0;
            if (lane == 0)
              for (int tries = 0; tries < 4 * nb; ++tries) {
                c = -1;
                int best = 0;
                for (int p = 0; p < nb; ++p) {
                  const unsigned w = *(volatile unsigned*)&F.sched[p];
                  if ((w & 3u) != PS_PARKED) continue;
                  const int rem = path_dmax(A.P, p, path_split(A.P, p)) - (int)(w >> 8) + 1;
                  if (rem > best) {
                    best = rem;
                    c = p;
                    cw = w;
                  }
                }
                if (c < 0 || atomicCAS(&F.sched[c], cw, (unsigned)PS_RUNNING) == cw) break;
                c = -1;
              }
            c = __shfl_sync(FULL, c, 0);
            cw = __shfl_sync(FULL, cw, 0);
            if (c >= 0) {
              id = c;
              w0 = cw;
            }
          }
          if (id < 0) break;
        }
        PathOut o = trace_out(A, tr, id, shot);
        o.status = &res_status[id];
        o.pm = &res_pm[id];
        o.ebits = res_e + (size_t)id * L.sw;
        if (A.keep) o.keep = A.kpath + ((size_t)blockIdx.x * nb + id) * A.ns_max;
        F.chain = (fork && F.n_nodes > 0) ? A.F.chain + (size_t)id * A.dmx : nullptr;
        F.src = nullptr;
        if ((w0 & 3u) == PS_PARKED) {  // its own parking snapshot
          __threadfence();
          F.src = F.pool + (size_t)(F.n_nodes + id) * F.stride;
        } else if (F.chain) {  // the deepest ready snapshot on this path's chain
          int node = -1;
          if (lane == 0) {
            const int dm = path_dmax(A.P, id, path_split(A.P, id));
            for (int D = dm; D >= 1 && node < 0; --D) {
              const int n = F.chain[D - 1];
              if (n >= 0 && *(volatile int*)&F.flags[n] == 2) node = n;
            }
          }
          node = __shfl_sync(FULL, node, 0);
          if (node >= 0) {
            __threadfence();  // the snapshot's contents after its flag
            F.src = F.pool + (size_t)node * F.stride;
          }
        }
        next = run_path<LW>(A.P, G, B, id, g, o, A.dmx, F, &next_w);
      }
    }
    __syncthreads();
    // ---- a8: least path metric, ties to the lowest id ----
    if (tid == 0) {
      int best = -1;
      double bp = CUDART_INF;
      for (int id = 0; id < A.P.nb; ++id)
        if (res_status[id] == BR_CONVERGED && res_pm[id] < bp) {
          bp = res_pm[id];
          best = id;
        }
      misc[1] = best;
      misc[4] = best >= 0 ? best : fallback_path(A.P, res_pm);
    }
    __syncthreads();
    winner = misc[1];
    const int outp = misc[4];
    const uint32_t* eb = res_e + (size_t)outp * L.sw;
    for (int k = tid; k < n_short; k += blockDim.x)
      if ((eb[k >> 5] >> (k & 31)) & 1u) atomicOr(&cbits[sel[k] >> 5], 1u << (sel[k] & 31));
    if (A.keep) {
      const float* kp = A.kpath + ((size_t)blockIdx.x * A.P.nb + outp) * A.ns_max;
      keep_for_next(A, sm, shot, kp, n_short);
    }
    __syncthreads();
  } else if (A.keep) {
    keep_for_next(A, sm, shot, nullptr, 0, (const float*)(union_base<UG>(A, sm) + L.p_post));
  }
  write_outputs(A, sm, shot, conv, winner, n_short, t_run, tr);
}

template <bool LW, bool UG>
__global__ void __launch_bounds__(256, 2) decode_shot_kernel(DecodeArgs A) {
  extern __shared__ __align__(16) char sm[];
  int* misc = (int*)(sm + A.L.misc);
  Stager stg = stager_init((char*)(misc + 8), &A.counters[4]);
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      misc[0] = atomicAdd(A.work, 1);
      misc[2] = 0;  // decision-path queue, path 0 first
    }
    // no snapshot yet, every path queued
    if (threadIdx.x < 2 * kMaxForkNodes) ((int*)(sm + A.L.red))[threadIdx.x] = 0;
    __syncthreads();
    const long long shot = misc[0];
    if (shot >= A.n_shots) break;
    shot_body<LW, UG>(A, shot, sm, stg);
  }
}

// ---- batched shot mode: one persistent launch over the same window step of
// several decoders (codes and window sizes of different shapes).  Shots are
// numbered across the members in table order; a CTA takes the next one and
// runs it with that member's graph, layout and buffers.  A member's layout
// has as many path slots as fit in the launch's shared memory (at most one
// per warp): small windows use every warp, large ones fewer. ----
template <bool LW>
__global__ void __launch_bounds__(256, 2) decode_batch_kernel(const __grid_constant__ BatchArgs B) {
  extern __shared__ __align__(16) char sm[];
  int* q = (int*)(sm + B.q_off);
  Stager stg = stager_init((char*)(q + 4), &B.seg[0].counters[4]);
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) q[0] = atomicAdd(B.work, 1);
    __syncthreads();
    const long long g = q[0];
    if (g >= B.seg_end[B.n_seg - 1]) break;
    int m = 0;
    while (g >= B.seg_end[m]) ++m;
    const DecodeArgs& A = B.seg[m];
    const long long shot = g - (m ? B.seg_end[m - 1] : 0);
    if (threadIdx.x == 0) ((int*)(sm + A.L.misc))[2] = 0;
    // no snapshot yet, every path queued
    if (A.F.pool && threadIdx.x < 2 * kMaxForkNodes) ((int*)(sm + A.L.red))[threadIdx.x] = 0;
    __syncthreads();
    shot_body<LW, false>(A, shot, sm, stg);
  }
}

// ---- path mode: one CTA per (shot, path); the last CTA of a shot decides ----
template <bool LW>
__global__ void __launch_bounds__(512, 1) decode_path_kernel(DecodeArgs A) {
  extern __shared__ __align__(16) char sm[];
  const Layout& L = A.L;
  const int tid = threadIdx.x;
  const int nb = A.P.nb;
  const long long shot = blockIdx.x / A.cps;
  const int id = blockIdx.x % A.cps;
  int* misc = (int*)(sm + L.misc);
  char* tr = A.trace ? A.trace + (size_t)shot * A.tr_bytes : nullptr;
  Stager stg = stager_init((char*)(misc + 8), &A.counters[4]);
  // stage the window graph in shared memory (one CTA per SM in this mode)
  WinDev W = A.W;
  if (L.g_bytes) {
    const WinDev& G = A.W;
    uint16_t* cp = (uint16_t*)(sm + L.g_colptr);
    uint16_t* cr = (uint16_t*)(sm + L.g_colrows);
    uint16_t* rp = (uint16_t*)(sm + L.g_rowptr);
    uint32_t* re = (uint32_t*)(sm + L.g_rowent);
    float* ll = (float*)(sm + L.g_llr);
    const StagePiece pc[5] = {{cp, G.col_ptr, al16(2u * (G.n_cols + 1))}, {cr, G.col_rows, al16(2u * G.n_edges)},
                              {rp, G.row_ptr, al16(2u * (G.n_rows + 1))}, {re, G.row_ent, al16(4u * G.n_edges)},
                              {ll, G.llr, al16(4u * G.n_cols)}};
    stage_pieces(stg, pc, 5);
    W.col_ptr = cp;
    W.col_rows = cr;
    W.row_ptr = rp;
    W.row_ent = re;
    W.llr = ll;
  }
  int t_run = 0;
  const bool conv = window_prefix<LW, true, false>(A, W, sm, shot, &t_run, stg);
  if (id >= nb) return;  // a CTA that only shared the pre-BP of its cluster
  if (conv) {
    if (id == 0) {
      write_outputs(A, sm, shot, true, -1, 0, t_run, tr);
      if (A.keep) keep_for_next(A, sm, shot, nullptr, 0, (const float*)(union_base<false>(A, sm) + L.p_post));
    }
    return;
  }
  const int n_short = A.W.n_short;
  const ShortG G = short_graph(sm, L, A.W, n_short);
  const Slot B = make_slot(union_base<false>(A, sm), L);
  const CtaGrp g{tid, (int)blockDim.x, sm + L.red};
  const size_t rb = path_result_bytes(A.sw_max);
  char* mine = A.path_res + ((size_t)shot * nb + id) * rb;
  PathOut o = trace_out(A, tr, id, shot);
  o.status = (int*)mine;
  o.pm = (double*)(mine + 8);
  o.ebits = (uint32_t*)(mine + 16);
  if (A.keep) o.keep = A.kpath + ((size_t)shot * nb + id) * A.ns_max;
  run_path<LW>(A.P, G, B, id, g, o, A.dmx, ForkCtx{});
  // publish, then count arrivals; the last CTA of the shot reduces
  __threadfence();
  __syncthreads();
  if (tid == 0) misc[3] = (atomicAdd(&A.arrive[shot], 1) == nb - 1);
  __syncthreads();
  if (!misc[3]) return;
  __threadfence();
  if (tid == 0) {
    int best = -1, fb = 0;
    double bp = CUDART_INF, bk = CUDART_INF;
    for (int q = 0; q < nb; ++q) {
      const char* r = A.path_res + ((size_t)shot * nb + q) * rb;
      const int st = __ldcg((const int*)r);
      const double pm = __ldcg((const double*)(r + 8));
      if (st == BR_CONVERGED && pm < bp) {
        bp = pm;
        best = q;
      }
      if (A.P.fallback && st != BR_CONVERGED && pm < bk) {  // the fallback key (see fallback_path)
        bk = pm;
        fb = q;
      }
    }
    misc[1] = best;
    misc[4] = best >= 0 ? best : fb;
    A.arrive[shot] = 0;  // ready for the next launch
  }
  __syncthreads();
  const int winner = misc[1];
  const int outp = misc[4];
  const uint32_t* eb = (const uint32_t*)(A.path_res + ((size_t)shot * nb + outp) * rb + 16);
  uint32_t* cbits = (uint32_t*)(sm + L.cbits);
  const uint16_t* sel = (const uint16_t*)(sm + L.sel);
  for (int k = tid; k < n_short; k += blockDim.x)
    if ((__ldcg(&eb[k >> 5]) >> (k & 31)) & 1u) atomicOr(&cbits[sel[k] >> 5], 1u << (sel[k] & 31));
  if (A.keep) keep_for_next(A, sm, shot, A.kpath + ((size_t)shot * nb + outp) * A.ns_max, n_short);
  __syncthreads();
  write_outputs(A, sm, shot, false, winner, n_short, t_run, tr);
}

// ---- Philox4x32-10 (Salmon et al., SC'11) ----
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
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
      const uint4 u = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)shot, (uint32_t)(shot >> 32), 0u), key);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int c = 4 * g + r;
        if (c < n_cols && uu[r] < thr[c]) {
          for (int e = cptr[c]; e < cptr[c + 1]; ++e) {
            const int d = cdet[e];
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

// Commit (Eq. (10)) + residue test (Eq. (11)) of shot s.
__device__ void commit_one(const CommitArgs& C, long long s) {
  const uint32_t* c = C.corr + (size_t)s * C.corr_words;
  uint32_t* d = C.det + (size_t)s * C.det_words;
  uint32_t ob = 0;
  const int nw = (C.n_commit + 31) >> 5;
  for (int x = 0; x < nw; ++x) {
    uint32_t m = c[x];
    const int rem = C.n_commit - 32 * x;
    if (rem < 32) m &= (1u << rem) - 1u;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int col = 32 * x + b;
      for (int e = C.cptr[col]; e < C.cptr[col + 1]; ++e) {
        const int q = C.cdet[e];
        d[q >> 5] ^= 1u << (q & 31);
      }
      ob ^= C.cobs[col];
    }
  }
  C.obs_pred[s] ^= ob;
  uint32_t bad = 0;
  for (int q = C.b0; q < C.b1;) {
    const int wq = q >> 5, lo = q & 31;
    const int hiq = min(C.b1, (wq + 1) * 32);
    uint32_t m = d[wq] >> lo;
    const int nb = hiq - q;
    if (nb < 32) m &= (1u << nb) - 1u;
    bad |= m;
    q = hiq;
  }
  if (bad) C.resid[s] |= 1u;
}

// one thread per shot
__global__ void commit_kernel(const CommitArgs C) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < C.n) commit_one(C, s);
}

// one thread per shot over several decoders' shots
__global__ void commit_batch_kernel(const __grid_constant__ CommitBatch B) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= B.seg_end[B.n_seg - 1]) return;
  int m = 0;
  while (g >= B.seg_end[m]) ++m;
  commit_one(B.seg[m], g - (m ? B.seg_end[m - 1] : 0));
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
  const unsigned m = __ballot_sync(FULL, f != 0);
  if (n_fail && (threadIdx.x & 31) == 0 && m) atomicAdd((unsigned long long*)n_fail, (unsigned long long)__popc(m));
}

}  // namespace dev

// ---------------------------------------------------------------------------
// Host-side launch wrappers (declared in qdec_internal.h).

size_t trace_bytes_per_shot(int nb, int dmx, int ns_max) { return dev::trace_bytes(nb, dmx, ns_max); }

cudaError_t set_decode_smem(size_t bytes) {
  const int b = (int)bytes;
  cudaError_t e =
      cudaFuncSetAttribute(dev::decode_shot_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dev::decode_shot_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dev::decode_shot_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dev::decode_shot_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dev::decode_path_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dev::decode_path_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dev::decode_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dev::decode_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

cudaError_t batch_occupancy(int threads, size_t smem, int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dev::decode_batch_kernel<false>, threads, smem);
}

cudaError_t launch_decode_batch(cudaStream_t st, int grid, int threads, size_t smem, unsigned q_off, int* work,
                                const BatchMember* m, int n) {
  if (n <= 0 || n > kMaxBatch) return n <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  dev::BatchArgs B{};
  B.n_seg = n;
  B.q_off = q_off;
  B.work = work;
  bool lw = false;
  long long end = 0;
  for (int i = 0; i < n; ++i) {
    const BatchMember& x = m[i];
    end += x.n;
    B.seg_end[i] = end;
    B.seg[i] = dev::DecodeArgs{*x.P,   *x.W,   *x.L,     x.det,      x.det_words, x.n,      x.corr,
                               x.corr_words, nullptr, nullptr, 0,     x.dmx,    x.ns_max, nullptr,
                               x.counters, nullptr, nullptr, x.sw_max, nullptr, 0, 1,
                               x.counters ? x.counters + 5 : nullptr, x.fork ? *x.fork : ForkDev{}};
    lw = lw || x.W->wts != nullptr;
  }
  if (lw) dev::decode_batch_kernel<true><<<grid, threads, smem, st>>>(B);
  else dev::decode_batch_kernel<false><<<grid, threads, smem, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_commit_batch(cudaStream_t st, const BatchMember* m, int n) {
  if (n <= 0 || n > kMaxBatch) return n <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  dev::CommitBatch B{};
  B.n_seg = n;
  long long end = 0;
  for (int i = 0; i < n; ++i) {
    const BatchMember& x = m[i];
    end += x.n;
    B.seg_end[i] = end;
    B.seg[i] = dev::CommitArgs{x.n_commit, x.cptr, x.cdet, x.cobs, x.corr_words, x.corr, x.n,
                               (uint32_t*)x.det, x.det_words, x.obs_pred, x.resid, x.b0, x.b1};
  }
  if (end == 0) return cudaSuccess;
  const int tpb = 128;
  dev::commit_batch_kernel<<<(unsigned)((end + tpb - 1) / tpb), tpb, 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t decode_occupancy(int mode, int threads, size_t smem, int* blocks) {
  if (mode == 1)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dev::decode_path_kernel<false>, threads, smem);
  if (mode == 3)  // shot mode with the union region in global memory
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dev::decode_shot_kernel<false, true>, threads, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dev::decode_shot_kernel<false, false>, threads, smem);
}

cudaError_t path_cluster_occupancy(int threads, size_t smem, int cluster, int* clusters) {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  cfg.gridDim = dim3((unsigned)cluster);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(clusters, dev::decode_path_kernel<false>, &cfg);
}

cudaError_t launch_decode(int mode, int grid, int threads, size_t smem, cudaStream_t st, const KParams& P,
                          const WinDev& W, const Layout& L, const uint32_t* det, int det_words, long long n,
                          uint32_t* corr, int corr_words, int32_t* status, char* trace, size_t tr_bytes, int dmx,
                          int ns_max, int* work, long long* counters, char* path_res, int* arrive, int sw_max,
                          char* uglob, size_t ubytes, int cps, int cluster, const ForkDev* fork,
                          const ReuseDev* reuse) {
  // counters[5]: the GDG edge visits the launch executed (counters[1] adds
  // the resumed prefixes every path counts as its own)
  const dev::DecodeArgs A{P,     W,        L,     det,      det_words, n,     corr,     corr_words, status,
                          trace, tr_bytes, dmx,   ns_max,   work,      counters, path_res, arrive,     sw_max,
                          uglob, ubytes,   cps,   counters ? counters + 5 : nullptr, fork ? *fork : ForkDev{},
                          reuse ? reuse->keep : nullptr, reuse ? reuse->keep_ld : 0, reuse ? reuse->prev : nullptr,
                          reuse ? reuse->kpath : nullptr};
  const bool lw = W.wts != nullptr;
  if (mode == 1) {  // one cluster of `cluster` CTAs shares each shot's pre-BP
    // every path needs its CTA, and a cluster never spans two shots
    if (cluster < 1 || cps < P.nb || cps % cluster || grid % cps) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (lw) return cudaLaunchKernelEx(&cfg, dev::decode_path_kernel<true>, A);
    return cudaLaunchKernelEx(&cfg, dev::decode_path_kernel<false>, A);
  } else {
    if (uglob) {
      if (lw) dev::decode_shot_kernel<true, true><<<grid, threads, smem, st>>>(A);
      else dev::decode_shot_kernel<false, true><<<grid, threads, smem, st>>>(A);
    } else {
      if (lw) dev::decode_shot_kernel<true, false><<<grid, threads, smem, st>>>(A);
      else dev::decode_shot_kernel<false, false><<<grid, threads, smem, st>>>(A);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_sample(cudaStream_t st, int n_cols, const uint32_t* thr, const int* cptr, const int* cdet,
                          const uint32_t* cobs, int det_words, unsigned long long seed, unsigned long long off,
                          long long n, uint32_t* det, uint32_t* obs) {
  if (n <= 0) return cudaSuccess;
  const int wpb = 8;
  const long long blocks = (n + wpb - 1) / wpb;
  dev::sample_kernel<<<(unsigned)blocks, 32 * wpb, sizeof(uint32_t) * wpb * det_words, st>>>(
      n_cols, thr, cptr, cdet, cobs, det_words, seed, off, n, det, obs);
  return cudaGetLastError();
}

cudaError_t launch_commit(cudaStream_t st, int n_commit, const int* cptr, const int* cdet, const uint32_t* cobs,
                          int corr_words, const uint32_t* corr, long long n, uint32_t* det, int det_words,
                          uint32_t* obs_pred, uint32_t* resid, int b0, int b1) {
  if (n <= 0) return cudaSuccess;
  const int tpb = 128;
  const dev::CommitArgs C{n_commit, cptr, cdet, cobs, corr_words, corr, n, det, det_words, obs_pred, resid, b0, b1};
  dev::commit_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(C);
  return cudaGetLastError();
}

cudaError_t launch_evaluate(cudaStream_t st, const uint32_t* pred, const uint32_t* obs, const uint32_t* resid,
                            long long n, uint32_t* fail, long long* n_fail) {
  if (n <= 0) return cudaSuccess;
  const int tpb = 256;
  dev::evaluate_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(pred, obs, resid, n, fail, n_fail);
  return cudaGetLastError();
}

}  // namespace qd
