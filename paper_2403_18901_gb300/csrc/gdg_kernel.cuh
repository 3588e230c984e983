// gdg_kernel.cuh -- shared definitions of the window decoder (host and device).
//
// Message representation.  Min-sum (Eq. (1)) sends from check j to variable i
//   mu_{j->i} = (-1)^{s_j} * (alpha * min_{i' != i} |mu_{i'->j}|) * prod_{i' != i} sign(mu_{i'->j})
// which only depends on the check's two smallest |mu| (min1, min2), the edge
// holding min1 (amin), the sign parity of all its inputs xor s_j, and the sign
// of the receiving edge's own input.  The kernel keeps exactly that per check
// (one 16-byte record) plus one sign byte per edge, instead of two FP32
// messages per edge.  The VN->CN message of Eq. (3) is recomputed where it is
// needed as clip(Lambda_i^(t) - mu_{j->i}), the same FP32 operations the
// explicit form performs, so every value is bit-identical to it.  All FP32
// operations are __fadd_rn / __fsub_rn / __fmul_rn (never contracted).
#pragma once
#include <cstddef>
#include <cstdint>

namespace qd {

constexpr int kMaxBatch = 16;  // decoders in one batched launch

struct KParams {
  float alpha, clip, pa_main, pa_other, pb_main, pb_other, pb_d1, pc, pd;
  int n_pre, ips, dmax_main, dmax_other, k, low_err, peel_init, pc_max_depth, n_unsat_min;
  int nb;        // decision paths: 2^k tree + side branches
  int side_max;  // side branches split off the main branch at D_split = k .. side_max (0: none)
  int reinit;    // 1: a path continuing from another's snapshot restarts its messages there
  int ips1;      // BP iterations of the first decimation step (0: ips)
  int fallback;  // output when no path converges: 0 path 0, 1 fewest unsatisfied checks, 2 committed ones first
  // learned decimation ranker (NULL: the argmin of Alg. 1): rkq = the
  // grid-rounded W1[64][8], b1[64], W2[64], b2; rkb[t][lane] = the BF16 pair
  // (W1[8t + lane/4][2 (lane%4)], W1[8t + lane/4][2 (lane%4) + 1]), the B
  // fragment of an m16n8k8 MMA for hidden units 8t..8t+7
  const float* rkq;
  const uint32_t* rkb;
  // candidate dump of path 0 (ranker training data; NULL: off)
  struct RankRec* dump;
  int* dump_n;
  int dump_cap;
};

// One ranker candidate (layout of qd_rank_rec_t): features, shot, window
// column, selection depth, path; flags bit 0 = [L <= 0], bit 1 = selected.
struct RankRec {
  float x[8];
  int32_t shot, wcol;
  int16_t depth, path;
  int32_t flags;
};

// Side-branch split depth of path `id` (Fig. 2): 0 for the main and tree
// branches.  With side branches, id 1 (contrary only at D = k) is the one
// splitting at D = k and ids 2^k.. split at D = k + 1 ...
__host__ __device__ inline int path_split(const KParams& P, int id) {
  if (P.side_max <= 0) return 0;
  const int nt = 1 << P.k;
  if (id >= nt) return P.k + 1 + (id - nt);
  return (id == 1 && P.k >= 1) ? P.k : 0;
}

// Depth after whose decimation path `id` restarts its messages (reinit
// reading: side branches at their split, odd tree ids at D = k); 0: never.
__host__ __device__ inline int path_reinit(const KParams& P, int id, int split) {
  if (!P.reinit) return 0;
  if (split) return split;
  return (id >= 1 && (id & 1) && P.k >= 1) ? P.k : 0;
}

// D_max of path `id` with side-branch split `split` (Fig. 2): the main
// branch's own; a side branch runs as many steps past its split as a tree
// branch runs past depth k.
__host__ __device__ inline int path_dmax(const KParams& P, int id, int split) {
  return id == 0 ? P.dmax_main : (split ? split + (P.dmax_other - P.k) : P.dmax_other);
}

// Shot-mode queue order: the main branch, side branches from the deepest
// split down, then the tree branches -- the longest paths first when the main
// branch's D_max is the largest (the circuit-level presets; the code-capacity
// tree's deepest side branches outlast its main branch).  The order only
// schedules the paths; every result is kept by path id.
__host__ __device__ inline int path_at(const KParams& P, int pos) {
  const int nside = P.nb - (1 << P.k);
  if (pos == 0) return 0;
  if (pos <= nside) return P.nb - pos;
  return pos - nside;
}

// One window's Tanner graph in global memory (read-only for all shots).
struct WinDev {
  int n_rows, n_cols, n_edges, row0, n_short, es_max, rows_per_block;
  const uint16_t *col_ptr, *col_rows, *row_ptr;
  const uint32_t* row_ent;  // CSR entry: CSC edge id | (column << 16)
  const float* llr;
  // learned weighted min-sum: wts[(min(t, wT) - 1) * n_edges + e] replaces
  // alpha at iteration t (counted from message initialisation); NULL = alpha
  const float* wts;
  int wT;
  const uint16_t* vperm;  // pre-BP processing order of the columns (descending degree)
  int n_commit_rows;      // rows [0, n_commit_rows) are the ones the window commits
};

// Shot mode's plan for resuming decision paths from snapshots of shared
// prefixes (see ForkCtx in gdg_kernel.cu): the queue order, and for every path
// p and depth D the snapshot node of p after the BP of step D
// (chain[p * dmx + D - 1], -1: none).  Snapshots of CTA b live at
// pool + b * cta_bytes, nodes `stride` bytes apart; pool = nullptr: no
// snapshots, the path-queue order of path_at.
// node flags, then path states, live in the shot-mode CTA's 512-byte reduction area
constexpr int kMaxForkNodes = 64;
constexpr unsigned kSnapHeaderBytes = 32;  // a snapshot's header, before the copy of the slot
// fnode / fdep: each path's planned snapshot node (-1: none) and its depth;
// sched != 0: preemption at step boundaries, each path's parking snapshot
// after the n_nodes node snapshots of the CTA's pool.
struct ForkDev {
  const int16_t* order;
  const int16_t* chain;
  const int16_t* fnode;
  const int16_t* fdep;
  char* pool;
  size_t cta_bytes;
  int n_nodes, pool_ctas, sched;
};

// Message reuse between windows (see DecodeArgs::keep); keep = nullptr: off.
struct ReuseDev {
  float* keep;
  int keep_ld;
  const int16_t* prev;
  float* kpath;
};

// A window's Tanner graph for the learned weighted min-sum (training kernels).
struct WmsGraph {
  int nr, nc, ne, rw, T, ckpt;
  const uint16_t *col_ptr, *col_rows, *row_ptr;
  const uint32_t* row_ent;  // CSC edge id | column << 16
  const float* llr;
  float clip;
};

// Compressed state of one check node: two smallest |input| and the edge
// holding the smallest (ac).  Plain decoder: the magnitudes multiplied by
// alpha (alpha * clip twice when exactly one input is active), each negated
// when the sign parity xor s_j is 1, and ac = the edge.  Learned weights: the
// magnitudes unscaled, ac = edge | parity << 16 | (exactly one active input)
// << 17.
struct __align__(16) CNState {
  float m1, m2;
  uint32_t ac, pad;
};

struct BranchTrace {
  int32_t status, depth, iters, pad;
  double pm;
};
struct StepTrace {
  int16_t g;
  int8_t value, pad;
  int16_t n_agg, n_peel;
};

// Result of one decision path in the path-per-CTA launch (global scratch).
__host__ __device__ inline size_t path_result_bytes(int sw) { return (16 + 4 * (size_t)sw + 15) & ~(size_t)15; }

// Shared-memory layout of one CTA (byte offsets), identical on host and device.
struct Layout {
  // persistent
  unsigned sbits, cbits, sel, s_colptr, s_colrows, s_rowptr, s_rowent, s_llr, s_vdeg, s_efull, s_cperm, s_vperm, rowcnt,
      res_status, res_pm, res_ebits, red, misc;
  // window graph staged in shared memory (path mode only; 0 bytes otherwise)
  unsigned g_colptr, g_colrows, g_rowptr, g_rowent, g_llr, g_bytes;
  unsigned U;  // start of the union region
  // pre-BP (relative to U)
  unsigned p_post, p_key, p_cns, p_sign, p_par, p_sort, p_end;
  // the window graph staged for the pre-BP loop in otherwise idle union bytes
  // (from p_sort on; overwritten by the sort that follows); pre_stage = 0: none
  unsigned pre_stage, q_colptr, q_colrows, q_rowptr, q_rowent, q_llr, q_vperm;
  // one path slot (relative to the slot base)
  unsigned b_post, b_acc, b_hfl, b_status, b_sign, b_cns, b_deg, b_sp, b_unsat, b_hq, b_size;
  unsigned total;
  int rw, cw, sw, sortn, nslots;
};

__host__ __device__ inline unsigned al16(unsigned x) { return (x + 15u) & ~15u; }

// lw: the shortened edges' full-window edge ids (s_efull) are kept, which
// only learned weights read
__host__ __device__ inline Layout make_layout(int nr, int nc, int ne, int ns, int es, int nb,
                                              int nslots, bool stage_graph = false, bool ranker = false,
                                              bool lw = true) {
  Layout L{};
  L.rw = (nr + 31) / 32;
  L.cw = (nc + 31) / 32;
  L.sw = (ns + 31) / 32;
  L.nslots = nslots;
  int sn = 1;
  while (sn < nc) sn <<= 1;
  L.sortn = sn;
  unsigned o = 0;
  L.sbits = o; o = al16(o + 4u * L.rw);
  L.cbits = o; o = al16(o + 4u * L.cw);
  L.sel = o; o = al16(o + 2u * ns);
  L.s_colptr = o; o = al16(o + 2u * (ns + 1));
  L.s_colrows = o; o = al16(o + 2u * es);
  L.s_rowptr = o; o = al16(o + 2u * (nr + 1));
  L.s_rowent = o; o = al16(o + 4u * es);
  L.s_llr = o; o = al16(o + 4u * ns);
  L.s_vdeg = o; o = al16(o + 1u * ns);
  L.s_efull = o; o = al16(o + (lw ? 2u * es : 0u));
  L.s_cperm = o; o = al16(o + 2u * nr);
  L.s_vperm = o; o = al16(o + 2u * ns);
  L.rowcnt = o; o = al16(o + 4u * (nr + 1));
  L.res_status = o; o = al16(o + 4u * nb);
  L.res_pm = o; o = al16(o + 8u * nb);
  L.res_ebits = o; o = al16(o + 4u * L.sw * nb);
  L.red = o; o = al16(o + 16u * 32);
  L.misc = o; o = al16(o + 64u);
  const unsigned g0 = o;
  if (stage_graph) {
    L.g_colptr = o; o = al16(o + 2u * (nc + 1));
    L.g_colrows = o; o = al16(o + 2u * ne);
    L.g_rowptr = o; o = al16(o + 2u * (nr + 1));
    L.g_rowent = o; o = al16(o + 4u * ne);
    L.g_llr = o; o = al16(o + 4u * nc);
  }
  L.g_bytes = o - g0;
  L.U = o;
  unsigned u = 0;
  L.p_post = u; u = al16(u + 4u * nc);
  L.p_key = u; u = al16(u + 4u * nc);
  L.p_cns = u; u = al16(u + 16u * nr);
  L.p_sign = u; u = al16(u + 1u * ne);
  L.p_par = u; u = al16(u + 8u * L.rw);
  L.p_sort = u; u = al16(u + 8u * sn);
  L.p_end = u;
  unsigned b = 0;
  L.b_post = b; b = al16(b + 4u * ns);
  L.b_acc = b; b = al16(b + 4u * ns);
  L.b_hfl = b; b = al16(b + 1u * ns);
  L.b_status = b; b = al16(b + 1u * ns);
  L.b_sign = b; b = al16(b + 1u * es);
  L.b_cns = b; b = al16(b + 16u * nr);
  L.b_deg = b; b = al16(b + 4u * nr);
  L.b_sp = b; b = al16(b + 4u * L.rw);
  L.b_unsat = b; b = al16(b + 4u * L.rw);
  L.b_hq = b; b = al16(b + (ranker ? 4u * ns : 0u));
  L.b_size = b;
  unsigned ub = L.p_end > b * (unsigned)nslots ? L.p_end : b * (unsigned)nslots;
  if (!stage_graph) {
    unsigned q = L.p_sort;
    L.q_colptr = q; q = al16(q + 2u * (nc + 1));
    L.q_colrows = q; q = al16(q + 2u * ne);
    L.q_rowptr = q; q = al16(q + 2u * (nr + 1));
    L.q_rowent = q; q = al16(q + 4u * ne);
    L.q_llr = q; q = al16(q + 4u * nc);
    L.q_vperm = q; q = al16(q + 2u * nc);
    L.pre_stage = q <= ub ? 1u : 0u;
  }
  L.total = L.U + ub;
  return L;
}

}  // namespace qd
