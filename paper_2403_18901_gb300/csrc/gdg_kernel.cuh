// gdg_kernel.cuh -- device code of the window decoder (one CTA per shot).
//
// Message representation.  Min-sum (Eq. (1)) sends from check j to variable i
//   mu_{j->i} = (-1)^{s_j} * (alpha * min_{i' != i} |mu_{i'->j}|) * prod_{i' != i} sign(mu_{i'->j})
// which only depends on the check's two smallest |mu| (min1, min2), the edge
// holding min1 (amin), the sign parity of all its inputs xor s_j, and the sign
// of the receiving edge's own input.  The kernel keeps exactly that per check
// plus one sign byte per edge, instead of two FP32 messages per edge.  The
// VN->CN message of Eq. (3) is recomputed where it is needed as
// clip(Lambda_i^(t) - mu_{j->i}), the same FP32 operations the explicit
// form performs, so every value is bit-identical to it.  All FP32 operations
// are __fadd_rn / __fmul_rn (never contracted into FMA).
#pragma once
#include <cstdint>

namespace qd {

struct KParams {
  float alpha, clip, pa_main, pa_other, pb_main, pb_other, pb_d1, pc, pd;
  int n_pre, ips, dmax_main, dmax_other, k, low_err, peel_init, pc_max_depth, n_unsat_min;
  int nb;  // 2^k
};

// One window's Tanner graph in global memory (read-only for all shots).
struct WinDev {
  int n_rows, n_cols, n_edges, row0, n_short, es_max;
  const uint16_t *col_ptr, *col_rows, *row_ptr, *row_edges, *edge_col;
  const float* llr;
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

// Shared-memory layout of one CTA (byte offsets), identical on host and device.
struct Layout {
  // persistent
  unsigned sbits, cbits, sel, s_colptr, s_colrows, s_rowptr, s_rowedges, s_edgecol, s_llr, s_vdeg,
      rowcnt, res_status, res_pm, res_ebits, misc;
  unsigned U;  // start of the union region
  // pre-BP (relative to U)
  unsigned p_post, p_key, p_min1, p_min2, p_amin, p_cfl, p_sign, p_par, p_sort, p_end;
  // one branch slot (relative to the slot base)
  unsigned b_post, b_acc, b_hfl, b_status, b_sign, b_min1, b_min2, b_amin, b_cfl, b_deg, b_sp,
      b_par, b_unsat, b_size;
  unsigned total;
  int rw, cw, sw, sortn;
};

__host__ __device__ inline unsigned al16(unsigned x) { return (x + 15u) & ~15u; }

__host__ __device__ inline Layout make_layout(int nr, int nc, int ne, int ns, int es, int nb,
                                              int nwarps) {
  Layout L{};
  L.rw = (nr + 31) / 32;
  L.cw = (nc + 31) / 32;
  L.sw = (ns + 31) / 32;
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
  L.s_rowedges = o; o = al16(o + 2u * es);
  L.s_edgecol = o; o = al16(o + 2u * es);
  L.s_llr = o; o = al16(o + 4u * ns);
  L.s_vdeg = o; o = al16(o + 1u * ns);
  L.rowcnt = o; o = al16(o + 4u * (nr + 1));
  L.res_status = o; o = al16(o + 4u * nb);
  L.res_pm = o; o = al16(o + 8u * nb);
  L.res_ebits = o; o = al16(o + 4u * L.sw * nb);
  L.misc = o; o = al16(o + 64u);
  L.U = o;
  unsigned u = 0;
  L.p_post = u; u = al16(u + 4u * nc);
  L.p_key = u; u = al16(u + 4u * nc);
  L.p_min1 = u; u = al16(u + 4u * nr);
  L.p_min2 = u; u = al16(u + 4u * nr);
  L.p_amin = u; u = al16(u + 2u * nr);
  L.p_cfl = u; u = al16(u + 1u * nr);
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
  L.b_min1 = b; b = al16(b + 4u * nr);
  L.b_min2 = b; b = al16(b + 4u * nr);
  L.b_amin = b; b = al16(b + 2u * nr);
  L.b_cfl = b; b = al16(b + 1u * nr);
  L.b_deg = b; b = al16(b + 4u * nr);
  L.b_sp = b; b = al16(b + 4u * L.rw);
  L.b_par = b; b = al16(b + 8u * L.rw);
  L.b_unsat = b; b = al16(b + 4u * L.rw);
  L.b_size = b;
  unsigned ub = L.p_end > b * (unsigned)nwarps ? L.p_end : b * (unsigned)nwarps;
  L.total = L.U + ub;
  return L;
}

}  // namespace qd
