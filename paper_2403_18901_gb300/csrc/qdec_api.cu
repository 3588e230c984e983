// qdec_api.cu -- the C ABI of libqdec (see include/qdec.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gdg_kernel.cuh"
#include "qdec_internal.h"

namespace qd {
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
}  // namespace qd

using qd::set_error;

#define QD_CK(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
      return QD_ECUDA;                                                                \
    }                                                                                 \
  } while (0)

#define QD_CK_ST(call)             \
  do {                             \
    const qd_status s_ = (call);   \
    if (s_ != QD_OK) return s_;    \
  } while (0)

#define QD_REQ(cond, msg)    \
  do {                       \
    if (!(cond)) {           \
      set_error(msg);        \
      return QD_EINVAL;      \
    }                        \
  } while (0)

struct qd_dem {
  qd::DemHost h;
  // device copies, uploaded on first device use (so that the host-side
  // queries work on a machine without a GPU)
  mutable int* d_cptr = nullptr;
  mutable int* d_cdet = nullptr;
  mutable uint32_t* d_cobs = nullptr;
  mutable uint32_t* d_thr = nullptr;
};

namespace {

// Launch shapes of the decode kernel: shot mode (persistent CTAs of up to
// kShotWarps warps, one warp per decision path, as many as fit in shared
// memory) and path mode (one CTA of kPathThreads threads per (shot, path)).
constexpr int kShotWarps = 8;
constexpr int kPathThreads = 512;
constexpr long long kPathModeMaxShots = 64;
constexpr int kCounters = 8;

struct WinGpu {
  qd::WindowHost h;
  qd::WinDev dv{};
  qd::Layout L{};   // shot mode
  qd::Layout Lp{};  // path mode
  void* d_graph = nullptr;
  int* d_ccptr = nullptr;  // committed columns: CSR of their global detector ids
  int* d_ccdet = nullptr;
  uint32_t* d_ccobs = nullptr;
  int grid_per_sm = 1;
  int shot_warps = kShotWarps;
  uint32_t* d_wthr = nullptr;  // window-local sampling thresholds (on first use)
  // union region in global memory (windows too large for shared memory, or
  // launch mode 3): layout, CTAs per SM, and whether the shared-memory
  // layouts fit at all
  qd::Layout Lg{};
  int grid_g = 1;
  bool fits = true, path_fits = true;
  int pcl = 1;  // path mode: CTAs per cluster sharing a shot's pre-BP
  // shot mode's snapshot plan (qd::ForkDev): queue order [nb], then the
  // node chain [nb][dmx]; fork_nodes = 0: none
  int16_t* d_fork = nullptr;
  int fork_nodes = 0;
  bool fork_on = false;
  // message reuse: this window's column -> the previous window's column of
  // the same DEM column (-1: none); nullptr for the first window
  int16_t* d_prev = nullptr;
};

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  size_t n = std::max<size_t>(v.size(), 1);
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  if (!v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

qd_status ensure_device(const qd_dem* d) {
  if (d->d_thr) return QD_OK;
  QD_CK(upload(&d->d_cptr, d->h.col_ptr));
  QD_CK(upload(&d->d_cdet, d->h.col_dets));
  QD_CK(upload(&d->d_cobs, d->h.col_obs));
  QD_CK(upload(&d->d_thr, d->h.col_thr));
  return QD_OK;
}

}  // namespace

struct qd_decoder {
  const qd_dem* dem = nullptr;
  qd_gdg_params P{};
  qd::KParams kp{};
  long long max_shots = 0;
  std::vector<WinGpu> wins;
  int corr_words = 0, dmx = 0, ns_max = 0, sm_count = 0, sw_max = 0;
  int launch_mode = 0;  // 0 automatic, 1 shot mode, 2 path mode, 3 shot mode with the union region in global memory
  char* d_uscratch = nullptr;  // global union regions (one per resident CTA)
  size_t uscratch_bytes = 0;
  char* d_path_res = nullptr;
  int* d_arrive = nullptr;
  size_t trace_bytes = 0, smem_max = 0;
  int smem_optin = 0;
  bool hist_on = false;  // layouts hold the quantised history (ranker or dump)
  bool lw_on = false;    // layouts keep the shortened edges' full-window ids (learned weights)
  void* d_ranker = nullptr;  // grid-rounded parameters (644 floats), then the 256 B fragments
  int* d_work = nullptr;
  long long* d_counters = nullptr;  // kCounters entries (qd_decoder_counters_ex)
  uint32_t* d_corr = nullptr;
  // shot mode's snapshots of shared path prefixes: one pool per resident CTA
  char* d_snap = nullptr;
  size_t snap_cta_bytes = 0;
  int snap_ctas = 0;
  bool fork_on = true;
  bool sched_on = true;  // preemption at step boundaries (with fork_on)
  // message reuse between windows (qd_gdg_params.reuse_msgs): per shot the
  // values a window keeps for the next [max_shots][keep_ld], and every
  // candidate path's values [slots][nb][ns_max]
  float* d_keep = nullptr;
  int keep_ld = 0;
  float* d_kpath = nullptr;
  size_t kpath_slots = 0;
  uint32_t *d_det = nullptr, *d_obs = nullptr, *d_pred = nullptr, *d_fail = nullptr, *d_resid = nullptr;
  long long* d_nfail = nullptr;
};

namespace {
// Shared-memory layouts of every window: as many decision-path slots (warps)
// as fit in shot mode, then the path-mode layout with the window graph staged
// in shared memory when it fits too.  The ranker and the candidate dump add
// the quantised history (4 bytes per short column) to every slot.
// Global union regions for the windows that need them (all windows when
// `all`): one region per resident CTA, allocated once, never on a decode call.
qd_status ensure_uscratch(qd_decoder* dec, bool all) {
  size_t need = 0;
  for (const WinGpu& g : dec->wins)
    if (all || !g.fits)
      need = std::max(need, (size_t)dec->sm_count * g.grid_g * (size_t)(g.Lg.total - g.Lg.U));
  if (need <= dec->uscratch_bytes) return QD_OK;
  cudaFree(dec->d_uscratch);
  dec->d_uscratch = nullptr;
  dec->uscratch_bytes = 0;
  QD_CK(cudaMalloc(&dec->d_uscratch, need));
  dec->uscratch_bytes = need;
  return QD_OK;
}

// Shot mode's plan for sharing path prefixes (qd::ForkDev).  The decision of
// path p at depth d is summarised as (contrary value at d, main-branch
// thresholds of Alg. 3 at d (when Alg. 3 is on), message restart after d);
// two paths with equal summaries at depths 1..D-1 hold the same state after
// the BP of step D.  The queue order runs `wave` paths at once first, each
// sharing as little as possible with those before it, then takes the paths
// that share the deepest prefix with a path before them; node = the deepest
// state such a later path shares with an earlier one.
struct ForkPlan {
  std::vector<int16_t> order, chain, fnode, fdep;
  int n_nodes = 0;
  bool on = false;  // more paths than warps: a plan (preemption, and snapshots when n_nodes > 0)
};

ForkPlan fork_plan(const qd::KParams& P, int dmx, int wave) {
  const int nb = P.nb;
  auto dmax = [&](int p) { return qd::path_dmax(P, p, qd::path_split(P, p)); };
  auto sig = [&](int p, int d) {
    const int split = qd::path_split(P, p);
    const int contrary = split ? (d == split ? 1 : 0) : (d <= P.k ? (p >> (P.k - d)) & 1 : 0);
    const int mainr = P.low_err ? 0 : ((p == 0 || (split && d <= split)) ? 1 : 0);
    const int re = qd::path_reinit(P, p, split) == d ? 1 : 0;
    return contrary | (mainr << 1) | (re << 2);
  };
  // deepest D with equal summaries below it that both paths reach
  auto shared = [&](int p, int q) {
    const int m = std::min(dmax(p), dmax(q));
    int D = 1;
    while (D < m && sig(p, D) == sig(q, D)) ++D;
    return D;
  };
  ForkPlan F;
  std::vector<int> order;
  std::vector<char> used(nb, 0);
  std::vector<int> share(nb, 0);  // deepest prefix shared with a path before it in the order
  for (int pos = 0; pos < nb; ++pos) {
    int best = -1, bkey = 0, bs = 0;
    for (int q = 0; q < nb; ++q) {
      if (used[q]) continue;
      int s = 0;
      for (int p : order) s = std::max(s, shared(p, q));
      const int key = pos < wave ? -s : s;
      if (best < 0 || key > bkey || (key == bkey && dmax(q) > dmax(best))) {
        best = q;
        bkey = key;
        bs = s;
      }
    }
    used[best] = 1;
    share[best] = pos < wave ? 0 : bs;
    order.push_back(best);
  }
  // nodes: (depth, summaries below it) of every later path's shared prefix
  std::vector<std::vector<int>> keys;
  auto key_of = [&](int p, int D) {
    std::vector<int> k{D};
    for (int d = 1; d < D; ++d) k.push_back(sig(p, d));
    return k;
  };
  for (int q = 0; q < nb; ++q)
    if (share[q] >= 1) {
      const std::vector<int> k = key_of(q, share[q]);
      if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
    }
  if (nb <= wave || nb > qd::kMaxForkNodes || (int)keys.size() > qd::kMaxForkNodes) return F;
  F.on = true;
  F.n_nodes = (int)keys.size();
  F.order.assign(order.begin(), order.end());
  F.chain.assign((size_t)nb * dmx, (int16_t)-1);
  F.fnode.assign(nb, (int16_t)-1);
  F.fdep.assign(nb, (int16_t)0);
  for (int p = 0; p < nb; ++p) {
    for (int D = 1; D <= dmax(p) && D <= dmx; ++D) {
      const auto it = std::find(keys.begin(), keys.end(), key_of(p, D));
      if (it != keys.end()) F.chain[(size_t)p * dmx + D - 1] = (int16_t)(it - keys.begin());
    }
    if (share[p] >= 1) {
      F.fnode[p] = F.chain[(size_t)p * dmx + share[p] - 1];
      F.fdep[p] = (int16_t)share[p];
    }
  }
  return F;
}

qd_status configure_layouts(qd_decoder* dec, bool hist, const char* who) {
  struct Conf {
    qd::Layout L, Lp, Lg;
    int shot_warps, grid_per_sm, grid_g, pcl;
    bool fits, path_fits;
  };
  const int optin = dec->smem_optin;
  const int nb = dec->kp.nb;
  size_t smem_max = 0;
  std::vector<Conf> cf(dec->wins.size());
  for (size_t w = 0; w < cf.size(); ++w) {
    Conf& c = cf[w];
    c.pcl = 1;
    const auto& h = dec->wins[w].h;
    auto lay = [&](int slots, bool stage) {
      return qd::make_layout(h.n_rows, h.n_cols, h.n_edges, h.n_short, h.short_edges_max, nb, slots, stage, hist,
                             dec->lw_on);
    };
    // the most resident decision-path warps per SM (slots per CTA x CTAs per
    // SM); ties to more slots per CTA
    int best = 0;
    c.shot_warps = 1;
    for (int sw = kShotWarps; sw >= 1; --sw) {
      const qd::Layout Ls = lay(sw, false);
      if (Ls.total > (unsigned)optin) continue;
      int blocks = 0;
      QD_CK(qd::decode_occupancy(0, 32 * sw, Ls.total, &blocks));
      if (sw * blocks > best) {
        best = sw * blocks;
        c.shot_warps = sw;
      }
    }
    // the union region in global memory: eight path slots, shared memory for
    // the persistent part only, no pre-BP staging (its copies need shared memory)
    c.Lg = lay(kShotWarps, false);
    c.Lg.pre_stage = 0;
    if (c.Lg.U > (unsigned)optin) {
      set_error(std::string(who) + ": window " + std::to_string(w) + " needs " + std::to_string(c.Lg.U) +
                " B of shared memory even with its path state in global memory (limit " +
                std::to_string(optin) + ")");
      return QD_EUNSUPPORTED;
    }
    int bg = 0;
    QD_CK(qd::decode_occupancy(3, 32 * kShotWarps, c.Lg.U, &bg));
    c.grid_g = std::max(1, bg);
    c.L = lay(c.shot_warps, false);
    c.fits = c.L.total <= (unsigned)optin;
    if (!c.fits) c.L = c.Lg;  // shot mode streams the path state through L2 / HBM
    c.Lp = lay(1, true);
    if (c.Lp.total > (unsigned)optin) c.Lp = lay(1, false);
    c.path_fits = c.Lp.total <= (unsigned)optin;
    // path mode: the largest cluster (8, 4 or 2 CTAs, at most the number of
    // paths) that can be resident, its CTAs splitting the pre-BP of a shot
    c.pcl = 1;
    for (int C = 8; C >= 2 && c.path_fits; C >>= 1) {
      if (C > nb || h.n_rows < 2 * C || h.n_cols < 2 * C) continue;
      int ncl = 0;
      if (qd::path_cluster_occupancy(kPathThreads, c.Lp.total, C, &ncl) != cudaSuccess) {
        (void)cudaGetLastError();
        continue;
      }
      if (ncl >= 1) {
        c.pcl = C;
        break;
      }
    }
    smem_max = std::max<size_t>(smem_max, std::max(c.fits ? c.L.total : c.Lg.U, c.path_fits ? c.Lp.total : 0u));
    int blocks = 0;
    QD_CK(qd::decode_occupancy(c.fits ? 0 : 3, 32 * (c.fits ? c.shot_warps : kShotWarps), c.fits ? c.L.total : c.Lg.U,
                               &blocks));
    c.grid_per_sm = std::max(1, blocks);
  }
  for (size_t w = 0; w < cf.size(); ++w) {
    WinGpu& g = dec->wins[w];
    g.L = cf[w].L;
    g.Lp = cf[w].Lp;
    g.Lg = cf[w].Lg;
    g.grid_g = cf[w].grid_g;
    g.fits = cf[w].fits;
    g.path_fits = cf[w].path_fits;
    g.pcl = cf[w].pcl;
    g.shot_warps = cf[w].fits ? cf[w].shot_warps : kShotWarps;
    g.grid_per_sm = cf[w].grid_per_sm;
  }
  QD_CK_ST(ensure_uscratch(dec, dec->launch_mode == 3));
  // shot mode's snapshot plans (one per window: the first wave is its slot
  // count) and one snapshot pool per resident CTA
  size_t cta_bytes = 0;
  int ctas = 0;
  for (WinGpu& g : dec->wins) {
    const ForkPlan F = fork_plan(dec->kp, dec->dmx, std::max(1, g.L.nslots));
    g.fork_on = F.on;
    g.fork_nodes = F.n_nodes;
    if (!F.on) continue;
    std::vector<int16_t> v(F.order);
    v.insert(v.end(), F.chain.begin(), F.chain.end());
    v.insert(v.end(), F.fnode.begin(), F.fnode.end());
    v.insert(v.end(), F.fdep.begin(), F.fdep.end());
    if (!g.d_fork) QD_CK(cudaMalloc(&g.d_fork, sizeof(int16_t) * (size_t)dec->kp.nb * (3 + dec->dmx)));
    QD_CK(cudaMemcpy(g.d_fork, v.data(), sizeof(int16_t) * v.size(), cudaMemcpyHostToDevice));
    // node snapshots, then one parking snapshot per path
    cta_bytes = std::max(cta_bytes, (size_t)(F.n_nodes + dec->kp.nb) * (qd::kSnapHeaderBytes + g.L.b_size));
    ctas = std::max(ctas, dec->sm_count * std::max(g.grid_per_sm, g.grid_g));
  }
  if (cta_bytes > dec->snap_cta_bytes || ctas > dec->snap_ctas) {
    const size_t cb = std::max(cta_bytes, dec->snap_cta_bytes);
    const int nc = std::max(ctas, dec->snap_ctas);
    cudaFree(dec->d_snap);
    dec->d_snap = nullptr;
    dec->snap_cta_bytes = 0;
    dec->snap_ctas = 0;
    QD_CK(cudaMalloc(&dec->d_snap, cb * nc));
    dec->snap_cta_bytes = cb;
    dec->snap_ctas = nc;
  }
  if (dec->P.reuse_msgs) {  // candidate paths' kept values: one set per resident CTA, or per path-mode shot
    int cmax = 0;
    for (const WinGpu& g : dec->wins) cmax = std::max(cmax, dec->sm_count * std::max(g.grid_per_sm, g.grid_g));
    const size_t slots = std::max<size_t>(cmax, (size_t)std::min<long long>(dec->max_shots, kPathModeMaxShots));
    if (slots > dec->kpath_slots) {
      cudaFree(dec->d_kpath);
      dec->d_kpath = nullptr;
      dec->kpath_slots = 0;
      QD_CK(cudaMalloc(&dec->d_kpath, sizeof(float) * slots * dec->kp.nb * std::max(1, dec->ns_max)));
      dec->kpath_slots = slots;
    }
  }
  dec->smem_max = smem_max;
  dec->hist_on = hist;
  return QD_OK;
}

// Lay the windows out again when the need for the quantised history changes.
qd_status update_hist(qd_decoder* dec, const char* who) {
  const bool want = dec->kp.rkq != nullptr || dec->kp.dump != nullptr;
  if (want == dec->hist_on) return QD_OK;
  return configure_layouts(dec, want, who);
}
}  // namespace

extern "C" {

const char* qd_last_error_message(void) { return qd::g_err.c_str(); }

qd_status qd_build_dem(const qd_bb_code* code, const qd_noise* noise, qd_dem** out) {
  QD_REQ(code && noise && out, "qd_build_dem: null argument");
  QD_REQ(code->l >= 1 && code->m >= 1 && code->l * code->m <= 4096, "qd_build_dem: bad l, m");
  QD_REQ(noise->rounds >= 1 && noise->rounds <= 1000, "qd_build_dem: bad rounds");
  QD_REQ(noise->p > 0.0 && noise->p < 0.5, "qd_build_dem: p outside (0, 0.5)");
  std::unique_ptr<qd_dem> d(new (std::nothrow) qd_dem());
  if (!d) return QD_ENOMEM;
  if (!qd::build_dem_host(*code, *noise, d->h)) return QD_EINVAL;
  for (float l : d->h.col_llr)
    if (!(l > std::ldexp(1.0f, -15) && l < 16.0f)) {
      set_error("qd_build_dem: prior LLR outside (2^-15, 16); Eq. (5) would not be exact");
      return QD_EUNSUPPORTED;
    }
  *out = d.release();
  return QD_OK;
}

qd_status qd_build_dem_code_capacity(const qd_bb_code* code, double p_data, double p_synd, qd_dem** out) {
  QD_REQ(code && out, "qd_build_dem_code_capacity: null argument");
  QD_REQ(code->l >= 1 && code->m >= 1 && code->l * code->m <= 4096, "qd_build_dem_code_capacity: bad l, m");
  QD_REQ(p_data > 0.0 && p_data < 0.5, "qd_build_dem_code_capacity: p_data outside (0, 0.5)");
  QD_REQ(p_synd >= 0.0 && p_synd < 0.5, "qd_build_dem_code_capacity: p_synd outside [0, 0.5)");
  std::unique_ptr<qd_dem> d(new (std::nothrow) qd_dem());
  if (!d) return QD_ENOMEM;
  if (!qd::build_dem_code_capacity(*code, p_data, p_synd, d->h)) return QD_EINVAL;
  for (float l : d->h.col_llr)
    if (!(l > std::ldexp(1.0f, -15) && l < 16.0f)) {
      set_error("qd_build_dem_code_capacity: prior LLR outside (2^-15, 16); Eq. (5) would not be exact");
      return QD_EUNSUPPORTED;
    }
  *out = d.release();
  return QD_OK;
}

qd_status qd_dem_info(const qd_dem* d, qd_dem_info_t* o) {
  QD_REQ(d && o, "qd_dem_info: null argument");
  o->n_det = d->h.n_det;
  o->n_cols = d->h.n_cols;
  o->n_obs = d->h.K;
  o->n_blocks = d->h.R + 1;
  o->w = d->h.w;
  o->det_words = (d->h.n_det + 31) / 32;
  o->n_edges = (int)d->h.col_dets.size();
  return QD_OK;
}

qd_status qd_dem_columns(const qd_dem* d, int* col_ptr, int* col_dets, uint32_t* obs, double* prob,
                         float* llr) {
  QD_REQ(d, "qd_dem_columns: null dem");
  const auto& h = d->h;
  if (col_ptr) std::copy(h.col_ptr.begin(), h.col_ptr.end(), col_ptr);
  if (col_dets) std::copy(h.col_dets.begin(), h.col_dets.end(), col_dets);
  if (obs) std::copy(h.col_obs.begin(), h.col_obs.end(), obs);
  if (prob) std::copy(h.col_p.begin(), h.col_p.end(), prob);
  if (llr) std::copy(h.col_llr.begin(), h.col_llr.end(), llr);
  return QD_OK;
}

qd_status qd_dem_window(const qd_dem* d, int W, int F, int k, int merge_h1, int info[7], int* gcols, int* col_ptr,
                        int* col_rows, float* llr) {
  QD_REQ(d && info, "qd_dem_window: null argument");
  QD_REQ(W >= 1 && F >= 1 && F <= W, "qd_dem_window: need 1 <= F <= W");
  QD_REQ(k >= 0 && k < qd::n_windows(d->h, W, F), "qd_dem_window: window out of range");
  QD_REQ(merge_h1 >= 0 && merge_h1 <= 2, "qd_dem_window: merge_h1 must be 0, 1 or 2");
  qd::WindowHost h;
  if (!qd::build_window(d->h, W, F, k, false, h, merge_h1)) return QD_EINVAL;
  const int v[7] = {h.r0, h.n_blocks, h.n_rows, h.n_cols, h.n_edges, h.n_commit, h.last};
  std::copy(v, v + 7, info);
  if (gcols) {
    std::copy(h.gcols.begin(), h.gcols.end(), gcols);
    std::copy(h.col_ptr.begin(), h.col_ptr.end(), col_ptr);
    std::copy(h.col_rows.begin(), h.col_rows.end(), col_rows);
    std::copy(h.llr.begin(), h.llr.end(), llr);
  }
  return QD_OK;
}

qd_status qd_path_plan(const qd_gdg_params* p, int wave, int info[3], int16_t* order, int16_t* chain, int16_t* fnode,
                       int16_t* fdep) {
  QD_REQ(p && info, "qd_path_plan: null argument");
  QD_REQ(p->k_guess >= 0 && p->k_guess <= 5 && wave >= 1, "qd_path_plan: k_guess outside [0, 5] or wave < 1");
  QD_REQ(p->side_max == 0 || (p->side_max >= p->k_guess && p->side_max <= 32), "qd_path_plan: bad side_max");
  qd::KParams k{};
  k.dmax_main = p->d_max_main;
  k.dmax_other = p->d_max_other;
  k.k = p->k_guess;
  k.low_err = p->low_error_mode;
  k.side_max = p->side_max;
  k.reinit = p->reinit_on_split != 0;
  k.nb = (1 << p->k_guess) + (p->side_max > p->k_guess ? p->side_max - p->k_guess : 0);
  int dmx = 0;
  for (int id = 0; id < k.nb; ++id) dmx = std::max(dmx, qd::path_dmax(k, id, qd::path_split(k, id)));
  const ForkPlan F = fork_plan(k, dmx, wave);
  info[0] = k.nb;
  info[1] = dmx;
  info[2] = F.on ? F.n_nodes : -1;
  if (F.on && order) {
    std::copy(F.order.begin(), F.order.end(), order);
    std::copy(F.chain.begin(), F.chain.end(), chain);
    std::copy(F.fnode.begin(), F.fnode.end(), fnode);
    std::copy(F.fdep.begin(), F.fdep.end(), fdep);
  }
  return QD_OK;
}

qd_status qd_dem_destroy(qd_dem* d) {
  if (!d) return QD_OK;
  if (d->d_thr) {
    cudaFree(d->d_cptr);
    cudaFree(d->d_cdet);
    cudaFree(d->d_cobs);
    cudaFree(d->d_thr);
  }
  delete d;
  return QD_OK;
}

qd_status qd_sample_shots(const qd_dem* d, uint64_t seed, uint64_t shot_offset, int64_t n_shots,
                          uint32_t* det_bits, uint32_t* obs_bits, qd_stream_t stream) {
  QD_REQ(d && det_bits && obs_bits, "qd_sample_shots: null argument");
  QD_REQ(n_shots >= 0, "qd_sample_shots: n_shots < 0");
  if (qd_status st = ensure_device(d)) return st;
  QD_CK(qd::launch_sample((cudaStream_t)stream, d->h.n_cols, d->d_thr, d->d_cptr, d->d_cdet, d->d_cobs,
                          (d->h.n_det + 31) / 32, seed, shot_offset, n_shots, det_bits, obs_bits));
  return QD_OK;
}

qd_status qd_decoder_destroy(qd_decoder* dec) {
  if (!dec) return QD_OK;
  for (auto& w : dec->wins) {
    cudaFree(w.d_graph);
    cudaFree(w.d_ccptr);
    cudaFree(w.d_ccdet);
    cudaFree(w.d_ccobs);
    cudaFree(w.d_wthr);
    cudaFree(w.d_fork);
    cudaFree(w.d_prev);
  }
  cudaFree(dec->d_snap);
  cudaFree(dec->d_keep);
  cudaFree(dec->d_kpath);
  cudaFree(dec->d_work);
  cudaFree(dec->d_uscratch);
  cudaFree(dec->d_ranker);
  cudaFree(dec->d_path_res);
  cudaFree(dec->d_arrive);
  cudaFree(dec->d_counters);
  cudaFree(dec->d_corr);
  cudaFree(dec->d_det);
  cudaFree(dec->d_obs);
  cudaFree(dec->d_pred);
  cudaFree(dec->d_fail);
  cudaFree(dec->d_resid);
  cudaFree(dec->d_nfail);
  delete dec;
  return QD_OK;
}

qd_status qd_decoder_create(const qd_dem* dem, const qd_gdg_params* p, int64_t max_shots,
                            qd_decoder** out) {
  QD_REQ(dem && p && out, "qd_decoder_create: null argument");
  QD_REQ(max_shots >= 1, "qd_decoder_create: max_shots < 1");
  QD_REQ(p->W >= 1 && p->F >= 1 && p->F <= p->W, "qd_decoder_create: need 1 <= F <= W");
  QD_REQ(p->n_pre >= 0 && p->iters_per_step >= 1 && p->d_max_main >= 1 && p->d_max_other >= 1,
         "qd_decoder_create: bad iteration counts");
  QD_REQ(p->alpha > 0.0f && p->clip > 0.0f, "qd_decoder_create: alpha and clip must be positive");
  if (p->iters_per_step < 4 || (p->iters_first != 0 && p->iters_first < 4)) {
    set_error("qd_decoder_create: iters_per_step or iters_first < 4 is not implemented on the GPU");
    return QD_EUNSUPPORTED;
  }
  QD_REQ(p->iters_first >= 0, "qd_decoder_create: iters_first < 0");
  QD_REQ(p->merge_h1 >= 0 && p->merge_h1 <= 2, "qd_decoder_create: merge_h1 must be 0, 1 or 2");
  QD_REQ(p->reuse_msgs == 0 || p->reuse_msgs == 1, "qd_decoder_create: reuse_msgs must be 0 or 1");
  QD_REQ(p->fallback >= 0 && p->fallback <= 2, "qd_decoder_create: fallback must be 0, 1 or 2");
  QD_REQ(p->side_max == 0 || (p->side_max >= p->k_guess && p->side_max <= 32),
         "qd_decoder_create: side_max must be 0 or in [k_guess, 32]");
  QD_REQ(p->d_max_other >= p->k_guess, "qd_decoder_create: d_max_other < k_guess");
  if (p->k_guess < 0 || p->k_guess > 5) {
    set_error("qd_decoder_create: k_guess must be in [0, 5]");
    return QD_EUNSUPPORTED;
  }
  if (qd_status st = ensure_device(dem)) return st;
  std::unique_ptr<qd_decoder> dec(new (std::nothrow) qd_decoder());
  if (!dec) return QD_ENOMEM;
  dec->dem = dem;
  dec->P = *p;
  dec->max_shots = max_shots;
  qd::KParams& k = dec->kp;
  k.alpha = p->alpha;
  k.clip = p->clip;
  k.pa_main = p->pa_main;
  k.pa_other = p->pa_other;
  k.pb_main = p->pb_main;
  k.pb_other = p->pb_other;
  k.pb_d1 = p->pb_d1;
  k.pc = p->pc;
  k.pd = p->pd;
  k.n_pre = p->n_pre;
  k.ips = p->iters_per_step;
  k.ips1 = p->iters_first;
  k.fallback = p->fallback;
  k.dmax_main = p->d_max_main;
  k.dmax_other = p->d_max_other;
  k.k = p->k_guess;
  k.low_err = p->low_error_mode;
  k.peel_init = p->peel_at_init;
  k.pc_max_depth = p->pc_max_depth;
  k.n_unsat_min = p->n_unsat_min;
  k.side_max = p->side_max;
  k.reinit = p->reinit_on_split != 0;
  k.nb = (1 << p->k_guess) + (p->side_max > p->k_guess ? p->side_max - p->k_guess : 0);
  dec->dmx = 0;  // the deepest path, by the kernels' own rule (trace sizing)
  for (int id = 0; id < k.nb; ++id) dec->dmx = std::max(dec->dmx, qd::path_dmax(k, id, qd::path_split(k, id)));

  int dev = 0, optin = 0;
  QD_CK(cudaGetDevice(&dev));
  QD_CK(cudaDeviceGetAttribute(&dec->sm_count, cudaDevAttrMultiProcessorCount, dev));
  QD_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

  const int nwin = qd::n_windows(dem->h, p->W, p->F);
  dec->wins.resize(nwin);
  for (int w = 0; w < nwin; ++w) {
    WinGpu& g = dec->wins[w];
    if (!qd::build_window(dem->h, p->W, p->F, w, p->shorten != 0, g.h, p->merge_h1)) return QD_EINVAL;
    const auto& h = g.h;
    dec->corr_words = std::max(dec->corr_words, (h.n_cols + 31) / 32);
    dec->ns_max = std::max(dec->ns_max, h.n_short);
    dec->sw_max = std::max(dec->sw_max, (h.n_short + 31) / 32);
    // graph arrays in one allocation
    // every array starts on a 16-byte boundary and is padded to a multiple of
    // 16 bytes, as the kernels' bulk (TMA) copies into shared memory require
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    size_t o_cp = 0, o_cr = a16(o_cp + 2 * h.col_ptr.size()), o_rp = a16(o_cr + 2 * h.col_rows.size()),
           o_re = a16(o_rp + 2 * h.row_ptr.size()), o_ll = a16(o_re + 4 * h.row_ent.size()),
           o_vp = a16(o_ll + 4 * h.llr.size()), tot = a16(o_vp + 2 * (size_t)h.n_cols);
    // pre-BP processing order of the variables: descending degree, ties by index
    std::vector<uint16_t> vperm(h.n_cols);
    for (int c = 0; c < h.n_cols; ++c) vperm[c] = (uint16_t)c;
    std::stable_sort(vperm.begin(), vperm.end(), [&](uint16_t a, uint16_t b) {
      return h.col_ptr[a + 1] - h.col_ptr[a] > h.col_ptr[b + 1] - h.col_ptr[b];
    });
    std::vector<char> blob(tot);
    memcpy(blob.data() + o_vp, vperm.data(), 2 * vperm.size());
    memcpy(blob.data() + o_cp, h.col_ptr.data(), 2 * h.col_ptr.size());
    memcpy(blob.data() + o_cr, h.col_rows.data(), 2 * h.col_rows.size());
    memcpy(blob.data() + o_rp, h.row_ptr.data(), 2 * h.row_ptr.size());
    memcpy(blob.data() + o_re, h.row_ent.data(), 4 * h.row_ent.size());
    memcpy(blob.data() + o_ll, h.llr.data(), 4 * h.llr.size());
    QD_CK(cudaMalloc(&g.d_graph, tot));
    QD_CK(cudaMemcpy(g.d_graph, blob.data(), tot, cudaMemcpyHostToDevice));
    char* b = (char*)g.d_graph;
    g.dv = qd::WinDev{h.n_rows, h.n_cols, h.n_edges, h.row0, h.n_short, h.short_edges_max, h.n_rows / h.n_blocks,
                      (const uint16_t*)(b + o_cp), (const uint16_t*)(b + o_cr), (const uint16_t*)(b + o_rp),
                      (const uint32_t*)(b + o_re), (const float*)(b + o_ll), nullptr, 0,
                      (const uint16_t*)(b + o_vp),
                      h.last ? h.n_rows : std::min(h.n_rows, dec->P.F * (h.n_rows / h.n_blocks))};
    // committed columns: their full detector sets and observables
    std::vector<int> cc_ptr(1, 0), cc_det;
    std::vector<uint32_t> cc_obs;
    for (int c = 0; c < h.n_commit; ++c) {
      int gc = h.gcols[c];
      for (int e = dem->h.col_ptr[gc]; e < dem->h.col_ptr[gc + 1]; ++e) cc_det.push_back(dem->h.col_dets[e]);
      cc_ptr.push_back((int)cc_det.size());
      cc_obs.push_back(dem->h.col_obs[gc]);
    }
    QD_CK(upload(&g.d_ccptr, cc_ptr));
    QD_CK(upload(&g.d_ccdet, cc_det));
    QD_CK(upload(&g.d_ccobs, cc_obs));
  }
  dec->smem_optin = optin;
  // the kernels' dynamic shared-memory allowance is the device limit, so
  // decoders of different sizes coexist (the launch asks for what it needs)
  QD_CK(qd::set_decode_smem((size_t)optin));
  if (qd_status st = configure_layouts(dec.get(), false, "qd_decoder_create")) return st;
  dec->trace_bytes = qd::trace_bytes_per_shot(k.nb, dec->dmx, dec->ns_max);
  QD_CK(cudaMalloc(&dec->d_work, sizeof(int) * (nwin + 1)));
  const long long pm_shots = std::min<long long>(max_shots, kPathModeMaxShots);
  QD_CK(cudaMalloc(&dec->d_path_res, qd::path_result_bytes(dec->sw_max) * k.nb * pm_shots));
  QD_CK(cudaMalloc(&dec->d_arrive, sizeof(int) * pm_shots));
  QD_CK(cudaMemset(dec->d_arrive, 0, sizeof(int) * pm_shots));
  QD_CK(cudaMalloc(&dec->d_counters, sizeof(long long) * kCounters));
  QD_CK(cudaMemset(dec->d_counters, 0, sizeof(long long) * kCounters));
  const int dw = (dem->h.n_det + 31) / 32;
  QD_CK(cudaMalloc(&dec->d_corr, sizeof(uint32_t) * (size_t)max_shots * dec->corr_words));
  QD_CK(cudaMalloc(&dec->d_det, sizeof(uint32_t) * (size_t)max_shots * dw));
  QD_CK(cudaMalloc(&dec->d_obs, sizeof(uint32_t) * (size_t)max_shots));
  QD_CK(cudaMalloc(&dec->d_pred, sizeof(uint32_t) * (size_t)max_shots));
  QD_CK(cudaMalloc(&dec->d_fail, sizeof(uint32_t) * (size_t)max_shots));
  QD_CK(cudaMalloc(&dec->d_resid, sizeof(uint32_t) * (size_t)max_shots));
  QD_CK(cudaMalloc(&dec->d_nfail, sizeof(long long)));
  if (p->reuse_msgs) {
    for (const WinGpu& g : dec->wins) dec->keep_ld = std::max(dec->keep_ld, g.h.n_cols);
    QD_CK(cudaMalloc(&dec->d_keep, sizeof(float) * (size_t)max_shots * std::max(1, dec->keep_ld)));
    for (int w = 1; w < nwin; ++w) {
      const auto& a = dec->wins[w - 1].h;
      const auto& b = dec->wins[w].h;
      if (!a.n_cols || !b.n_cols) continue;  // nothing kept across a window without columns
      std::vector<int> at(dem->h.n_cols, -1);
      for (int c = 0; c < a.n_cols; ++c) at[a.gcols[c]] = c;  // a repeated DEM column: its last column
      std::vector<int16_t> prev(b.n_cols);
      for (int c = 0; c < b.n_cols; ++c) prev[c] = (int16_t)at[b.gcols[c]];
      QD_CK(upload(&dec->wins[w].d_prev, prev));
    }
  }
  *out = dec.release();
  return QD_OK;
}

qd_status qd_decoder_n_windows(const qd_decoder* dec, int* n) {
  QD_REQ(dec && n, "null argument");
  *n = (int)dec->wins.size();
  return QD_OK;
}

qd_status qd_decoder_path_info(const qd_decoder* dec, int out[2]) {
  QD_REQ(dec && out, "null argument");
  out[0] = dec->kp.nb;
  out[1] = dec->dmx;
  return QD_OK;
}

qd_status qd_decoder_corr_words(const qd_decoder* dec, int* cw) {
  QD_REQ(dec && cw, "null argument");
  *cw = dec->corr_words;
  return QD_OK;
}

qd_status qd_decoder_trace_bytes(const qd_decoder* dec, size_t* b) {
  QD_REQ(dec && b, "null argument");
  *b = dec->trace_bytes;
  return QD_OK;
}

qd_status qd_window_info(const qd_decoder* dec, int k, qd_window_info_t* o, int* gcols) {
  QD_REQ(dec && o, "null argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_window_info: window out of range");
  const auto& h = dec->wins[k].h;
  *o = qd_window_info_t{h.r0, h.n_blocks, h.n_rows, h.n_cols, h.n_edges, h.n_commit, h.last, h.n_short};
  if (gcols) std::copy(h.gcols.begin(), h.gcols.end(), gcols);
  return QD_OK;
}

}  // extern "C"

namespace {
// message reuse buffers for window g (keep = nullptr: off)
qd::ReuseDev reuse_dev(const qd_decoder* dec, const WinGpu& g) {
  qd::ReuseDev R{};
  if (!dec->d_keep) return R;
  R.keep = dec->d_keep;
  R.keep_ld = dec->keep_ld;
  R.prev = g.d_prev;
  R.kpath = dec->d_kpath;
  return R;
}

// shot mode's snapshot plan of window g (pool = nullptr: none, or turned off)
qd::ForkDev fork_dev(const qd_decoder* dec, const WinGpu& g) {
  qd::ForkDev F{};
  // the candidate dump records path 0's every step, so path 0 runs from the root
  if (!dec->fork_on || !g.fork_on || !dec->d_snap || dec->kp.dump) return F;
  const int nb = dec->kp.nb;
  F.order = g.d_fork;
  F.chain = g.d_fork + nb;
  F.fnode = F.chain + (size_t)nb * dec->dmx;
  F.fdep = F.fnode + nb;
  F.pool = dec->d_snap;
  F.cta_bytes = dec->snap_cta_bytes;
  F.n_nodes = g.fork_nodes;
  F.pool_ctas = dec->snap_ctas;
  F.sched = dec->sched_on ? 1 : 0;
  return F;
}
}  // namespace

extern "C" {

qd_status qd_decode_windows(qd_decoder* dec, int k, const uint32_t* det_bits, int64_t n_shots,
                            uint32_t* win_correction, int32_t* status, void* trace, qd_stream_t stream) {
  QD_REQ(dec && det_bits && win_correction, "qd_decode_windows: null argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_decode_windows: window out of range");
  QD_REQ(n_shots >= 0 && n_shots <= dec->max_shots, "qd_decode_windows: n_shots outside [0, max_shots]");
  if (n_shots == 0) return QD_OK;
  const WinGpu& g = dec->wins[k];
  cudaStream_t st = (cudaStream_t)stream;
  const int dw = (dec->dem->h.n_det + 31) / 32;
  if (g.h.n_cols == 0) {
    // a window without columns decides nothing (the commit tests its residue)
    QD_CK(cudaMemsetAsync(win_correction, 0, sizeof(uint32_t) * (size_t)n_shots * dec->corr_words, st));
    if (status) QD_CK(cudaMemsetAsync(status, 0xFF, sizeof(int32_t) * (size_t)n_shots, st));
    return QD_OK;
  }
  // the path state in global memory when the window does not fit shared memory
  // (or on request); otherwise path mode while a batch leaves most SMs idle
  const bool global = !g.fits || dec->launch_mode == 3;
  bool path_mode = dec->launch_mode == 2;
  if (dec->launch_mode == 0) path_mode = n_shots * 4 <= dec->sm_count;
  if (path_mode && (n_shots > std::min<long long>(dec->max_shots, kPathModeMaxShots) || !g.path_fits || global))
    path_mode = false;
  const qd::ForkDev fk = fork_dev(dec, g);
  const qd::ReuseDev ru = reuse_dev(dec, g);
  if (global) {
    QD_CK(cudaMemsetAsync(dec->d_work + k, 0, sizeof(int), st));
    const long long grid = std::min<long long>(n_shots, (long long)dec->sm_count * g.grid_g);
    QD_CK(qd::launch_decode(0, (int)grid, 32 * kShotWarps, g.Lg.U, st, dec->kp, g.dv, g.Lg, det_bits, dw, n_shots,
                            win_correction, dec->corr_words, status, (char*)trace, dec->trace_bytes, dec->dmx,
                            dec->ns_max, dec->d_work + k, dec->d_counters, nullptr, nullptr, dec->sw_max,
                            dec->d_uscratch, g.Lg.total - g.Lg.U, 1, 1, &fk, &ru));
    return QD_OK;
  }
  if (path_mode) {
    const int cps = (dec->kp.nb + g.pcl - 1) / g.pcl * g.pcl;
    QD_CK(qd::launch_decode(1, (int)(n_shots * cps), kPathThreads, g.Lp.total, st, dec->kp, g.dv, g.Lp, det_bits,
                            dw, n_shots, win_correction, dec->corr_words, status, (char*)trace, dec->trace_bytes,
                            dec->dmx, dec->ns_max, nullptr, dec->d_counters, dec->d_path_res, dec->d_arrive,
                            dec->sw_max, nullptr, 0, cps, g.pcl, nullptr, &ru));
    return QD_OK;
  }
  QD_CK(cudaMemsetAsync(dec->d_work + k, 0, sizeof(int), st));
  const long long grid = std::min<long long>(n_shots, (long long)dec->sm_count * g.grid_per_sm);
  QD_CK(qd::launch_decode(0, (int)grid, 32 * g.shot_warps, g.L.total, st, dec->kp, g.dv, g.L, det_bits, dw,
                          n_shots, win_correction, dec->corr_words, status, (char*)trace, dec->trace_bytes,
                          dec->dmx, dec->ns_max, dec->d_work + k, dec->d_counters, nullptr, nullptr, dec->sw_max,
                          nullptr, 0, 1, 1, &fk, &ru));
  return QD_OK;
}

qd_status qd_commit_and_slide(qd_decoder* dec, int k, const uint32_t* win_correction, int64_t n_shots,
                              uint32_t* det_bits, uint32_t* obs_pred, uint32_t* residue_fail,
                              qd_stream_t stream) {
  QD_REQ(dec && win_correction && det_bits && obs_pred && residue_fail, "qd_commit_and_slide: null argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_commit_and_slide: window out of range");
  QD_REQ(n_shots >= 0, "qd_commit_and_slide: n_shots < 0");
  const WinGpu& g = dec->wins[k];
  const int w = dec->dem->h.w;
  QD_CK(qd::launch_commit((cudaStream_t)stream, g.h.n_commit, g.d_ccptr, g.d_ccdet, g.d_ccobs,
                          dec->corr_words, win_correction, n_shots, det_bits, (dec->dem->h.n_det + 31) / 32,
                          obs_pred, residue_fail, g.h.r0 * w, g.h.commit_b1 * w));
  return QD_OK;
}

qd_status qd_evaluate(const uint32_t* obs_pred, const uint32_t* obs_true, const uint32_t* residue_fail,
                      int64_t n_shots, uint32_t* fail, long long* n_fail, qd_stream_t stream) {
  QD_REQ(obs_pred && obs_true && residue_fail, "qd_evaluate: null argument");
  QD_REQ(n_shots >= 0, "qd_evaluate: n_shots < 0");
  QD_CK(qd::launch_evaluate((cudaStream_t)stream, obs_pred, obs_true, residue_fail, n_shots, fail, n_fail));
  return QD_OK;
}

qd_status qd_decode_all(qd_decoder* dec, uint32_t* det_bits, const uint32_t* obs_true, int64_t n_shots,
                        uint32_t* obs_pred, uint32_t* fail, long long* n_fail, qd_stream_t stream) {
  QD_REQ(dec && det_bits && obs_true && obs_pred, "qd_decode_all: null argument");
  QD_REQ(n_shots >= 0 && n_shots <= dec->max_shots, "qd_decode_all: n_shots outside [0, max_shots]");
  if (n_shots == 0) return QD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  QD_CK(cudaMemsetAsync(obs_pred, 0, sizeof(uint32_t) * n_shots, st));
  QD_CK(cudaMemsetAsync(dec->d_resid, 0, sizeof(uint32_t) * n_shots, st));
  for (int k = 0; k < (int)dec->wins.size(); ++k) {
    qd_status s = qd_decode_windows(dec, k, det_bits, n_shots, dec->d_corr, nullptr, nullptr, stream);
    if (s != QD_OK) return s;
    s = qd_commit_and_slide(dec, k, dec->d_corr, n_shots, det_bits, obs_pred, dec->d_resid, stream);
    if (s != QD_OK) return s;
  }
  return qd_evaluate(obs_pred, obs_true, dec->d_resid, n_shots, fail, n_fail, stream);
}

qd_status qd_decode_shots_host(qd_decoder* dec, const uint32_t* det_bits, const uint32_t* obs_true,
                               int64_t n_shots, uint32_t* obs_pred, uint32_t* fail, long long* n_fail,
                               qd_stream_t stream) {
  QD_REQ(dec && det_bits && obs_true, "qd_decode_shots_host: null argument");
  QD_REQ(n_shots >= 0 && n_shots <= dec->max_shots, "qd_decode_shots_host: n_shots outside [0, max_shots]");
  if (n_shots == 0) return QD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t dw = (dec->dem->h.n_det + 31) / 32;
  QD_CK(cudaMemcpyAsync(dec->d_det, det_bits, sizeof(uint32_t) * dw * n_shots, cudaMemcpyHostToDevice, st));
  QD_CK(cudaMemcpyAsync(dec->d_obs, obs_true, sizeof(uint32_t) * n_shots, cudaMemcpyHostToDevice, st));
  QD_CK(cudaMemsetAsync(dec->d_nfail, 0, sizeof(long long), st));
  qd_status s = qd_decode_all(dec, dec->d_det, dec->d_obs, n_shots, dec->d_pred, dec->d_fail, dec->d_nfail, stream);
  if (s != QD_OK) return s;
  if (obs_pred)
    QD_CK(cudaMemcpyAsync(obs_pred, dec->d_pred, sizeof(uint32_t) * n_shots, cudaMemcpyDeviceToHost, st));
  if (fail) QD_CK(cudaMemcpyAsync(fail, dec->d_fail, sizeof(uint32_t) * n_shots, cudaMemcpyDeviceToHost, st));
  if (n_fail) QD_CK(cudaMemcpyAsync(n_fail, dec->d_nfail, sizeof(long long), cudaMemcpyDeviceToHost, st));
  QD_CK(cudaStreamSynchronize(st));
  return QD_OK;
}

qd_status qd_decoder_set_weights(qd_decoder* dec, int k, const float* w, int T) {
  QD_REQ(dec, "null argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_decoder_set_weights: window out of range");
  QD_REQ(w == nullptr || T >= 1, "qd_decoder_set_weights: T must be >= 1");
  const float* old_w = dec->wins[k].dv.wts;
  const int old_t = dec->wins[k].dv.wT;
  dec->wins[k].dv.wts = w;
  dec->wins[k].dv.wT = w ? T : 0;
  // the layouts keep the shortened edges' full-window ids only while some
  // window has learned weights
  bool want = false;
  for (const WinGpu& g : dec->wins) want = want || g.dv.wts != nullptr;
  if (want != dec->lw_on) {
    dec->lw_on = want;
    if (qd_status st = configure_layouts(dec, dec->hist_on, "qd_decoder_set_weights")) {
      dec->wins[k].dv.wts = old_w;
      dec->wins[k].dv.wT = old_t;
      dec->lw_on = !want;
      return st;
    }
  }
  return QD_OK;
}

qd_status qd_decoder_set_ranker(qd_decoder* dec, const float* params) {
  QD_REQ(dec, "null argument");
  if (!params) {
    dec->kp.rkq = nullptr;
    dec->kp.rkb = nullptr;
    return update_hist(dec, "qd_decoder_set_ranker");
  }
  // the grids of the exact first layer (the same rule as the reference model)
  auto grid = [](float x, float scale, float lim) {
    float v = std::rint(x * scale);
    v = v > lim ? lim : (v < -lim ? -lim : v);
    return v / scale;
  };
  std::vector<float> q(644, 0.0f);
  for (int i = 0; i < 641; ++i)
    QD_REQ(std::isfinite(params[i]), "qd_decoder_set_ranker: non-finite parameter");
  for (int i = 0; i < 512; ++i) q[i] = grid(params[i], 64.0f, 128.0f);
  for (int u = 0; u < 64; ++u) q[512 + u] = grid(params[512 + u], 128.0f, 65536.0f);
  for (int u = 0; u < 64; ++u) q[576 + u] = grid(params[576 + u], 64.0f, 128.0f);
  q[640] = params[640];
  std::vector<uint32_t> frag(256);
  for (int t = 0; t < 8; ++t)
    for (int lane = 0; lane < 32; ++lane) {
      const int u = 8 * t + lane / 4, kk = 2 * (lane % 4);
      uint32_t lo, hi;
      memcpy(&lo, &q[u * 8 + kk], 4);
      memcpy(&hi, &q[u * 8 + kk + 1], 4);
      frag[32 * t + lane] = (lo >> 16) | (hi & 0xFFFF0000u);  // exact: 7 significant bits
    }
  if (!dec->d_ranker) QD_CK(cudaMalloc(&dec->d_ranker, 644 * 4 + 256 * 4));
  QD_CK(cudaMemcpy(dec->d_ranker, q.data(), 644 * 4, cudaMemcpyHostToDevice));
  QD_CK(cudaMemcpy((char*)dec->d_ranker + 644 * 4, frag.data(), 256 * 4, cudaMemcpyHostToDevice));
  const float* old_q = dec->kp.rkq;
  const uint32_t* old_b = dec->kp.rkb;
  dec->kp.rkq = (const float*)dec->d_ranker;
  dec->kp.rkb = (const uint32_t*)((char*)dec->d_ranker + 644 * 4);
  if (qd_status st = update_hist(dec, "qd_decoder_set_ranker")) {
    dec->kp.rkq = old_q;
    dec->kp.rkb = old_b;
    return st;
  }
  return QD_OK;
}

qd_status qd_decoder_set_dump(qd_decoder* dec, void* records, int* count, int capacity) {
  QD_REQ(dec, "null argument");
  QD_REQ(!records || (count && capacity >= 0), "qd_decoder_set_dump: need count and capacity >= 0");
  dec->kp.dump = (qd::RankRec*)records;
  dec->kp.dump_n = records ? count : nullptr;
  dec->kp.dump_cap = records ? capacity : 0;
  if (qd_status st = update_hist(dec, "qd_decoder_set_dump")) {
    dec->kp.dump = nullptr;
    dec->kp.dump_n = nullptr;
    dec->kp.dump_cap = 0;
    return st;
  }
  return QD_OK;
}

qd_status qd_decoder_launch_info(const qd_decoder* dec, int k, int out[8]) {
  QD_REQ(dec && out, "null argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_decoder_launch_info: window out of range");
  const WinGpu& g = dec->wins[k];
  out[0] = (int)g.L.total;
  out[1] = 32 * g.shot_warps;
  out[2] = g.grid_per_sm;
  out[3] = (int)g.Lp.total;
  out[4] = kPathThreads;
  out[5] = dec->sm_count;
  out[6] = g.pcl;
  out[7] = (dec->kp.nb + g.pcl - 1) / g.pcl * g.pcl;
  return QD_OK;
}

qd_status qd_decoder_set_launch(qd_decoder* dec, int mode) {
  QD_REQ(dec, "null argument");
  QD_REQ(mode >= 0 && mode <= 3, "qd_decoder_set_launch: mode must be 0, 1, 2 or 3");
  if (mode == 3) QD_CK_ST(ensure_uscratch(dec, true));
  dec->launch_mode = mode;
  return QD_OK;
}

qd_status qd_decoder_counters(qd_decoder* dec, long long out[5]) {
  QD_REQ(dec && out, "null argument");
  QD_CK(cudaMemcpy(out, dec->d_counters, sizeof(long long) * 5, cudaMemcpyDeviceToHost));
  return QD_OK;
}

qd_status qd_decoder_counters_ex(qd_decoder* dec, long long* out, int n) {
  QD_REQ(dec && out, "null argument");
  QD_REQ(n >= 1 && n <= kCounters, "qd_decoder_counters_ex: n outside [1, 8]");
  QD_CK(cudaMemcpy(out, dec->d_counters, sizeof(long long) * n, cudaMemcpyDeviceToHost));
  return QD_OK;
}

qd_status qd_decoder_set_fork(qd_decoder* dec, int on) {
  QD_REQ(dec, "null argument");
  QD_REQ(on >= 0 && on <= 2, "qd_decoder_set_fork: on must be 0, 1 or 2");
  dec->fork_on = on != 0;
  dec->sched_on = on == 2;
  return QD_OK;
}

qd_status qd_decoder_reset_counters(qd_decoder* dec, qd_stream_t stream) {
  QD_REQ(dec, "null argument");
  QD_CK(cudaMemsetAsync(dec->d_counters, 0, sizeof(long long) * kCounters, (cudaStream_t)stream));
  return QD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free decode + commit (qd_decode_commit_static).
//
// The per-shot window corrections and the work-queue counter that
// qd_decode_windows / qd_commit_and_slide keep in decoder-owned or
// caller-owned device buffers live here in one fixed array that is part of
// the library image.  Every GPU that loads the library holds these
// QD_STATIC_SCRATCH_BYTES until the process exits.
namespace {
constexpr size_t kStaticScratchBytes = QD_STATIC_SCRATCH_BYTES;
constexpr size_t kStaticHeader = 256;  // the work counter, then padding to the corrections' alignment
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[256] = {};  // device address of g_static_scratch, per device ordinal

// The array's name in host code is only a host-side stand-in; the device
// address must come from the runtime, once per device, with that device current.
qd_status static_scratch_address(void** out) {
  int dev = 0;
  QD_CK(cudaGetDevice(&dev));
  QD_REQ(dev >= 0 && dev < 256, "qd_decode_commit_static: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    QD_CK(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return QD_OK;
}
}  // namespace

extern "C" qd_status qd_decode_commit_static(qd_decoder* dec, int k, uint32_t* det_bits, int64_t n_shots,
                                             uint32_t* obs_pred, uint32_t* residue_fail,
                                             qd_stream_t stream) {
  QD_REQ(dec && det_bits && obs_pred && residue_fail, "qd_decode_commit_static: null argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_decode_commit_static: window out of range");
  QD_REQ(n_shots >= 0, "qd_decode_commit_static: n_shots < 0");
  const size_t need = kStaticHeader + sizeof(uint32_t) * (size_t)n_shots * dec->corr_words;
  if (need > kStaticScratchBytes) {
    set_error("qd_decode_commit_static: " + std::to_string(n_shots) + " shots need " +
              std::to_string(need) + " B of static scratch, more than the library's fixed " +
              std::to_string(kStaticScratchBytes) + " B; use at most " +
              std::to_string((kStaticScratchBytes - kStaticHeader) / (sizeof(uint32_t) * dec->corr_words)) +
              " shots per call");
    return QD_EINVAL;
  }
  if (n_shots == 0) return QD_OK;
  QD_REQ(!dec->d_keep || n_shots <= dec->max_shots, "qd_decode_commit_static: n_shots > max_shots with message reuse");
  void* base = nullptr;
  if (qd_status st = static_scratch_address(&base)) return st;
  int* work = (int*)base;
  uint32_t* corr = (uint32_t*)((char*)base + kStaticHeader);
  const WinGpu& g = dec->wins[k];
  const qd::ReuseDev ru = reuse_dev(dec, g);
  cudaStream_t st = (cudaStream_t)stream;
  const int dw = (dec->dem->h.n_det + 31) / 32;
  if (g.h.n_cols > 0) {
    // the launch shape qd_decode_windows would take; every buffer it needs
    // besides the corrections and the work counter was allocated with the
    // decoder (path results and arrival counters, global union regions), and
    // the work counters go to the decoder's own (qd_decoder_counters)
    const bool global = !g.fits || dec->launch_mode == 3;
    bool path_mode = dec->launch_mode == 2;
    if (dec->launch_mode == 0) path_mode = n_shots * 4 <= dec->sm_count;
    if (path_mode && (n_shots > std::min<long long>(dec->max_shots, kPathModeMaxShots) || !g.path_fits || global))
      path_mode = false;
    if (path_mode) {
      const int cps = (dec->kp.nb + g.pcl - 1) / g.pcl * g.pcl;
      QD_CK(qd::launch_decode(1, (int)(n_shots * cps), kPathThreads, g.Lp.total, st, dec->kp, g.dv, g.Lp, det_bits,
                              dw, n_shots, corr, dec->corr_words, nullptr, nullptr, 0, dec->dmx, dec->ns_max, nullptr,
                              dec->d_counters, dec->d_path_res, dec->d_arrive, dec->sw_max, nullptr, 0, cps, g.pcl,
                              nullptr, &ru));
    } else {
      // the array keeps the previous call's contents: the work counter restarts at 0
      QD_CK(cudaMemsetAsync(work, 0, sizeof(int), st));
      const qd::ForkDev fk = fork_dev(dec, g);
      const qd::Layout& L = global ? g.Lg : g.L;
      const long long grid =
          std::min<long long>(n_shots, (long long)dec->sm_count * (global ? g.grid_g : g.grid_per_sm));
      QD_CK(qd::launch_decode(0, (int)grid, 32 * (global ? kShotWarps : g.shot_warps), global ? L.U : L.total, st,
                              dec->kp, g.dv, L, det_bits, dw, n_shots, corr, dec->corr_words, nullptr, nullptr, 0,
                              dec->dmx, dec->ns_max, work, dec->d_counters, nullptr, nullptr, dec->sw_max,
                              global ? dec->d_uscratch : nullptr, global ? L.total - L.U : 0, 1, 1, &fk, &ru));
    }
  }
  const int w = dec->dem->h.w;
  QD_CK(qd::launch_commit(st, g.h.n_commit, g.d_ccptr, g.d_ccdet, g.d_ccobs, dec->corr_words, corr, n_shots,
                          det_bits, dw, obs_pred, residue_fail, g.h.r0 * w, g.h.commit_b1 * w));
  return QD_OK;
}

// ---------------------------------------------------------------------------
// Batched window steps over several decoders (codes / window sizes).
struct qd_batch {
  std::vector<qd_decoder*> mem;
  int n_steps = 0, sm_count = 0, optin = 0;
  size_t budget2 = 0;  // dynamic shared bytes that leave room for two CTAs per SM
  struct Step {
    int warps = 1, blocks = 1;
    size_t budget = 0, smem = 0;
    unsigned q_off = 0;
    std::vector<qd::Layout> L;  // per member (unused where the member has no such window)
  };
  std::vector<Step> steps;
  int* d_work = nullptr;  // one counter per step
  std::vector<qd::ForkDev> forks;  // per member: the current step's path-scheduling plan
};

namespace {
// CTAs of `warps` warps with at most `budget` bytes of dynamic shared memory:
// each member's layout takes as many path slots (<= warps) as fit.
qd_status batch_plan(qd_batch* b, int j, int warps, size_t budget) {
  qd_batch::Step S;
  S.L.assign(b->mem.size(), qd::Layout{});
  unsigned mx = 0;
  for (size_t i = 0; i < b->mem.size(); ++i) {
    const qd_decoder* d = b->mem[i];
    if (j >= (int)d->wins.size()) continue;
    const auto& h = d->wins[j].h;
    int s = warps;
    for (; s >= 1; --s) {
      S.L[i] = qd::make_layout(h.n_rows, h.n_cols, h.n_edges, h.n_short, h.short_edges_max, d->kp.nb, s, false,
                               d->hist_on, d->lw_on);
      if (qd::al16(S.L[i].total) + 32 <= budget) break;
    }
    if (s < 1) {
      set_error("qd_batch: member " + std::to_string(i) + " window " + std::to_string(j) + " needs " +
                std::to_string(S.L[i].total + 32) + " B of shared memory with one path slot (budget " +
                std::to_string(budget) + ")");
      return QD_EUNSUPPORTED;
    }
    mx = std::max(mx, S.L[i].total);
  }
  S.q_off = qd::al16(mx);
  S.smem = S.q_off + 32;  // work slot, then the staging mbarrier and its flag
  S.warps = warps;
  S.budget = budget;
  int blocks = 0;
  QD_CK(qd::batch_occupancy(32 * warps, S.smem, &blocks));
  S.blocks = std::max(1, blocks);
  b->steps[j] = S;
  return QD_OK;
}

// The member table of step j; returns the number of members with work.
int batch_members(qd_batch* b, int j, uint32_t* const* det, const int64_t* n, uint32_t* const* obs_pred,
                  uint32_t* const* resid, std::vector<qd::BatchMember>& out) {
  out.clear();
  // heavier windows first, so the tail of the persistent launch is short
  std::vector<int> order;
  for (size_t i = 0; i < b->mem.size(); ++i)
    if (j < (int)b->mem[i]->wins.size() && n[i] > 0) order.push_back((int)i);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->mem[x]->wins[j].h.n_edges > b->mem[y]->wins[j].h.n_edges;
  });
  for (int i : order) {
    qd_decoder* d = b->mem[i];
    const WinGpu& g = d->wins[j];
    qd::BatchMember m{};
    m.P = &d->kp;
    m.W = &g.dv;
    m.L = &b->steps[j].L[i];
    m.det = det[i];
    m.det_words = (d->dem->h.n_det + 31) / 32;
    m.n = n[i];
    m.corr = d->d_corr;
    m.corr_words = d->corr_words;
    m.dmx = d->dmx;
    m.ns_max = d->ns_max;
    m.sw_max = d->sw_max;
    m.counters = d->d_counters;
    m.n_commit = g.h.n_commit;
    m.cptr = g.d_ccptr;
    m.cdet = g.d_ccdet;
    m.cobs = g.d_ccobs;
    m.obs_pred = obs_pred ? obs_pred[i] : nullptr;
    m.resid = resid ? resid[i] : nullptr;
    const int w = d->dem->h.w;
    m.b0 = g.h.r0 * w;
    m.b1 = g.h.commit_b1 * w;
    b->forks.resize(b->mem.size());
    b->forks[i] = fork_dev(d, g);
    m.fork = &b->forks[i];
    out.push_back(m);
  }
  return (int)out.size();
}

qd_status batch_decode(qd_batch* b, int j, const std::vector<qd::BatchMember>& all, cudaStream_t st) {
  const qd_batch::Step& S = b->steps[j];
  // windows without columns decide nothing; their commits still test the residue
  std::vector<qd::BatchMember> m;
  for (const auto& x : all)
    if (x.W->n_cols > 0) m.push_back(x);
  if (m.empty()) return QD_OK;
  long long tot = 0;
  for (const auto& x : m) tot += x.n;
  QD_CK(cudaMemsetAsync(b->d_work + j, 0, sizeof(int), st));
  const long long grid = std::min<long long>(tot, (long long)b->sm_count * S.blocks);
  QD_CK(qd::launch_decode_batch(st, (int)grid, 32 * S.warps, S.smem, S.q_off, b->d_work + j, m.data(),
                                (int)m.size()));
  return QD_OK;
}
}  // namespace

extern "C" {

qd_status qd_batch_create(qd_decoder* const* members, int n_members, qd_batch** out) {
  QD_REQ(members && out, "qd_batch_create: null argument");
  QD_REQ(n_members >= 1 && n_members <= qd::kMaxBatch,
         "qd_batch_create: need 1 <= n_members <= " + std::to_string(qd::kMaxBatch));
  std::unique_ptr<qd_batch> b(new (std::nothrow) qd_batch());
  if (!b) return QD_ENOMEM;
  for (int i = 0; i < n_members; ++i) {
    QD_REQ(members[i], "qd_batch_create: null member");
    if (members[i]->P.reuse_msgs) {
      set_error("qd_batch_create: message reuse between windows is not supported in batched steps");
      return QD_EUNSUPPORTED;
    }
    b->mem.push_back(members[i]);
    b->n_steps = std::max(b->n_steps, (int)members[i]->wins.size());
  }
  int dev = 0;
  QD_CK(cudaGetDevice(&dev));
  QD_CK(cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev));
  QD_CK(cudaDeviceGetAttribute(&b->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  QD_CK(qd::set_decode_smem((size_t)b->optin));
  int per_sm = 0, reserved = 0;
  QD_CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  QD_CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  b->budget2 = (size_t)std::max(0, per_sm / 2 - reserved);
  b->steps.resize(b->n_steps);
  // default shape: 8 warps, two CTAs per SM when every member fits a slot
  for (int j = 0; j < b->n_steps; ++j)
    if (batch_plan(b.get(), j, kShotWarps, b->budget2) != QD_OK)
      QD_CK_ST(batch_plan(b.get(), j, kShotWarps, (size_t)b->optin));
  QD_CK(cudaMalloc(&b->d_work, sizeof(int) * std::max(1, b->n_steps)));
  *out = b.release();
  return QD_OK;
}

qd_status qd_batch_destroy(qd_batch* b) {
  if (!b) return QD_OK;
  cudaFree(b->d_work);
  delete b;
  return QD_OK;
}

qd_status qd_batch_n_steps(const qd_batch* b, int* n) {
  QD_REQ(b && n, "null argument");
  *n = b->n_steps;
  return QD_OK;
}

qd_status qd_batch_set_shape(qd_batch* b, int step, int warps, int ctas_per_sm) {
  QD_REQ(b, "null argument");
  QD_REQ(step >= 0 && step < b->n_steps, "qd_batch_set_shape: step out of range");
  QD_REQ(warps >= 1 && warps <= kShotWarps, "qd_batch_set_shape: warps must be in [1, 8]");
  QD_REQ(ctas_per_sm == 1 || ctas_per_sm == 2, "qd_batch_set_shape: ctas_per_sm must be 1 or 2");
  const qd_batch::Step keep = b->steps[step];
  if (qd_status st = batch_plan(b, step, warps, ctas_per_sm == 2 ? b->budget2 : (size_t)b->optin)) {
    b->steps[step] = keep;
    return st;
  }
  return QD_OK;
}

qd_status qd_batch_info(const qd_batch* b, int step, int out[4]) {
  QD_REQ(b && out, "null argument");
  QD_REQ(step >= 0 && step < b->n_steps, "qd_batch_info: step out of range");
  const auto& S = b->steps[step];
  out[0] = S.warps;
  out[1] = (int)S.smem;
  out[2] = S.blocks;
  int active = 0;
  for (auto* d : b->mem) active += step < (int)d->wins.size();
  out[3] = active;
  return QD_OK;
}

qd_status qd_batch_step(qd_batch* b, int step, uint32_t* const* det_bits, const int64_t* n_shots,
                        uint32_t* const* obs_pred, uint32_t* const* residue_fail, qd_stream_t stream) {
  QD_REQ(b && det_bits && n_shots && obs_pred && residue_fail, "qd_batch_step: null argument");
  QD_REQ(step >= 0 && step < b->n_steps, "qd_batch_step: step out of range");
  for (size_t i = 0; i < b->mem.size(); ++i) {
    QD_REQ(n_shots[i] >= 0 && n_shots[i] <= b->mem[i]->max_shots,
           "qd_batch_step: n_shots of member " + std::to_string(i) + " outside [0, max_shots]");
    QD_REQ(n_shots[i] == 0 || (det_bits[i] && obs_pred[i] && residue_fail[i]),
           "qd_batch_step: null buffer of member " + std::to_string(i));
  }
  std::vector<qd::BatchMember> m;
  if (!batch_members(b, step, det_bits, n_shots, obs_pred, residue_fail, m)) return QD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (qd_status s = batch_decode(b, step, m, st)) return s;
  QD_CK(qd::launch_commit_batch(st, m.data(), (int)m.size()));
  return QD_OK;
}

qd_status qd_batch_autotune(qd_batch* b, int step, uint32_t* const* det_bits, const int64_t* n_shots, int reps,
                            qd_stream_t stream, float* best_ms) {
  QD_REQ(b && det_bits && n_shots, "qd_batch_autotune: null argument");
  QD_REQ(step >= 0 && step < b->n_steps, "qd_batch_autotune: step out of range");
  QD_REQ(reps >= 1, "qd_batch_autotune: reps < 1");
  for (size_t i = 0; i < b->mem.size(); ++i)
    QD_REQ(n_shots[i] >= 0 && n_shots[i] <= b->mem[i]->max_shots, "qd_batch_autotune: n_shots outside range");
  std::vector<qd::BatchMember> m;
  if (!batch_members(b, step, det_bits, n_shots, nullptr, nullptr, m)) return QD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  QD_CK(cudaEventCreate(&e0));
  QD_CK(cudaEventCreate(&e1));
  const qd_batch::Step keep = b->steps[step];
  float best = 0.0f;
  int pick_w = 0;
  size_t pick_b = 0;
  qd_status st_out = QD_OK;
  const size_t budgets[2] = {b->budget2, (size_t)b->optin};
  for (int w = kShotWarps; w >= 4 && st_out == QD_OK; --w)
    for (size_t bud : budgets) {
      if (batch_plan(b, step, w, bud) != QD_OK) continue;
      // the member table points at this step's layouts, which batch_plan rebuilt
      batch_members(b, step, det_bits, n_shots, nullptr, nullptr, m);
      if ((st_out = batch_decode(b, step, m, st)) != QD_OK) break;  // warm-up
      cudaError_t e = cudaEventRecord(e0, st);
      for (int r = 0; r < reps && e == cudaSuccess; ++r)
        if ((st_out = batch_decode(b, step, m, st)) != QD_OK) break;
      if (st_out != QD_OK) break;
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        set_error(std::string("qd_batch_autotune: ") + cudaGetErrorString(e));
        st_out = QD_ECUDA;
        break;
      }
      ms /= reps;
      if (!pick_w || ms < best) {
        best = ms;
        pick_w = w;
        pick_b = bud;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st_out != QD_OK || !pick_w) {
    b->steps[step] = keep;
    return st_out;
  }
  QD_CK_ST(batch_plan(b, step, pick_w, pick_b));
  if (best_ms) *best_ms = best;
  return QD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned weighted min-sum: training on window samples.
struct qd_wms {
  qd::WmsGraph G{};
  int k = 0;
  uint32_t* d_thr = nullptr;
  float* d_scratch = nullptr;
  size_t scratch_per_cta = 0;
  int* d_work = nullptr;
  int grid = 0;
  size_t smem = 0;
};

extern "C" {

qd_status qd_wms_create(const qd_decoder* dec, int k, int T, int ckpt, qd_wms** out) {
  QD_REQ(dec && out, "qd_wms_create: null argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_wms_create: window out of range");
  QD_REQ(T >= 1 && T <= 1000 && ckpt >= 1 && ckpt <= T, "qd_wms_create: need 1 <= ckpt <= T");
  std::unique_ptr<qd_wms> m(new (std::nothrow) qd_wms());
  if (!m) return QD_ENOMEM;
  const WinGpu& g = dec->wins[k];
  m->k = k;
  m->G = qd::WmsGraph{g.h.n_rows, g.h.n_cols, g.h.n_edges, (g.h.n_rows + 31) / 32, T, ckpt,
                      g.dv.col_ptr, g.dv.col_rows, g.dv.row_ptr, g.dv.row_ent, g.dv.llr, dec->P.clip};
  std::vector<uint32_t> thr(g.h.n_cols);
  for (int c = 0; c < g.h.n_cols; ++c) thr[c] = dec->dem->h.col_thr[g.h.gcols[c]];
  QD_CK(upload(&m->d_thr, thr));
  m->smem = qd::wms_smem_bytes(m->G.ne, m->G.nc, m->G.rw);
  int optin = 0, dev = 0;
  QD_CK(cudaGetDevice(&dev));
  QD_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (m->smem > (size_t)optin) {
    set_error("qd_wms_create: window too large for shared memory");
    return QD_EUNSUPPORTED;
  }
  QD_CK(qd::wms_set_smem(m->smem));
  int blocks = 0;
  QD_CK(qd::wms_occupancy(m->smem, &blocks));
  m->grid = dec->sm_count * std::max(1, blocks);
  m->scratch_per_cta = qd::wms_scratch_per_cta(m->G.ne, T, ckpt);
  QD_CK(cudaMalloc(&m->d_scratch, sizeof(float) * m->scratch_per_cta * m->grid));
  QD_CK(cudaMalloc(&m->d_work, sizeof(int)));
  *out = m.release();
  return QD_OK;
}

qd_status qd_wms_destroy(qd_wms* m) {
  if (!m) return QD_OK;
  cudaFree(m->d_thr);
  cudaFree(m->d_scratch);
  cudaFree(m->d_work);
  delete m;
  return QD_OK;
}

qd_status qd_wms_info(const qd_wms* m, int out[6]) {
  QD_REQ(m && out, "null argument");
  out[0] = m->G.nr;
  out[1] = m->G.nc;
  out[2] = m->G.ne;
  out[3] = m->G.T;
  out[4] = m->G.ckpt;
  out[5] = m->G.rw;
  return QD_OK;
}

qd_status qd_wms_sample(qd_wms* m, uint64_t seed, uint64_t offset, int64_t n, uint32_t* synd, qd_stream_t stream) {
  QD_REQ(m && synd && n >= 0, "qd_wms_sample: bad argument");
  QD_CK(qd::launch_wms_sample((cudaStream_t)stream, m->G, m->d_thr, seed, offset, n, 1u + (unsigned)m->k, synd,
                              nullptr, 0, 0, nullptr, 0));
  return QD_OK;
}

static qd_status wms_run(qd_wms* m, const float* w, const uint32_t* synd, int64_t n, int backward, float scale,
                         float* grad_w, float* loss, float* post, qd_stream_t stream) {
  QD_REQ(m && w && synd && n >= 0, "qd_wms: bad argument");
  if (n == 0) return QD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  QD_CK(cudaMemsetAsync(m->d_work, 0, sizeof(int), st));
  const int grid = (int)std::min<long long>(n, m->grid);
  QD_CK(qd::launch_wms(st, grid, m->smem, m->G, w, synd, n, backward, scale, grad_w, loss, post, m->d_scratch,
                       m->scratch_per_cta, m->d_work));
  return QD_OK;
}

qd_status qd_wms_loss(qd_wms* m, const float* w, const uint32_t* synd, int64_t n, float* loss, float* post,
                      qd_stream_t stream) {
  QD_REQ(loss, "qd_wms_loss: loss is required");
  return wms_run(m, w, synd, n, 0, 0.0f, nullptr, loss, post, stream);
}

qd_status qd_wms_grad(qd_wms* m, const float* w, const uint32_t* synd, int64_t n, float grad_scale, float* grad_w,
                      float* loss, qd_stream_t stream) {
  QD_REQ(grad_w, "qd_wms_grad: grad_w is required");
  return wms_run(m, w, synd, n, 1, grad_scale, grad_w, loss, nullptr, stream);
}

qd_status qd_window_sample(qd_decoder* dec, int k, uint64_t seed, uint64_t offset, int64_t n, uint32_t* det_bits,
                           uint32_t* fault_bits, qd_stream_t stream) {
  QD_REQ(dec && det_bits && n >= 0, "qd_window_sample: bad argument");
  QD_REQ(k >= 0 && k < (int)dec->wins.size(), "qd_window_sample: window out of range");
  WinGpu& g = dec->wins[k];
  if (!g.d_wthr) {
    std::vector<uint32_t> thr(g.h.n_cols);
    for (int c = 0; c < g.h.n_cols; ++c) thr[c] = dec->dem->h.col_thr[g.h.gcols[c]];
    QD_CK(upload(&g.d_wthr, thr));
  }
  const qd::WmsGraph G{g.h.n_rows, g.h.n_cols, g.h.n_edges, (g.h.n_rows + 31) / 32, 1, 1,
                       g.dv.col_ptr, g.dv.col_rows, g.dv.row_ptr, g.dv.row_ent, g.dv.llr, dec->P.clip};
  QD_CK(qd::launch_wms_sample((cudaStream_t)stream, G, g.d_wthr, seed, offset, n, 1u + (unsigned)k, nullptr,
                              det_bits, (dec->dem->h.n_det + 31) / 32, g.h.row0, fault_bits, dec->corr_words));
  return QD_OK;
}

qd_status qd_ranker_eval(const float* params, const void* records, const uint8_t* labels, int64_t n, int quantize,
                         float pos_weight, float grad_scale, float* grad, float* loss, float* score,
                         qd_stream_t stream) {
  QD_REQ(params && records && n >= 0, "qd_ranker_eval: bad argument");
  QD_REQ(!(grad || loss) || labels, "qd_ranker_eval: labels are required for grad and loss");
  QD_CK(qd::launch_ranker((cudaStream_t)stream, params, (const qd::RankRec*)records, labels, n, quantize,
                          pos_weight, grad_scale, grad, loss, score));
  return QD_OK;
}

qd_status qd_adam_step(float* w, const float* g, float* m1, float* m2, int64_t n, float lr, float beta1, float beta2,
                       float eps, int step, qd_stream_t stream) {
  QD_REQ(w && g && m1 && m2 && n >= 0 && step >= 1, "qd_adam_step: bad argument");
  QD_CK(qd::launch_adam((cudaStream_t)stream, w, g, m1, m2, n, lr, beta1, beta2, eps, step));
  return QD_OK;
}

}  // extern "C"
