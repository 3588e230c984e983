// dem_host.cpp -- detector error model and window matrices of libqdec (host).
//
// Circuit: Z-basis memory experiment of a BB code with the depth-8 syndrome
// cycle of Bravyi et al. (Fig. 7 there; cited in Sec. III), R noisy rounds and
// a noiseless data readout (appendix "Stim circuit implementation").  Per round
// (X-check ancilla Xi, Z-check ancilla Zi, L/R data, A = A1+A2+A3,
// B = B1+B2+B3, a term Mk maps check i to data i + shift(Mk)):
//   layer 1: RX(Xi)            CNOT(R[i - a1] -> Zi)      L idle
//   layer 2: CNOT(Xi -> L[i+a2])  CNOT(R[i - a3] -> Zi)
//   layer 3: CNOT(Xi -> R[i+b2])  CNOT(L[i - b1] -> Zi)
//   layer 4: CNOT(Xi -> R[i+b1])  CNOT(L[i - b2] -> Zi)
//   layer 5: CNOT(Xi -> R[i+b3])  CNOT(L[i - b3] -> Zi)
//   layer 6: CNOT(Xi -> L[i+a1])  CNOT(R[i - a2] -> Zi)
//   layer 7: CNOT(Xi -> L[i+a3])  MZ(Zi)                  R idle
//   layer 8: MRX(Xi)              RZ(Zi) (not after R)    L, R idle
// Noise of rate p (Sec. II): DEPOLARIZE2 after each CNOT (X patterns XI, IX,
// XX at 4p/15 each), DEPOLARIZE1 on idle data (X at 2p/3), X flip p after
// each Z reset (data and Z ancillas before round 1) and before each Z
// measurement.  Only the X part of a fault is visible to the Z-basis
// experiment (Sec. II, X and Z decoded separately).
//
// Method: one BACKWARD sweep.  eff[q] is the set of detectors and observables
// an X on qubit q flips when injected at the current point of the circuit.  At
// the end it is the readout's contribution (final-block detectors H_Z d and
// logical observables L_Z d); walking back, CNOT(c,t) gives
// eff[c] ^= eff[t], a Z measurement adds its two detectors (blocks r-1 and r
// of its check), a reset clears eff[q].  A noise location reads off eff of its
// qubit(s).  Mechanisms with identical (detectors, observables) merge as
// independent flips (Sec. II-B), p <- p(1-q) + q(1-p) in ascending q; the
// prior is Lambda = log((1-p)/p) (Sec. II-A).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>

#include "qdec_internal.h"

namespace qd {
namespace {

struct Group {
  int l, m;
  int idx(int a, int b) const { return (((a % l) + l) % l) * m + (((b % m) + m) % m); }
  int add(int i, int a, int b) const { return idx(i / m + a, i % m + b); }
};

// ---- GF(2) helpers on 64-bit word bitsets ----
struct Bits {
  int n = 0;
  std::vector<uint64_t> w;
  explicit Bits(int n_ = 0) : n(n_), w((n_ + 63) / 64, 0) {}
  bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
  void flip(int i) { w[i >> 6] ^= 1ull << (i & 63); }
  void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
  void x(const Bits& o) {
    for (size_t k = 0; k < w.size(); ++k) w[k] ^= o.w[k];
  }
  bool any() const {
    for (uint64_t v : w)
      if (v) return true;
    return false;
  }
  int lowest() const {
    for (size_t k = 0; k < w.size(); ++k)
      if (w[k]) return (int)(k * 64 + __builtin_ctzll(w[k]));
    return -1;
  }
};

// Canonical logical-Z basis: the reduced-row-echelon kernel basis of H_X
// (free columns ascending, v = e_f + sum of the pivots whose row has a 1 in
// column f), keeping each vector that is independent of rowspace(H_Z) plus
// the vectors already kept.
std::vector<Bits> logical_z(const std::vector<Bits>& HX, const std::vector<Bits>& HZ, int n) {
  std::vector<Bits> R = HX;
  std::vector<int> pivcol;
  int rank = 0;
  for (int c = 0; c < n && rank < (int)R.size(); ++c) {
    int p = -1;
    for (int r = rank; r < (int)R.size(); ++r)
      if (R[r].get(c)) { p = r; break; }
    if (p < 0) continue;
    std::swap(R[p], R[rank]);
    for (int r = 0; r < (int)R.size(); ++r)
      if (r != rank && R[r].get(c)) R[r].x(R[rank]);
    pivcol.push_back(c);
    ++rank;
  }
  std::vector<char> is_piv(n, 0);
  for (int c : pivcol) is_piv[c] = 1;
  // echelon basis keyed by lowest set bit
  std::vector<Bits> basis;
  std::vector<int> lead;
  auto reduce = [&](Bits v) {
    bool changed = true;
    while (changed && v.any()) {
      changed = false;
      int lo = v.lowest();
      for (size_t b = 0; b < basis.size(); ++b)
        if (lead[b] == lo) { v.x(basis[b]); changed = true; break; }
    }
    return v;
  };
  auto insert = [&](const Bits& v) {
    Bits r = reduce(v);
    if (!r.any()) return false;
    basis.push_back(r);
    lead.push_back(r.lowest());
    return true;
  };
  for (const Bits& z : HZ) insert(z);
  std::vector<Bits> out;
  for (int f = 0; f < n; ++f) {
    if (is_piv[f]) continue;
    Bits v(n);
    v.set(f);
    for (int r = 0; r < rank; ++r)
      if (R[r].get(f)) v.set(pivcol[r]);
    if (insert(v)) out.push_back(v);
  }
  return out;
}

enum OpT { CNOT, MZ, RZ, RX, MRX, NOISE2, NOISE1, XFLIP };
struct Op {
  OpT t;
  int a, b;  // qubits; for MZ: b = detector id of block r-1 for this check
};

struct Mech {
  std::vector<int> dets;
  uint32_t obs;
  double p;
};

bool mech_key_less(const Mech& x, const Mech& y) {
  if (x.dets != y.dets) return std::lexicographical_compare(x.dets.begin(), x.dets.end(),
                                                            y.dets.begin(), y.dets.end());
  return x.obs < y.obs;
}
bool mech_key_eq(const Mech& x, const Mech& y) { return x.dets == y.dets && x.obs == y.obs; }

// H_X = [A|B], H_Z = [B^T|A^T] as bitsets over the 2w data qubits (L then R).
void code_matrices(const qd_bb_code& code, std::vector<Bits>& HX, std::vector<Bits>& HZ) {
  const Group G{code.l, code.m};
  const int w = code.l * code.m, n = 2 * w;
  HX.assign(w, Bits(n));
  HZ.assign(w, Bits(n));
  for (int i = 0; i < w; ++i)
    for (int k = 0; k < 3; ++k) {
      HX[i].flip(G.add(i, code.a_x[k], code.a_y[k]));
      HX[i].flip(w + G.add(i, code.b_x[k], code.b_y[k]));
      HZ[i].flip(G.add(i, -code.b_x[k], -code.b_y[k]));
      HZ[i].flip(w + G.add(i, -code.a_x[k], -code.a_y[k]));
    }
}

// Merge mechanisms with identical (detectors, observables) as independent
// flips, p <- p(1-q) + q(1-p) in ascending q (Sec. II-B), in canonical column
// order (detector lists lexicographically, then observables); the prior is
// Lambda = log((1-p)/p) (Sec. II-A) and the sampling threshold round(p 2^32).
void finish_columns(std::vector<Mech>& mechs, DemHost& D) {
  std::sort(mechs.begin(), mechs.end(), [](const Mech& x, const Mech& y) {
    if (!mech_key_eq(x, y)) return mech_key_less(x, y);
    return x.p < y.p;
  });
  D.col_ptr.assign(1, 0);
  D.col_dets.clear();
  D.col_obs.clear();
  D.col_p.clear();
  D.col_llr.clear();
  D.col_thr.clear();
  for (size_t a = 0; a < mechs.size();) {
    size_t b = a;
    double pm = 0.0;
    while (b < mechs.size() && mech_key_eq(mechs[a], mechs[b])) {
      double q = mechs[b].p;
      pm = pm * (1.0 - q) + q * (1.0 - pm);
      ++b;
    }
    D.col_dets.insert(D.col_dets.end(), mechs[a].dets.begin(), mechs[a].dets.end());
    D.col_ptr.push_back((int)D.col_dets.size());
    D.col_obs.push_back(mechs[a].obs);
    D.col_p.push_back(pm);
    D.col_llr.push_back((float)std::log((1.0 - pm) / pm));
    double t = std::floor(pm * 4294967296.0 + 0.5);
    D.col_thr.push_back(t >= 4294967295.0 ? 0xFFFFFFFFu : (t <= 0.0 ? 0u : (uint32_t)t));
    a = b;
  }
  D.n_cols = (int)D.col_obs.size();
}

}  // namespace

bool build_dem_host(const qd_bb_code& code, const qd_noise& noise, DemHost& D) {
  const Group G{code.l, code.m};
  const int w = code.l * code.m, n = 2 * w, R = noise.rounds;
  const double p = noise.p;
  D.code = code;
  D.noise = noise;
  D.w = w;
  D.R = R;
  D.n_det = (R + 1) * w;
  const int XA = 0, LD = w, RD = 2 * w, ZA = 3 * w, NQ = 4 * w;
  auto a_sh = [&](int k) { return std::make_pair(code.a_x[k], code.a_y[k]); };
  auto b_sh = [&](int k) { return std::make_pair(code.b_x[k], code.b_y[k]); };
  auto fwd = [&](int i, std::pair<int, int> s) { return G.add(i, s.first, s.second); };
  auto bwd = [&](int i, std::pair<int, int> s) { return G.add(i, -s.first, -s.second); };

  std::vector<Bits> HX, HZ;
  code_matrices(code, HX, HZ);
  std::vector<Bits> LZ = logical_z(HX, HZ, n);
  D.K = (int)LZ.size();
  if (D.K > 32) {
    set_error("more than 32 logical qubits");
    return false;
  }

  // ---- circuit, forward order ----
  std::vector<Op> ops;
  for (int q = 0; q < n; ++q) {
    ops.push_back({RZ, LD + q, 0});
    ops.push_back({XFLIP, LD + q, 0});
  }
  for (int i = 0; i < w; ++i) {
    ops.push_back({RZ, ZA + i, 0});
    ops.push_back({XFLIP, ZA + i, 0});
  }
  for (int r = 1; r <= R; ++r) {
    for (int i = 0; i < w; ++i) ops.push_back({RX, XA + i, 0});
    for (int i = 0; i < w; ++i) {
      int c = RD + bwd(i, a_sh(0));
      ops.push_back({CNOT, c, ZA + i});
      ops.push_back({NOISE2, c, ZA + i});
    }
    for (int i = 0; i < w; ++i) ops.push_back({NOISE1, LD + i, 0});
    struct { int xa; bool xb; int zk; bool za; } lay[6] = {
        {1, false, 2, true}, {1, true, 0, false}, {0, true, 1, false},
        {2, true, 2, false}, {0, false, 1, true}, {2, false, -1, false}};
    for (int t = 0; t < 6; ++t) {
      for (int i = 0; i < w; ++i) {
        int tgt = lay[t].xb ? RD + fwd(i, b_sh(lay[t].xa)) : LD + fwd(i, a_sh(lay[t].xa));
        ops.push_back({CNOT, XA + i, tgt});
        ops.push_back({NOISE2, XA + i, tgt});
      }
      if (lay[t].zk >= 0) {
        for (int i = 0; i < w; ++i) {
          int c = lay[t].za ? RD + bwd(i, a_sh(lay[t].zk)) : LD + bwd(i, b_sh(lay[t].zk));
          ops.push_back({CNOT, c, ZA + i});
          ops.push_back({NOISE2, c, ZA + i});
        }
      } else {
        for (int i = 0; i < w; ++i) {
          ops.push_back({XFLIP, ZA + i, 0});
          ops.push_back({MZ, ZA + i, (r - 1) * w + i});
        }
        for (int i = 0; i < w; ++i) ops.push_back({NOISE1, RD + i, 0});
      }
    }
    for (int i = 0; i < w; ++i) ops.push_back({MRX, XA + i, 0});
    if (r < R)
      for (int i = 0; i < w; ++i) {
        ops.push_back({RZ, ZA + i, 0});
        ops.push_back({XFLIP, ZA + i, 0});
      }
    for (int q = 0; q < n; ++q) ops.push_back({NOISE1, LD + q, 0});
  }

  // ---- backward sweep ----
  const int NB = D.n_det + D.K;
  std::vector<Bits> eff(NQ, Bits(NB));
  for (int q = 0; q < n; ++q) {
    for (int i = 0; i < w; ++i)
      if (HZ[i].get(q)) eff[LD + q].flip(R * w + i);
    for (int k = 0; k < D.K; ++k)
      if (LZ[k].get(q)) eff[LD + q].flip(D.n_det + k);
  }
  std::vector<Mech> mechs;
  auto emit = [&](const Bits& e, double pr) {
    Mech mm;
    mm.obs = 0;
    mm.p = pr;
    for (int b = 0; b < D.n_det; ++b)
      if (e.get(b)) mm.dets.push_back(b);
    for (int k = 0; k < D.K; ++k)
      if (e.get(D.n_det + k)) mm.obs |= 1u << k;
    if (mm.dets.empty() && mm.obs == 0) return;
    mechs.push_back(std::move(mm));
  };
  const double p2 = 4.0 * p / 15.0, p1 = 2.0 * p / 3.0;
  for (int k = (int)ops.size() - 1; k >= 0; --k) {
    const Op& o = ops[k];
    switch (o.t) {
      case CNOT: eff[o.a].x(eff[o.b]); break;
      case MZ:
        eff[o.a].flip(o.b);
        eff[o.a].flip(o.b + w);
        break;
      case RZ: case RX: case MRX: eff[o.a] = Bits(NB); break;
      case NOISE2: {
        Bits both = eff[o.a];
        both.x(eff[o.b]);
        emit(eff[o.a], p2);
        emit(eff[o.b], p2);
        emit(both, p2);
        break;
      }
      case NOISE1: emit(eff[o.a], p1); break;
      case XFLIP: emit(eff[o.a], p); break;
    }
  }

  finish_columns(mechs, D);
  return true;
}


// Code-capacity models of the appendices, decoded with H_X: BSC(pd) on the
// data qubits (block 0: H_X e) and, with ps > 0, BSC(ps) on the syndrome bits
// as one virtual column per check ([H_X | I]) plus a noiseless block 1 holding
// H_X e of the data error alone, whose Eq. (11) residue after the commit is
// the appendix's success test.  Observables: the logical operators such
// errors flip (kernel of H_Z modulo the row span of H_X).
bool build_dem_code_capacity(const qd_bb_code& code, double pd, double ps, DemHost& D) {
  const int w = code.l * code.m, n = 2 * w;
  D.code = code;
  D.noise = qd_noise{pd, 0};
  D.w = w;
  D.R = ps > 0.0 ? 1 : 0;
  D.n_det = (D.R + 1) * w;
  std::vector<Bits> HX, HZ;
  code_matrices(code, HX, HZ);
  std::vector<Bits> LX = logical_z(HZ, HX, n);
  D.K = (int)LX.size();
  if (D.K > 32) {
    set_error("more than 32 logical qubits");
    return false;
  }
  std::vector<Mech> mechs;
  for (int q = 0; q < n; ++q) {
    Mech m;
    m.obs = 0;
    m.p = pd;
    for (int b = 0; b <= D.R; ++b)
      for (int j = 0; j < w; ++j)
        if (HX[j].get(q)) m.dets.push_back(b * w + j);
    for (int k = 0; k < D.K; ++k)
      if (LX[k].get(q)) m.obs |= 1u << k;
    mechs.push_back(std::move(m));
  }
  if (ps > 0.0)
    for (int j = 0; j < w; ++j) mechs.push_back(Mech{{j}, 0u, ps});
  finish_columns(mechs, D);
  return true;
}

int n_windows(const DemHost& d, int W, int F) {
  const int B = d.R + 1;
  int k = 0;
  for (int r = 0;; r += F, ++k)
    if (r + W >= B) return k + 1;
}

namespace {
// Probability that an odd number of the independent mechanisms fire, folded
// in ascending (probability, column) order as the DEM's columns are.
double odd_probability(std::vector<std::pair<double, int>> v) {
  std::sort(v.begin(), v.end());
  double pm = 0.0;
  for (const auto& x : v) pm = pm * (1.0 - x.first) + x.first * (1.0 - pm);
  return pm;
}
}  // namespace

// The H_1 merge of Sec. III on window o (not the last window, W > F, so the
// merged columns are never committed).  H_1 = the window columns that reach
// past its last block, seen on the window's rows (all in the last block).
// merge = 1: the H_1 columns of each equal restriction become one column at
// the first one's place, with the odd-count probability of the class;
// merge = 2: all H_1 columns are replaced by one column per detector t of
// the last block (t ascending), probability the odd count of the H_1 columns
// whose restriction holds t.
static void merge_h1(const DemHost& d, int merge, int r1, WindowHost& o) {
  const int hi = r1 * d.w, last0 = (r1 - 1) * d.w - o.row0;
  const int nc = (int)o.gcols.size();  // (n_cols is set after the merge)
  std::vector<char> ext(nc, 0);
  for (int c = 0; c < nc; ++c) {
    const int g = o.gcols[c];
    ext[c] = d.col_dets[d.col_ptr[g + 1] - 1] >= hi;  // detectors ascend: the last one decides
  }
  auto rows_of = [&](int c) {
    return std::vector<uint16_t>(o.col_rows.begin() + o.col_ptr[c], o.col_rows.begin() + o.col_ptr[c + 1]);
  };
  std::vector<int> gcols;
  std::vector<uint16_t> cptr{0}, crows;
  std::vector<float> llr;
  std::map<std::vector<uint16_t>, std::vector<std::pair<double, int>>> cls;  // restriction -> members
  if (merge == 1)
    for (int c = 0; c < nc; ++c)
      if (ext[c]) cls[rows_of(c)].push_back({d.col_p[o.gcols[c]], o.gcols[c]});
  std::set<std::vector<uint16_t>> seen;
  for (int c = 0; c < nc; ++c) {
    float l = o.llr[c];
    if (ext[c]) {
      if (merge == 2) continue;
      const std::vector<uint16_t> r = rows_of(c);
      if (!seen.insert(r).second) continue;  // folded into its class's first column
      const double pm = odd_probability(cls[r]);
      l = (float)std::log((1.0 - pm) / pm);
    }
    gcols.push_back(o.gcols[c]);
    const std::vector<uint16_t> r = rows_of(c);
    crows.insert(crows.end(), r.begin(), r.end());
    cptr.push_back((uint16_t)crows.size());
    llr.push_back(l);
  }
  if (merge == 2)
    for (int t = 0; t < d.w; ++t) {
      std::vector<std::pair<double, int>> members;
      int rep = -1;
      for (int c = 0; c < nc; ++c) {
        if (!ext[c]) continue;
        for (int e = o.col_ptr[c]; e < o.col_ptr[c + 1]; ++e)
          if (o.col_rows[e] == last0 + t) {
            members.push_back({d.col_p[o.gcols[c]], o.gcols[c]});
            if (rep < 0) rep = o.gcols[c];
          }
      }
      if (members.empty()) continue;
      const double pm = odd_probability(members);
      gcols.push_back(rep);
      crows.push_back((uint16_t)(last0 + t));
      cptr.push_back((uint16_t)crows.size());
      llr.push_back((float)std::log((1.0 - pm) / pm));
    }
  o.gcols = gcols;
  o.col_ptr = cptr;
  o.col_rows = crows;
  o.llr = llr;
}

bool build_window(const DemHost& d, int W, int F, int k, bool shorten, WindowHost& o, int merge) {
  const int B = d.R + 1, w = d.w;
  o = WindowHost();
  o.k = k;
  o.r0 = k * F;
  o.last = (o.r0 + W >= B);
  const int r1 = o.last ? B : o.r0 + W;
  o.n_blocks = r1 - o.r0;
  o.n_rows = o.n_blocks * w;
  o.row0 = o.r0 * w;
  o.commit_b1 = o.last ? r1 : o.r0 + F;
  o.col_ptr.push_back(0);
  bool committing = true;
  for (int c = 0; c < d.n_cols; ++c) {
    const int a = d.col_ptr[c], b = d.col_ptr[c + 1];
    if (a == b) continue;  // undetectable: never decoded
    const int fb = d.col_dets[a] / w;
    if (fb < o.r0 || fb >= r1) continue;
    const bool com = o.last || fb < o.r0 + F;
    if (com && !committing) {
      set_error("committed columns are not a prefix of the window");
      return false;
    }
    committing = com;
    if (com) o.n_commit++;
    o.gcols.push_back(c);
    for (int e = a; e < b; ++e)
      if (d.col_dets[e] < r1 * w) o.col_rows.push_back((uint16_t)(d.col_dets[e] - o.row0));
    o.col_ptr.push_back((uint16_t)o.col_rows.size());
    o.llr.push_back(d.col_llr[c]);
  }
  if (merge && !o.last && W > F) merge_h1(d, merge, r1, o);
  for (float l : o.llr)
    if (!(l > std::ldexp(1.0f, -15) && l < 16.0f)) {
      set_error("window prior LLR outside (2^-15, 16); Eq. (5) would not be exact");
      return false;
    }
  o.n_cols = (int)o.gcols.size();
  o.n_edges = (int)o.col_rows.size();
  // 16-bit edge ids; row and column ids below 2^15, as the decoder packs
  // (index << 16) | label into one positive int for its tie-breaks
  if (o.n_edges >= 65535 || o.n_rows >= 32768 || o.n_cols >= 32768) {
    set_error("window larger than 16-bit edge / 15-bit node indices");
    return false;
  }
  o.row_ptr.assign(o.n_rows + 1, 0);
  for (uint16_t r : o.col_rows) o.row_ptr[r + 1]++;
  for (int j = 0; j < o.n_rows; ++j) o.row_ptr[j + 1] += o.row_ptr[j];
  std::vector<int> fill(o.row_ptr.begin(), o.row_ptr.end() - 1);
  o.row_ent.assign(o.n_edges, 0);
  for (int c = 0; c < o.n_cols; ++c)
    for (int e = o.col_ptr[c]; e < o.col_ptr[c + 1]; ++e)
      o.row_ent[fill[o.col_rows[e]]++] = (uint32_t)e | ((uint32_t)c << 16);
  o.n_short = (shorten && o.n_cols > 2 * o.n_rows) ? 2 * o.n_rows : o.n_cols;
  std::vector<int> deg(o.n_cols);
  for (int c = 0; c < o.n_cols; ++c) deg[c] = o.col_ptr[c + 1] - o.col_ptr[c];
  std::sort(deg.begin(), deg.end(), std::greater<int>());
  o.short_edges_max = 0;
  for (int c = 0; c < o.n_short; ++c) o.short_edges_max += deg[c];
  return true;
}

}  // namespace qd
