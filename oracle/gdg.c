/*
 * gdg.c -- CPU ORACLE (test infrastructure only): BP guided decimation
 * guessing (GDG) and the (W,F) sliding-window driver, written step by step in
 * the paper's order with explicit per-edge messages.
 *
 *   Eq. (1)        min-sum CN update (normalised by alpha, Sec. II-A)
 *   Eq. (2)-(3)    posterior and VN->CN messages, clipped to [-50, 50]
 *                  ("Do not waste guesses", Sec. IV)
 *   Eq. (4)        hard decision, early stop once H e = s
 *   Eq. (5)        path metric
 *   Sec. II-A      decimation: inactive VNs keep stale messages that their
 *                  CNs ignore; decimating to 1 flips the neighbours' syndromes
 *   Alg. 1         SELECT-VN on the four-iteration LLR history
 *   Alg. 3         aggressive decimation outside the low-error mode
 *   Sec. IV        peeling of degree-one CNs after each decimation step;
 *                  a contradiction kills the path (appendix "GDG implementation")
 *   Alg. 2, Fig. 2 decision paths; here the 2^k guessing tree: at depth D <= k
 *                  the branch takes bit (k-D) of its id (most significant
 *                  first) as b and decimates to b + (-1)^b f
 *   Sec. III       pre-BP on the full window, ranking by the sum of the last
 *                  four posteriors (ascending, ties by column index), GDG on
 *                  the first 2w' columns; commit and syndrome update Eq. (10);
 *                  success = Eq. (11) and Eq. (12)
 *
 * Readings where the paper is silent are marked READING and listed in the
 * design notes.  FP32 throughout, compiled with -ffp-contract=off.
 */
#include "qdo.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

int qdo__w(const qdo_dem* d);
int qdo__ncols(const qdo_dem* d);
int qdo__ndet(const qdo_dem* d);
int qdo__R(const qdo_dem* d);
const int* qdo__col_ptr(const qdo_dem* d);
const int* qdo__col_dets(const qdo_dem* d);
const uint32_t* qdo__col_obs(const qdo_dem* d);
const float* qdo__col_llr(const qdo_dem* d);

enum { BR_CONVERGED = 0, BR_MAXDEPTH = 1, BR_CONTRADICTION = 2, BR_NOCAND = 3 };

/* Tanner graph: CSC with ascending rows; CSR lists CSC edge ids. */
typedef struct {
  int nr, nc, ne;
  int *col_ptr, *col_rows;
  int *row_ptr, *row_edges;
  int *edge_col;
  float* llr;
  int* vdeg; /* static column weight */
  /* learned weights: w[(t-1) * wE + efull[e]] for iteration t (NULL: alpha) */
  const float* w;
  int wT, wE;
  const int* efull; /* edge -> full-window edge (NULL: identity) */
  int* vblock;      /* block (round) of the column's first detector in the window */
  const int* wcol;  /* column -> window column (NULL: identity) */
} graph_t;

/* The CN->VN multiplier of Eq. (1) at iteration t for edge e: alpha, or the
 * learned weight w[min(t, T)][e] of the full-window edge. */
static inline float edge_weight(const graph_t* g, float alpha, int t, int e) {
  if (!g->w) return alpha;
  int tt = t < g->wT ? t : g->wT;
  int ef = g->efull ? g->efull[e] : e;
  return g->w[(size_t)(tt - 1) * g->wE + ef];
}

static void graph_init(graph_t* g, int nr, int nc, const int* col_ptr, const int* col_rows,
                       const float* llr) {
  g->nr = nr;
  g->nc = nc;
  g->ne = col_ptr[nc];
  g->col_ptr = malloc(sizeof(int) * (nc + 1));
  memcpy(g->col_ptr, col_ptr, sizeof(int) * (nc + 1));
  g->col_rows = malloc(sizeof(int) * (g->ne > 0 ? g->ne : 1));
  memcpy(g->col_rows, col_rows, sizeof(int) * g->ne);
  g->llr = malloc(sizeof(float) * (nc > 0 ? nc : 1));
  memcpy(g->llr, llr, sizeof(float) * nc);
  g->row_ptr = calloc(nr + 1, sizeof(int));
  g->row_edges = malloc(sizeof(int) * (g->ne > 0 ? g->ne : 1));
  g->edge_col = malloc(sizeof(int) * (g->ne > 0 ? g->ne : 1));
  g->vdeg = malloc(sizeof(int) * (nc > 0 ? nc : 1));
  g->w = NULL;
  g->wT = 0;
  g->wE = 0;
  g->efull = NULL;
  g->wcol = NULL;
  g->vblock = calloc(nc > 0 ? nc : 1, sizeof(int));
  for (int e = 0; e < g->ne; ++e) g->row_ptr[col_rows[e] + 1]++;
  for (int j = 0; j < nr; ++j) g->row_ptr[j + 1] += g->row_ptr[j];
  int* fill = malloc(sizeof(int) * (nr > 0 ? nr : 1));
  memcpy(fill, g->row_ptr, sizeof(int) * nr);
  for (int i = 0; i < nc; ++i) {
    g->vdeg[i] = col_ptr[i + 1] - col_ptr[i];
    for (int e = col_ptr[i]; e < col_ptr[i + 1]; ++e) {
      g->edge_col[e] = i;
      g->row_edges[fill[col_rows[e]]++] = e;
    }
  }
  free(fill);
}

static void graph_free(graph_t* g) {
  free(g->vblock);
  free(g->col_ptr);
  free(g->col_rows);
  free(g->row_ptr);
  free(g->row_edges);
  free(g->edge_col);
  free(g->llr);
  free(g->vdeg);
}

/* BP / decimation state of one decision path. */
typedef struct {
  float *v2c, *c2v, *post;
  float* hist[4];   /* hist[0] oldest .. hist[3] newest posterior */
  int8_t* status;   /* -1 active, 0/1 decimated (vn_status of Sec. IV-A) */
  uint8_t* sp;      /* current syndrome s' (flipped by decimations to 1) */
  int* deg;         /* number of active VNs of each CN */
} state_t;

static void state_alloc(state_t* s, const graph_t* g) {
  int ne = g->ne > 0 ? g->ne : 1, nc = g->nc > 0 ? g->nc : 1, nr = g->nr > 0 ? g->nr : 1;
  s->v2c = malloc(sizeof(float) * ne);
  s->c2v = malloc(sizeof(float) * ne);
  s->post = malloc(sizeof(float) * nc);
  for (int k = 0; k < 4; ++k) s->hist[k] = malloc(sizeof(float) * nc);
  s->status = malloc(nc);
  s->sp = malloc(nr);
  s->deg = malloc(sizeof(int) * nr);
}

static void state_free(state_t* s) {
  free(s->v2c);
  free(s->c2v);
  free(s->post);
  for (int k = 0; k < 4; ++k) free(s->hist[k]);
  free(s->status);
  free(s->sp);
  free(s->deg);
}

/* t = 0 initialisation (Sec. II-A): mu_{i->j} = Lambda_i; the history starts
 * filled with the prior (READING: a history shorter than four iterations is
 * padded with Lambda_i). */
static void state_reset(state_t* s, const graph_t* g, const uint8_t* synd) {
  for (int e = 0; e < g->ne; ++e) {
    s->v2c[e] = g->llr[g->edge_col[e]];
    s->c2v[e] = 0.0f;
  }
  for (int i = 0; i < g->nc; ++i) {
    s->post[i] = g->llr[i];
    for (int k = 0; k < 4; ++k) s->hist[k][i] = g->llr[i];
    s->status[i] = -1;
  }
  for (int j = 0; j < g->nr; ++j) {
    s->sp[j] = synd[j];
    s->deg[j] = g->row_ptr[j + 1] - g->row_ptr[j];
  }
}

static inline float clipf(float x, float c) {
  if (x > c) return c;
  if (x < -c) return -c;
  return x;
}

/*
 * One flooding iteration: CN update Eq. (1) over active VNs only, then the VN
 * update Eq. (2)-(3) for active VNs.  The minimum over N(j)\i is the smallest
 * |mu| among the OTHER active edges of CN j: that is the second smallest
 * overall when e holds the (first) smallest, else the smallest.  The sign
 * product over N(j)\i is the full product times the sign of e.  sign(x) is -1
 * for x < 0 and +1 otherwise.  READING: a CN with a single active VN sends
 * alpha * clip (minimum over the empty set taken as the clip bound).
 */
static void bp_iteration(const graph_t* g, state_t* s, float alpha, float clip, int t) {
  for (int j = 0; j < g->nr; ++j) {
    float min1 = INFINITY, min2 = INFINITY;
    int amin = -1, neg = 0, na = 0;
    for (int q = g->row_ptr[j]; q < g->row_ptr[j + 1]; ++q) {
      int e = g->row_edges[q];
      if (s->status[g->edge_col[e]] != -1) continue; /* stale message: ignored */
      float a = fabsf(s->v2c[e]);
      if (a < min1) {
        min2 = min1;
        min1 = a;
        amin = e;
      } else if (a < min2) {
        min2 = a;
      }
      neg ^= (s->v2c[e] < 0.0f);
      ++na;
    }
    if (na == 0) continue;
    for (int q = g->row_ptr[j]; q < g->row_ptr[j + 1]; ++q) {
      int e = g->row_edges[q];
      if (s->status[g->edge_col[e]] != -1) continue;
      float m = (e == amin) ? min2 : min1;
      if (na == 1) m = clip;
      int sgn = neg ^ (s->v2c[e] < 0.0f) ^ s->sp[j];
      float mag = edge_weight(g, alpha, t, e) * m;
      s->c2v[e] = sgn ? -mag : mag;
    }
  }
  for (int i = 0; i < g->nc; ++i) {
    if (s->status[i] != -1) continue;
    float p = g->llr[i];
    for (int e = g->col_ptr[i]; e < g->col_ptr[i + 1]; ++e) p = p + s->c2v[e];
    s->post[i] = p;
    for (int e = g->col_ptr[i]; e < g->col_ptr[i + 1]; ++e) s->v2c[e] = clipf(p - s->c2v[e], clip);
  }
  /* history of the last four posteriors (Sec. IV-A) */
  for (int i = 0; i < g->nc; ++i) {
    s->hist[0][i] = s->hist[1][i];
    s->hist[1][i] = s->hist[2][i];
    s->hist[2][i] = s->hist[3][i];
    s->hist[3][i] = s->post[i];
  }
}

/* Eq. (4): e_i = 1 iff posterior <= 0; decimated VNs hold their value. */
static inline int hard(const state_t* s, int i) {
  if (s->status[i] != -1) return s->status[i];
  return s->post[i] <= 0.0f;
}

/* H e = s on the whole graph.  Decimated-to-one VNs are already folded into
 * s', so the check runs over active VNs against s'. */
static int converged(const graph_t* g, const state_t* s) {
  for (int j = 0; j < g->nr; ++j) {
    int par = s->sp[j];
    for (int q = g->row_ptr[j]; q < g->row_ptr[j + 1]; ++q) {
      int i = g->edge_col[g->row_edges[q]];
      if (s->status[i] == -1) par ^= (s->post[i] <= 0.0f);
    }
    if (par) return 0;
  }
  return 1;
}

/* Fix VN i to value v (Sec. II-A): it leaves the network; its CNs lose one
 * active neighbour and flip their syndrome when v = 1. */
static void decimate(const graph_t* g, state_t* s, int i, int v) {
  s->status[i] = (int8_t)v;
  for (int e = g->col_ptr[i]; e < g->col_ptr[i + 1]; ++e) {
    int j = g->col_rows[e];
    s->deg[j]--;
    if (v) s->sp[j] ^= 1;
  }
}

/* Peeling (Sec. IV "Do not waste guesses"): while some CN has exactly one
 * active VN, that VN must equal the CN's current syndrome.  A CN left with no
 * active VN and syndrome 1 is a contradiction (appendix "GDG implementation").
 * READING: the paper fixes no order; CNs are peeled one at a time, always the
 * lowest-index degree-one CN, after checking every CN for a contradiction.
 * Without a contradiction the result does not depend on the order (the forced
 * values are unique); with one, this order makes the killed path's partial
 * state well defined.  Returns the number of peeled VNs, or -1. */
static int peel(const graph_t* g, state_t* s) {
  int n = 0;
  for (;;) {
    int jmin = -1;
    for (int j = 0; j < g->nr; ++j) {
      if (s->deg[j] == 0 && s->sp[j]) return -1;
      if (s->deg[j] == 1 && jmin < 0) jmin = j;
    }
    if (jmin < 0) return n;
    int i = -1;
    for (int q = g->row_ptr[jmin]; q < g->row_ptr[jmin + 1]; ++q) {
      int c = g->edge_col[g->row_edges[q]];
      if (s->status[c] == -1) { i = c; break; }
    }
    decimate(g, s, i, s->sp[jmin]);
    ++n;
  }
}

/* Alg. 3, AGG-DEC.  "hist < P" means all four entries.  Returns 1, 0 or -1. */
static int agg_dec(const qdo_params* P, const float* h, float L, int D, int main_branch, int n_unsat) {
  float PA = main_branch ? P->pa_main : P->pa_other;
  float PB = main_branch ? P->pb_main : P->pb_other;
  if (D == 1) PB = P->pb_d1;
  if (h[0] < PA && h[1] < PA && h[2] < PA && h[3] < PA && L < PB) return 1;
  int allc = h[0] > P->pc && h[1] > P->pc && h[2] > P->pc && h[3] > P->pc;
  int alld = h[0] > P->pd && h[1] > P->pd && h[2] > P->pd && h[3] > P->pd;
  if ((allc && D <= P->pc_max_depth) || (alld && n_unsat >= P->n_unsat_min)) return 0;
  return -1;
}

/*
 * Learned decimation ranker (no counterpart in the paper; it stands in for
 * the argmin of Alg. 1).  Parameters are rounded to fixed grids -- W1, W2 to
 * multiples of 2^-6 in [-2, 2], b1 to multiples of 2^-7 in [-512, 512] (round half to even)
 * -- and the features of a candidate VN are
 *   x = (L/4, h0, h1, h2, h3     each rounded to the 1/2 grid within +-63.5,
 *        #unsatisfied CN neighbours (at most 127), static degree,
 *        block of the column's first detector within the window (at most 255)),
 * so that every product and partial sum of the first layer is a multiple of
 * 2^-7 below 2^13, i.e. exact in FP32 in any summation order.  Hidden unit
 * u: relu(b1[u] + sum_k W1[u][k] x_k).  The second layer is summed in FP32 in
 * a fixed order: for q = 0..3, s_q = sum over t = 0..7, c = 0..1 (in that
 * order) of W2[u] h[u] with u = 8t + 2q + c, starting from 0; score =
 * ((s_0 + s_1) + (s_2 + s_3)) + b2.
 */
typedef struct { float w1[64][8], b1[64], w2[64], b2; } ranker_t;

static float qgrid(float x, float scale, float lim) {
  float v = rintf(x * scale);
  if (v > lim) v = lim;
  if (v < -lim) v = -lim;
  return v / scale;
}

static void ranker_quantize(const float* raw, ranker_t* r) {
  for (int u = 0; u < 64; ++u)
    for (int k = 0; k < 8; ++k) r->w1[u][k] = qgrid(raw[u * 8 + k], 64.0f, 128.0f);
  for (int u = 0; u < 64; ++u) r->b1[u] = qgrid(raw[512 + u], 128.0f, 65536.0f);
  for (int u = 0; u < 64; ++u) r->w2[u] = qgrid(raw[576 + u], 64.0f, 128.0f);
  r->b2 = raw[640];
}

static float qfeat(float x) {
  float v = rintf(2.0f * (x > 63.5f ? 63.5f : (x < -63.5f ? -63.5f : x)));
  return v * 0.5f;
}

static float ranker_score(const ranker_t* r, const float* x) {
  float h[64];
  for (int u = 0; u < 64; ++u) {
    double a = r->b1[u];
    for (int k = 0; k < 8; ++k) a += (double)r->w1[u][k] * (double)x[k]; /* exact */
    float hf = (float)a;
    h[u] = hf > 0.0f ? hf : 0.0f;
  }
  float sq[4];
  for (int q = 0; q < 4; ++q) {
    float acc = 0.0f;
    for (int t = 0; t < 8; ++t)
      for (int c = 0; c < 2; ++c) {
        int u = 8 * t + 2 * q + c;
        float prod = r->w2[u] * h[u];
        acc = acc + prod;
      }
    sq[q] = acc;
  }
  return ((sq[0] + sq[1]) + (sq[2] + sq[3])) + r->b2;
}

/* Scores of n feature rows x [n][8] under raw parameters (test access). */
void qdo_ranker_score(const float* raw, const float* x, int n, float* out) {
  ranker_t r;
  ranker_quantize(raw, &r);
  for (int i = 0; i < n; ++i) out[i] = ranker_score(&r, x + 8 * i);
}

/* Alg. 1, SELECT-VN, with Alg. 3 applied to each candidate outside the low
 * error mode.  Candidates: active VNs of degree >= 3, in index order; strict
 * '<' keeps the lowest index on ties.  f = 1 iff L_min <= 0 (the sign of
 * L_min read through Eq. (4)).  Unsatisfied-neighbour counts are taken from
 * the state before the loop (an aggressive decision always equals the VN's
 * current hard decision, so it never changes any CN's satisfaction). */
static int select_vn(const graph_t* g, state_t* s, const qdo_params* P, int D, int main_branch,
                     int path0, int* f_out, int* n_agg) {
  int* nus = calloc(g->nc > 0 ? g->nc : 1, sizeof(int));
  if (!P->low_error_mode || P->ranker || P->dump) {
    for (int j = 0; j < g->nr; ++j) {
      int par = s->sp[j];
      for (int q = g->row_ptr[j]; q < g->row_ptr[j + 1]; ++q) {
        int i = g->edge_col[g->row_edges[q]];
        if (s->status[i] == -1) par ^= hard(s, i);
      }
      if (!par) continue;
      for (int q = g->row_ptr[j]; q < g->row_ptr[j + 1]; ++q) nus[g->edge_col[g->row_edges[q]]]++;
    }
  }
  float Lmin = INFINITY, Lt = INFINITY;
  int gmin = -1, gt = -1;
  ranker_t rk;
  float best = -INFINITY, Lbest = 0.0f;
  int gbest = -1;
  if (P->ranker) ranker_quantize(P->ranker, &rk);
  const int dumping = P->dump && path0;
  const int d0 = dumping ? *P->dump_n : 0;
  *n_agg = 0;
  for (int i = 0; i < g->nc; ++i) {
    if (s->status[i] != -1) continue;
    if (g->vdeg[i] <= 2) continue;
    float h[4] = {s->hist[0][i], s->hist[1][i], s->hist[2][i], s->hist[3][i]};
    float L = ((h[0] + h[1]) + h[2]) + h[3];
    if (!P->low_error_mode) {
      int b = agg_dec(P, h, L, D, main_branch, nus[i]);
      if (b != -1) {
        decimate(g, s, i, b);
        (*n_agg)++;
        continue;
      }
    }
    float x[8] = {qfeat(L * 0.25f), qfeat(h[0]), qfeat(h[1]), qfeat(h[2]), qfeat(h[3]),
                  (float)(nus[i] > 127 ? 127 : nus[i]), (float)g->vdeg[i],
                  (float)(g->vblock[i] > 255 ? 255 : g->vblock[i])};
    if (dumping) {
      int pos = (*P->dump_n)++;
      if (pos < P->dump_cap) {
        qdo_rank_rec* r = &P->dump[pos];
        memcpy(r->x, x, sizeof(x));
        r->shot = 0;
        r->wcol = g->wcol ? g->wcol[i] : i;
        r->depth = (int16_t)D;
        r->path = 0;
        r->flags = L <= 0.0f ? 1 : 0;
      }
    }
    if (P->ranker) {
      /* READING: the ranker replaces the argmin; ties keep the lowest index */
      float sc = ranker_score(&rk, x);
      if (sc > best) {
        best = sc;
        gbest = i;
        Lbest = L;
      }
      continue;
    }
    if (L < Lmin) {
      Lmin = L;
      gmin = i;
    }
    if (h[0] <= 0.0f && h[1] <= 0.0f && h[2] <= 0.0f && h[3] <= 0.0f && L < Lt) {
      Lt = L;
      gt = i;
    }
  }
  free(nus);
  int gsel;
  if (P->ranker) {
    /* f keeps Alg. 1's rule: 1 iff the selected VN's history sum is <= 0 */
    *f_out = (gbest != -1 && Lbest <= 0.0f) ? 1 : 0;
    gsel = gbest;
  } else if (gt != -1) {
    *f_out = 1;
    gsel = gt;
  } else {
    *f_out = (gmin != -1 && Lmin <= 0.0f) ? 1 : 0;
    gsel = gmin;
  }
  if (dumping && gsel >= 0) {
    int w = g->wcol ? g->wcol[gsel] : gsel;
    for (int q = d0; q < *P->dump_n && q < P->dump_cap; ++q)
      if (P->dump[q].wcol == w) P->dump[q].flags |= 2;
  }
  return gsel;
}

/* Test access to Alg. 3 for one VN: its four-iteration history h (oldest
 * first), depth D, main-branch flag and unsatisfied-neighbour count. */
int qdo_agg_dec(const qdo_params* P, const float* h, int D, int main_branch, int n_unsat) {
  float L = ((h[0] + h[1]) + h[2]) + h[3];
  return agg_dec(P, h, L, D, main_branch, n_unsat);
}

/* Test access to one call of Alg. 1 (with Alg. 3 outside the low-error mode)
 * on an explicit graph and path state: hist [4][nc] oldest first, whose
 * newest row is also the current posterior deciding e_i (Eq. (4)); status
 * [nc] (-1 active, else the decimated value) and synd [nr] = the current s'
 * are updated with the aggressive decisions.  Returns g (-1: no candidate)
 * and writes f and the number of aggressive decisions. */
int qdo_select_vn(const qdo_params* P, int nr, int nc, const int* col_ptr, const int* col_rows,
                  const float* hist, int8_t* status, uint8_t* synd, int D, int main_branch,
                  int* f_out, int* n_agg) {
  float* llr = calloc(nc > 0 ? nc : 1, sizeof(float));
  graph_t g;
  graph_init(&g, nr, nc, col_ptr, col_rows, llr);
  free(llr);
  state_t s;
  state_alloc(&s, &g);
  for (int i = 0; i < nc; ++i) {
    for (int k = 0; k < 4; ++k) s.hist[k][i] = hist[(size_t)k * nc + i];
    s.post[i] = hist[(size_t)3 * nc + i];
    s.status[i] = status[i];
  }
  for (int j = 0; j < nr; ++j) {
    s.sp[j] = synd[j];
    s.deg[j] = 0;
    for (int q = g.row_ptr[j]; q < g.row_ptr[j + 1]; ++q)
      if (s.status[g.edge_col[g.row_edges[q]]] == -1) s.deg[j]++;
  }
  int gsel = select_vn(&g, &s, P, D, main_branch, 0, f_out, n_agg);
  memcpy(status, s.status, nc);
  memcpy(synd, s.sp, nr);
  state_free(&s);
  graph_free(&g);
  return gsel;
}

/* Eq. (5) accumulated in double from the FP32 priors. */
static double path_metric(const graph_t* g, const state_t* s) {
  double pm = 0.0;
  for (int i = 0; i < g->nc; ++i)
    if (hard(s, i)) pm += (double)g->llr[i];
  return pm;
}

/*
 * The decision paths of Fig. 2 / Alg. 2.  Ids 0 .. 2^k - 1 form the guessing
 * tree (id 0 = the main branch; at depth D <= k path id takes bit k - D of
 * its id, most significant first, as b of b + (-1)^b f).  With side branches
 * (side_max >= k), ids 2^k .. add the side branches that split off the main
 * branch at D_split = k+1 .. side_max, and id 1 -- contrary only at D = k --
 * is the side branch with D_split = k.  A side branch takes f everywhere
 * except 1 - f at D_split and runs D_split + (d_max_other - k) steps; tree
 * branches run d_max_other = k + (steps after the last guess).
 * READING: a side branch is the main branch up to and including its split
 * step (main-branch thresholds of Alg. 3 there), as the paper's side threads
 * start from the main thread's status at the split; afterwards it uses the
 * other-branch thresholds.  Messages stay continuous along every path.
 */
int qdo_n_paths(const qdo_params* P) {
  int nt = 1 << P->k_guess;
  return nt + (P->side_max > P->k_guess ? P->side_max - P->k_guess : 0);
}

int qdo_path_dmax_all(const qdo_params* P) {
  int dmx = P->d_max_main > P->d_max_other ? P->d_max_main : P->d_max_other;
  int side = P->side_max + (P->d_max_other - P->k_guess);
  if (P->side_max > 0 && side > dmx) dmx = side;
  return dmx;
}

/* 0 = tree (or main) path, else the split depth of a side branch */
static int side_split(const qdo_params* P, int id) {
  int nt = 1 << P->k_guess;
  if (P->side_max <= 0) return 0;
  if (id >= nt) return P->k_guess + 1 + (id - nt);
  if (id == 1 && P->k_guess >= 1) return P->k_guess;
  return 0;
}

/*
 * READING (reinit_on_split = 1, the appendix's multi-thread implementation):
 * a path that continues from another path's status snapshot starts its BP
 * messages afresh there -- a side branch at D_split, and the second branch of
 * each neighbouring pair of tree branches (odd id, contrary at D = k).  Right
 * after that decimation (and its peeling) mu_{i->j} = Lambda_i for every
 * active VN, and the iteration count of the learned weights restarts.
 * Returns 0 for paths that never restart.
 */
static int reinit_depth(const qdo_params* P, int id, int split) {
  if (!P->reinit_on_split) return 0;
  if (split) return split;
  if (id >= 1 && (id & 1) && P->k_guess >= 1) return P->k_guess;
  return 0;
}

/* One decision path of Alg. 2 on graph g (the shortened window). */
static void run_branch(const graph_t* g, const uint8_t* synd, const qdo_params* P, int id,
                       state_t* s, qdo_branch_summary* out, qdo_step_record* steps) {
  const int split = side_split(P, id);
  const int d_reinit = reinit_depth(P, id, split);
  int tw = 0; /* iterations since the messages were (re)initialised */
  int dmax = id == 0 ? P->d_max_main : (split ? split + (P->d_max_other - P->k_guess) : P->d_max_other);
  state_reset(s, g, synd);
  out->status = BR_MAXDEPTH;
  out->depth = 0;
  out->iters = 0;
  out->pm = INFINITY;
  if (P->peel_at_init && peel(g, s) < 0) {
    out->status = BR_CONTRADICTION;
    return;
  }
  for (int D = 1; D <= dmax; ++D) {
    out->depth = D;
    /* READING: iters_first > 0 gives the first step its own length (the
     * initial BP run as GDG's first step, without pre-BP or shortening) */
    const int n_it = (D == 1 && P->iters_first > 0) ? P->iters_first : P->iters_per_step;
    for (int it = 0; it < n_it; ++it) {
      bp_iteration(g, s, P->alpha, P->clip, ++tw);
      out->iters++;
      if (converged(g, s)) {
        out->status = BR_CONVERGED;
        out->pm = path_metric(g, s);
        return;
      }
    }
    if (D == dmax) break; /* READING: no decimation after the last BP step */
    int f, nagg;
    int main_rules = id == 0 || (split && D <= split);
    int gsel = select_vn(g, s, P, D, main_rules, id == 0, &f, &nagg);
    qdo_step_record* rec = steps ? &steps[D - 1] : NULL;
    if (gsel < 0) {
      if (rec) { rec->g = -1; rec->value = -1; rec->n_agg = nagg; rec->n_peel = 0; }
      out->status = BR_NOCAND;
      return;
    }
    int v = f;
    if (split) {
      if (D == split) v = 1 - f; /* the one contrary decision of a side branch */
    } else if (D <= P->k_guess) {
      int b = (id >> (P->k_guess - D)) & 1;
      v = b ? 1 - f : f; /* b + (-1)^b f */
    }
    decimate(g, s, gsel, v);
    int np = peel(g, s);
    if (rec) { rec->g = gsel; rec->value = v; rec->n_agg = nagg; rec->n_peel = np < 0 ? -1 : np; }
    if (np < 0) {
      out->status = BR_CONTRADICTION;
      return;
    }
    if (D == d_reinit) {
      for (int e = 0; e < g->ne; ++e)
        if (s->status[g->edge_col[e]] == -1) s->v2c[e] = g->llr[g->edge_col[e]];
      tw = 0;
    }
  }
}

/* ---- plain BP on an explicit graph (used by tests) ---- */
int qdo_bp_run(int n_rows, int n_cols, const int* col_ptr, const int* col_rows, const float* llr,
               const uint8_t* synd, float alpha, float clip, int max_iter, int early_stop,
               uint8_t* e_out, float* post_out) {
  graph_t g;
  graph_init(&g, n_rows, n_cols, col_ptr, col_rows, llr);
  state_t s;
  state_alloc(&s, &g);
  state_reset(&s, &g, synd);
  int it = 0, conv = 0;
  while (it < max_iter) {
    bp_iteration(&g, &s, alpha, clip, it + 1);
    ++it;
    if (converged(&g, &s)) {
      conv = 1;
      if (early_stop) break;
    }
  }
  for (int i = 0; i < n_cols; ++i) {
    e_out[i] = (uint8_t)hard(&s, i);
    if (post_out) post_out[i] = s.post[i];
  }
  state_free(&s);
  graph_free(&g);
  return conv ? it : -it;
}

/* Unsatisfied checks of a path's estimate among rows [j0, j1): H e != s
 * (the test of converged() counted instead of stopped at the first). */
static int n_unsat_rows(const graph_t* g, const state_t* s, int j0, int j1) {
  int n = 0;
  for (int j = j0; j < j1; ++j) {
    int par = s->sp[j];
    for (int q = g->row_ptr[j]; q < g->row_ptr[j + 1]; ++q) {
      int i = g->edge_col[g->row_edges[q]];
      if (s->status[i] == -1) par ^= (s->post[i] <= 0.0f);
    }
    n += par;
  }
  return n;
}

/* GDG over all decision paths of graph g; returns the winning id or -1.
 * Rows [0, n_commit_rows) are those the window commits (the fallback rule 2
 * looks at them first). */
static int gdg_all(const graph_t* g, const uint8_t* synd, const qdo_params* P, uint8_t* e_out,
                   qdo_branch_summary* br_out, qdo_step_record* steps_out, int8_t* status_out,
                   float* keep_out, int n_commit_rows, uint8_t* est_out) {
  int nb = qdo_n_paths(P);
  int dmx = qdo_path_dmax_all(P);
  state_t s;
  state_alloc(&s, g);
  int best = -1;
  double best_pm = INFINITY;
  uint8_t* e0 = malloc(g->nc > 0 ? g->nc : 1);
  uint8_t* eb = malloc(g->nc > 0 ? g->nc : 1);
  /* what the output path leaves for the next window (message reuse): its
   * final posterior, or +-clip for a column it decimated to 0 / 1 */
  float* k0 = malloc(sizeof(float) * (g->nc > 0 ? g->nc : 1));
  float* kb = malloc(sizeof(float) * (g->nc > 0 ? g->nc : 1));
  long long key0 = 0;
  for (int id = 0; id < nb; ++id) {
    qdo_branch_summary sm;
    qdo_step_record* rec = steps_out ? steps_out + (size_t)id * dmx : NULL;
    if (rec)
      for (int q = 0; q < dmx; ++q) { rec[q].g = -2; rec[q].value = -1; rec[q].n_agg = 0; rec[q].n_peel = 0; }
    run_branch(g, synd, P, id, &s, &sm, rec);
    if (br_out) br_out[id] = sm;
    if (status_out) memcpy(status_out + (size_t)id * g->nc, s.status, g->nc);
    if (est_out)
      for (int i = 0; i < g->nc; ++i) est_out[(size_t)id * g->nc + i] = (uint8_t)hard(&s, i);
    /* READING (fallback rule, used only when no path converges): 0 keeps
     * path 0's estimate; 1 the estimate with the fewest unsatisfied checks
     * of the window; 2 the fewest among the committed rows, then among all
     * rows.  Ties keep the lowest id. */
    long long key = 0;
    if (P->fallback == 1) key = n_unsat_rows(g, &s, 0, g->nr);
    if (P->fallback == 2)
      key = (long long)n_unsat_rows(g, &s, 0, n_commit_rows) * (g->nr + 1) + n_unsat_rows(g, &s, 0, g->nr);
    if (id == 0 || key < key0) {
      key0 = key;
      for (int i = 0; i < g->nc; ++i) {
        e0[i] = (uint8_t)hard(&s, i);
        k0[i] = s.status[i] == -1 ? s.post[i] : (s.status[i] ? -P->clip : P->clip);
      }
    }
    /* Alg. 2: the estimate with the smallest path metric; ties keep the
     * lowest id */
    if (sm.status == BR_CONVERGED && sm.pm < best_pm) {
      best_pm = sm.pm;
      best = id;
      for (int i = 0; i < g->nc; ++i) {
        eb[i] = (uint8_t)hard(&s, i);
        kb[i] = s.status[i] == -1 ? s.post[i] : (s.status[i] ? -P->clip : P->clip);
      }
    }
  }
  /* no converged path: the fallback estimate above */
  memcpy(e_out, best >= 0 ? eb : e0, g->nc);
  if (keep_out) memcpy(keep_out, best >= 0 ? kb : k0, sizeof(float) * g->nc);
  free(e0);
  free(eb);
  free(k0);
  free(kb);
  state_free(&s);
  return best;
}

int qdo_gdg_graph(const qdo_params* P, int n_rows, int n_cols, const int* col_ptr,
                  const int* col_rows, const float* llr, const uint8_t* synd, uint8_t* corr,
                  qdo_branch_summary* br) {
  graph_t g;
  graph_init(&g, n_rows, n_cols, col_ptr, col_rows, llr);
  int best = gdg_all(&g, synd, P, corr, br, NULL, NULL, NULL, n_rows, NULL);
  graph_free(&g);
  return best;
}

/* Window of the DEM as a graph over its rows and columns. */
typedef struct {
  int k, r0, nb, nr, nc, ne, last;
  int *gcols, *col_ptr, *col_rows;
  uint8_t* commit;
  float* llr;
} window_t;

const double* qdo__col_p(const qdo_dem* d);
static void window_free(window_t* wd);

typedef struct { double p; int col; } pcol_t;
static int cmp_pcol(const void* a, const void* b) {
  const pcol_t* x = a;
  const pcol_t* y = b;
  if (x->p < y->p) return -1;
  if (x->p > y->p) return 1;
  return x->col < y->col ? -1 : (x->col > y->col);
}

/* XOR-probability of independent mechanisms (Sec. II-B merging), folded in
 * ascending (probability, DEM column), as the DEM's own merge does. */
static double xor_fold(pcol_t* v, int n) {
  qsort(v, n, sizeof(pcol_t), cmp_pcol);
  double pm = 0.0;
  for (int i = 0; i < n; ++i) pm = pm * (1.0 - v[i].p) + v[i].p * (1.0 - pm);
  return pm;
}

/*
 * Sec. III: the columns of H_1 -- the window columns that extend past the
 * window's last block, restricted to it -- are merged to an identity matrix
 * with recalculated priors.  READING (two variants, off by default; only for
 * windows that are not the last and commit fewer blocks than they hold, so
 * that no merged column is ever committed):
 *   merge = 1: exact merges only -- H_1 columns whose restrictions to the
 *     window are equal become one column at the first one's place, its
 *     probability the XOR of theirs; the window's parity-check problem is
 *     unchanged (the restrictions of weight one become the identity);
 *   merge = 2: the identity itself -- every H_1 column is removed, and one
 *     column per detector t of the last block is appended (t ascending),
 *     flipping t alone with probability the XOR of the H_1 columns whose
 *     restriction contains t (detector flips taken as independent).
 */
static void window_merge_h1(const qdo_dem* d, int merge, window_t* wd) {
  const int w = qdo__w(d), hi = (wd->r0 + wd->nb) * w, lo_last = (wd->r0 + wd->nb - 1) * w;
  const int* cptr = qdo__col_ptr(d);
  const int* cdet = qdo__col_dets(d);
  const double* cp = qdo__col_p(d);
  int nc = wd->nc;
  int* ext = calloc(nc > 0 ? nc : 1, sizeof(int));
  for (int c = 0; c < nc; ++c) {
    int g = wd->gcols[c];
    for (int e = cptr[g]; e < cptr[g + 1]; ++e)
      if (cdet[e] >= hi) ext[c] = 1;
  }
  int* gc = malloc(sizeof(int) * (nc + w + 1));
  int* cpn = malloc(sizeof(int) * (nc + w + 2));
  int* crn = malloc(sizeof(int) * (wd->ne + w + 1));
  uint8_t* com = malloc(nc + w + 1);
  float* ll = malloc(sizeof(float) * (nc + w + 1));
  pcol_t* grp = malloc(sizeof(pcol_t) * (nc + 1));
  int m = 0, ne = 0;
  cpn[0] = 0;
  for (int c = 0; c < nc; ++c) {
    if (ext[c] && merge == 2) continue;
    if (ext[c] && merge == 1) {
      /* the first column of its restriction class keeps the class */
      int first = 1;
      for (int c2 = 0; c2 < c && first; ++c2)
        if (ext[c2] && wd->col_ptr[c2 + 1] - wd->col_ptr[c2] == wd->col_ptr[c + 1] - wd->col_ptr[c] &&
            memcmp(wd->col_rows + wd->col_ptr[c2], wd->col_rows + wd->col_ptr[c],
                   sizeof(int) * (wd->col_ptr[c + 1] - wd->col_ptr[c])) == 0)
          first = 0;
      if (!first) continue;
      int n = 0;
      for (int c2 = c; c2 < nc; ++c2)
        if (ext[c2] && wd->col_ptr[c2 + 1] - wd->col_ptr[c2] == wd->col_ptr[c + 1] - wd->col_ptr[c] &&
            memcmp(wd->col_rows + wd->col_ptr[c2], wd->col_rows + wd->col_ptr[c],
                   sizeof(int) * (wd->col_ptr[c + 1] - wd->col_ptr[c])) == 0) {
          grp[n].p = cp[wd->gcols[c2]];
          grp[n].col = wd->gcols[c2];
          ++n;
        }
      double pm = xor_fold(grp, n);
      ll[m] = (float)log((1.0 - pm) / pm);
    } else {
      ll[m] = wd->llr[c];
    }
    gc[m] = wd->gcols[c];
    com[m] = wd->commit[c];
    for (int e = wd->col_ptr[c]; e < wd->col_ptr[c + 1]; ++e) crn[ne++] = wd->col_rows[e];
    cpn[++m] = ne;
  }
  if (merge == 2)
    for (int t = 0; t < w; ++t) {
      const int row = lo_last + t - wd->r0 * w;
      int n = 0, rep = -1;
      for (int c = 0; c < nc; ++c) {
        if (!ext[c]) continue;
        for (int e = wd->col_ptr[c]; e < wd->col_ptr[c + 1]; ++e)
          if (wd->col_rows[e] == row) {
            grp[n].p = cp[wd->gcols[c]];
            grp[n].col = wd->gcols[c];
            if (rep < 0) rep = wd->gcols[c];
            ++n;
          }
      }
      if (!n) continue;
      double pm = xor_fold(grp, n);
      gc[m] = rep;
      com[m] = 0;
      ll[m] = (float)log((1.0 - pm) / pm);
      crn[ne++] = row;
      cpn[++m] = ne;
    }
  free(grp);
  free(ext);
  free(wd->gcols);
  free(wd->col_ptr);
  free(wd->col_rows);
  free(wd->commit);
  free(wd->llr);
  wd->gcols = gc;
  wd->col_ptr = cpn;
  wd->col_rows = crn;
  wd->commit = com;
  wd->llr = ll;
  wd->nc = m;
  wd->ne = ne;
}

static void window_build(const qdo_dem* d, int W, int F, int k, int merge, window_t* wd) {
  int info[7];
  qdo_window_info(d, W, F, k, info);
  wd->k = k;
  wd->r0 = info[0];
  wd->nb = info[1];
  wd->nr = info[2];
  wd->nc = info[3];
  wd->ne = info[4];
  wd->last = info[6];
  wd->gcols = malloc(sizeof(int) * (wd->nc + 1));
  wd->col_ptr = malloc(sizeof(int) * (wd->nc + 1));
  wd->col_rows = malloc(sizeof(int) * (wd->ne + 1));
  wd->commit = malloc(wd->nc + 1);
  wd->llr = malloc(sizeof(float) * (wd->nc + 1));
  qdo_window_graph(d, W, F, k, wd->gcols, wd->col_ptr, wd->col_rows, wd->commit);
  const float* L = qdo__col_llr(d);
  for (int c = 0; c < wd->nc; ++c) wd->llr[c] = L[wd->gcols[c]];
  if (merge && !wd->last && W > F) window_merge_h1(d, merge, wd);
}

int qdo_window_build(const qdo_dem* d, int W, int F, int k, int merge, int* info, int* gcols, int* col_ptr,
                     int* col_rows, uint8_t* commit, float* llr) {
  window_t wd;
  window_build(d, W, F, k, merge, &wd);
  int ncom = 0;
  for (int c = 0; c < wd.nc; ++c) ncom += wd.commit[c];
  info[0] = wd.r0;
  info[1] = wd.nb;
  info[2] = wd.nr;
  info[3] = wd.nc;
  info[4] = wd.ne;
  info[5] = ncom;
  info[6] = wd.last;
  if (gcols) {
    memcpy(gcols, wd.gcols, sizeof(int) * wd.nc);
    memcpy(col_ptr, wd.col_ptr, sizeof(int) * (wd.nc + 1));
    memcpy(col_rows, wd.col_rows, sizeof(int) * wd.ne);
    memcpy(commit, wd.commit, wd.nc);
    memcpy(llr, wd.llr, sizeof(float) * wd.nc);
  }
  window_free(&wd);
  return 0;
}

static void window_free(window_t* wd) {
  free(wd->gcols);
  free(wd->col_ptr);
  free(wd->col_rows);
  free(wd->commit);
  free(wd->llr);
}

typedef struct { float key; int idx; } rank_t;
static int cmp_rank(const void* a, const void* b) {
  const rank_t* x = a;
  const rank_t* y = b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/*
 * Decode one window (Sec. III + Sec. IV):
 *   1. n_pre BP iterations on the full window with early stop; a converged
 *      pre-BP ends the window (READING);
 *   2. rank columns by ((h0+h1)+h2)+h3 ascending, ties by column index, keep
 *      the first 2w' (all columns if there are fewer);
 *   3. GDG on the kept columns (messages restart from the priors), winner by
 *      Eq. (5); dropped columns are decided 0.
 */
/*
 * READING of the message reuse between windows (Sec. VI leaves it to future
 * work, naming the branch with the minimum path metric as the source): the
 * next window's pre-BP starts its first VN->CN messages of every column it
 * shares with this window from what this window's output path ends with --
 * the column's final posterior, or +-clip for a column that path decimated
 * to 0 / 1; the pre-BP's own posterior when the pre-BP converged.  Columns
 * the output path did not hold (dropped by the shortening) and the next
 * window's new columns start from their prior.  keep[c] per window column
 * (NaN: nothing kept); init[c] the values kept for this window's columns
 * (NaN: the prior).
 */
static int decode_window_impl(const window_t* wd, const qdo_params* P, const uint8_t* synd,
                              uint8_t* corr, int* info, int* short_cols, qdo_branch_summary* br,
                              qdo_step_record* steps, int8_t* fstat, const float* init, float* keep,
                              uint8_t* est) {
  if (keep)
    for (int c = 0; c < wd->nc; ++c) keep[c] = NAN;
  if (wd->nc == 0) {
    /* READING: a window without columns decides nothing; the commit's
     * residue test sees its syndrome */
    if (info) { info[0] = 1; info[1] = -1; info[2] = 0; info[3] = 0; }
    return 0;
  }
  graph_t g;
  graph_init(&g, wd->nr, wd->nc, wd->col_ptr, wd->col_rows, wd->llr);
  const float* W = (P->wts && P->wT > 0) ? P->wts[wd->k] : NULL;
  g.w = W;
  g.wT = P->wT;
  g.wE = wd->ne;
  state_t s;
  state_alloc(&s, &g);
  state_reset(&s, &g, synd);
  if (init)
    for (int e = 0; e < g.ne; ++e)
      if (!isnan(init[g.edge_col[e]])) s.v2c[e] = init[g.edge_col[e]];
  int conv = 0, it = 0;
  for (it = 0; it < P->n_pre;) {
    bp_iteration(&g, &s, P->alpha, P->clip, it + 1);
    ++it;
    if (converged(&g, &s)) { conv = 1; break; }
  }
  if (P->n_pre == 0 && converged(&g, &s)) conv = 1;
  if (info) { info[0] = conv; info[1] = -1; info[2] = 0; info[3] = it; }
  if (conv) {
    for (int i = 0; i < wd->nc; ++i) corr[i] = (uint8_t)hard(&s, i);
    if (keep)
      for (int i = 0; i < wd->nc; ++i) keep[i] = s.post[i];
    state_free(&s);
    graph_free(&g);
    return 0;
  }
  int ns = wd->nc;
  int* sel = malloc(sizeof(int) * (wd->nc + 1));
  if (P->shorten && wd->nc > 2 * wd->nr) ns = 2 * wd->nr;
  rank_t* rk = malloc(sizeof(rank_t) * (wd->nc + 1));
  for (int i = 0; i < wd->nc; ++i) {
    rk[i].key = ((s.hist[0][i] + s.hist[1][i]) + s.hist[2][i]) + s.hist[3][i];
    rk[i].idx = i;
  }
  qsort(rk, wd->nc, sizeof(rank_t), cmp_rank);
  for (int k = 0; k < ns; ++k) sel[k] = rk[k].idx;
  free(rk);
  state_free(&s);
  /* shortened graph: kept columns in rank order, all window rows */
  int* cp = malloc(sizeof(int) * (ns + 1));
  int* cr = malloc(sizeof(int) * (wd->ne + 1));
  int* ef = malloc(sizeof(int) * (wd->ne + 1));
  float* ll = malloc(sizeof(float) * (ns + 1));
  cp[0] = 0;
  for (int k = 0; k < ns; ++k) {
    int c = sel[k];
    int n = 0;
    for (int e = wd->col_ptr[c]; e < wd->col_ptr[c + 1]; ++e) {
      ef[cp[k] + n] = e; /* the shortened edge keeps its full-window edge's weights */
      cr[cp[k] + n++] = wd->col_rows[e];
    }
    cp[k + 1] = cp[k] + n;
    ll[k] = wd->llr[c];
  }
  graph_t gs;
  graph_init(&gs, wd->nr, ns, cp, cr, ll);
  for (int k = 0; k < ns; ++k) gs.vblock[k] = wd->col_rows[wd->col_ptr[sel[k]]] / (wd->nr / wd->nb);
  gs.w = W;
  gs.wT = P->wT;
  gs.wE = wd->ne;
  gs.efull = ef;
  gs.wcol = sel;
  uint8_t* es = malloc(ns + 1);
  float* ks = keep ? malloc(sizeof(float) * (ns + 1)) : NULL;
  /* the committed rows: the first F blocks' (every row in the last window) */
  int ncr = wd->last ? wd->nr : (wd->nb > 0 ? P->F * (wd->nr / wd->nb) : wd->nr);
  if (ncr > wd->nr) ncr = wd->nr;
  uint8_t* eall = est ? calloc((size_t)qdo_n_paths(P) * ns + 1, 1) : NULL;
  int best = gdg_all(&gs, synd, P, es, br, steps, fstat, ks, ncr, eall);
  if (est) {
    for (int id = 0; id < qdo_n_paths(P); ++id)
      for (int k = 0; k < ns; ++k) est[(size_t)id * wd->nc + sel[k]] = eall[(size_t)id * ns + k];
    free(eall);
  }
  memset(corr, 0, wd->nc);
  for (int k = 0; k < ns; ++k) corr[sel[k]] = es[k];
  if (keep)
    for (int k = 0; k < ns; ++k) keep[sel[k]] = ks[k];
  free(ks);
  if (info) { info[1] = best; info[2] = ns; }
  if (short_cols) memcpy(short_cols, sel, sizeof(int) * ns);
  free(es);
  graph_free(&gs);
  free(cp);
  free(cr);
  free(ef);
  free(ll);
  free(sel);
  graph_free(&g);
  return 0;
}

int qdo_decode_window_ex(const qdo_dem* d, const qdo_params* P, int k, const uint8_t* synd, uint8_t* corr,
                         int* info, const float* init, float* keep) {
  window_t wd;
  window_build(d, P->W, P->F, k, P->merge_h1, &wd);
  int rc = decode_window_impl(&wd, P, synd, corr, info, NULL, NULL, NULL, NULL, init, keep, NULL);
  window_free(&wd);
  return rc;
}

int qdo_decode_window_paths(const qdo_dem* d, const qdo_params* P, int k, const uint8_t* synd, uint8_t* corr,
                            int* info, uint8_t* est) {
  window_t wd;
  window_build(d, P->W, P->F, k, P->merge_h1, &wd);
  int rc = decode_window_impl(&wd, P, synd, corr, info, NULL, NULL, NULL, NULL, NULL, NULL, est);
  window_free(&wd);
  return rc;
}

int qdo_decode_window(const qdo_dem* d, const qdo_params* P, int k, const uint8_t* synd,
                      uint8_t* corr, int* info, int* short_cols, qdo_branch_summary* br,
                      qdo_step_record* steps, int8_t* final_status) {
  window_t wd;
  window_build(d, P->W, P->F, k, P->merge_h1, &wd);
  int rc = decode_window_impl(&wd, P, synd, corr, info, short_cols, br, steps, final_status, NULL, NULL, NULL);
  window_free(&wd);
  return rc;
}

/*
 * The (W,F) sliding-window memory experiment (Sec. III).  For each window:
 * decode, then commit the window's committed columns: XOR their full
 * detector sets into the running syndrome (this is s_{r+1}' = s_{r+1} +
 * H_2 e_1, Eq. (10)) and their observable masks into the prediction.  After a
 * commit the committed blocks must read all zero (Eq. (11)); the final
 * prediction must equal the sampled observables (Eq. (12)).
 */
int qdo_run_shots(const qdo_dem* d, const qdo_params* P, const uint32_t* det_bits,
                  const uint32_t* obs_bits, int64_t n_shots, uint8_t* fail, uint32_t* obs_pred,
                  uint32_t* win_corr_words, int corr_words_per_window) {
  int W = P->W, F = P->F, w = qdo__w(d), ndet = qdo__ndet(d);
  int nwin = qdo_n_windows(d, W, F);
  int dw = (ndet + 31) / 32;
  const int* cptr = qdo__col_ptr(d);
  const int* cdet = qdo__col_dets(d);
  const uint32_t* cobs = qdo__col_obs(d);
  window_t* wins = malloc(sizeof(window_t) * nwin);
  int maxr = 0, maxc = 0;
  for (int k = 0; k < nwin; ++k) {
    window_build(d, W, F, k, P->merge_h1, &wins[k]);
    if (wins[k].nr > maxr) maxr = wins[k].nr;
    if (wins[k].nc > maxc) maxc = wins[k].nc;
  }
  uint32_t* det = malloc(sizeof(uint32_t) * dw);
  uint8_t* synd = malloc(maxr + 1);
  uint8_t* corr = malloc(maxc + 1);
  /* message reuse: what window k - 1 kept per column, and the window k
   * column of every DEM column (-1: none) */
  float* kept = malloc(sizeof(float) * (maxc + 1));
  float* init = malloc(sizeof(float) * (maxc + 1));
  int* at = malloc(sizeof(int) * (qdo__ncols(d) + 1));
  for (int64_t sh = 0; sh < n_shots; ++sh) {
    memcpy(det, det_bits + sh * dw, sizeof(uint32_t) * dw);
    uint32_t pred = 0;
    int fl = 0;
    for (int k = 0; k < nwin; ++k) {
      window_t* wd = &wins[k];
      int row0 = wd->r0 * w;
      for (int j = 0; j < wd->nr; ++j) synd[j] = (det[(row0 + j) >> 5] >> ((row0 + j) & 31)) & 1;
      const int reuse = P->reuse_msgs && k > 0;
      if (reuse) {  /* a column reuses what window k - 1 kept for the same DEM column */
        for (int c = 0; c < qdo__ncols(d); ++c) at[c] = -1;
        for (int c = 0; c < wins[k - 1].nc; ++c) at[wins[k - 1].gcols[c]] = c;
        for (int c = 0; c < wd->nc; ++c) init[c] = at[wd->gcols[c]] >= 0 ? kept[at[wd->gcols[c]]] : NAN;
      }
      decode_window_impl(wd, P, synd, corr, NULL, NULL, NULL, NULL, NULL, reuse ? init : NULL,
                         P->reuse_msgs ? kept : NULL, NULL);
      if (win_corr_words) {
        uint32_t* o = win_corr_words + ((size_t)sh * nwin + k) * corr_words_per_window;
        memset(o, 0, sizeof(uint32_t) * corr_words_per_window);
        for (int c = 0; c < wd->nc; ++c)
          if (corr[c]) o[c >> 5] |= 1u << (c & 31);
      }
      for (int c = 0; c < wd->nc; ++c) {
        if (!wd->commit[c] || !corr[c]) continue;
        int gc = wd->gcols[c];
        for (int e = cptr[gc]; e < cptr[gc + 1]; ++e) det[cdet[e] >> 5] ^= 1u << (cdet[e] & 31);
        pred ^= cobs[gc];
      }
      int cb1 = wd->last ? wd->r0 + wd->nb : wd->r0 + F;
      for (int q = wd->r0 * w; q < cb1 * w; ++q)
        if ((det[q >> 5] >> (q & 31)) & 1) fl |= 1;
    }
    if (pred != obs_bits[sh]) fl |= 2;
    fail[sh] = (uint8_t)fl;
    if (obs_pred) obs_pred[sh] = pred;
  }
  free(det);
  free(synd);
  free(corr);
  free(kept);
  free(init);
  free(at);
  for (int k = 0; k < nwin; ++k) window_free(&wins[k]);
  free(wins);
  return 0;
}
