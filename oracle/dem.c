/*
 * dem.c -- CPU ORACLE (test infrastructure only): Z-basis memory circuit of a
 * BB code, circuit-level noise, and the detector error model (DEM) obtained by
 * simulating every single fault DIRECTLY: the X part of the fault is injected
 * and pushed forward gate by gate through the rest of the circuit (a Pauli
 * frame), and the measurement flips it causes are turned into detector and
 * observable flips.
 *
 * Circuit (Sec. II-B, appendix "Stim circuit implementation"; schedule of the
 * depth-8 BB syndrome cycle of Bravyi et al., Fig. 7, cited in Sec. III):
 * qubits X-check ancillas [0,w), L data [w,2w), R data [2w,3w), Z-check
 * ancillas [3w,4w).  One noisy round r = 1..R has eight layers
 *   1: RX(X anc)              CNOT(R[A1^T], Z)          L idle
 *   2: CNOT(X, L[A2])         CNOT(R[A3^T], Z)
 *   3: CNOT(X, R[B2])         CNOT(L[B1^T], Z)
 *   4: CNOT(X, R[B1])         CNOT(L[B2^T], Z)
 *   5: CNOT(X, R[B3])         CNOT(L[B3^T], Z)
 *   6: CNOT(X, L[A1])         CNOT(R[A2^T], Z)
 *   7: CNOT(X, L[A3])         MZ(Z anc)                  R idle
 *   8: MRX(X anc)             RZ(Z anc) (not after R)    L, R idle
 * Before round 1 all data and Z ancillas are reset to |0>.  After round R
 * every data qubit is measured noiselessly in Z (no flips before it).
 * Noise (Sec. II, circuit-level depolarizing model with one rate p):
 * DEPOLARIZE2(p) after each CNOT, DEPOLARIZE1(p) on each idle qubit, X flip
 * with probability p after each Z-basis reset and before each Z measurement.
 * Z-type faults are invisible to the Z-basis experiment (Sec. II decodes X and
 * Z separately), so a channel contributes one mechanism per distinct X pattern:
 * XI, IX, XX with 4p/15 each for DEPOLARIZE2, X with 2p/3 for DEPOLARIZE1.
 *
 * Detectors (Sec. II-B): block 0 holds m_1, block b in 1..R-1 holds
 * m_{b+1} xor m_b, block R holds the readout syndrome H_Z d xor m_R.
 * Observables: K logical Z operators read from d (Eq. (12)).
 *
 * Merging (Sec. II-B): mechanisms with the same detectors and observables
 * merge into one column; their probabilities combine as independent flips,
 * p <- p(1-q) + q(1-p), taken in ascending order of q.  Prior LLR (Sec. II-A)
 * Lambda = log((1-p)/p) in double, rounded to float.
 * Columns are ordered by their sorted detector lists (lexicographically, a
 * proper prefix first) and then by observable mask.
 */
#include "qdo.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { OP_CNOT = 0, OP_MZ = 1, OP_RZ = 2, OP_RX = 3, OP_MRX = 4, OP_NOISE = 5 };
enum { NZ_DEP2 = 0, NZ_DEP1 = 1, NZ_XERR = 2 };

typedef struct { int type, q0, q1, aux; double p; } op_t; /* aux: record index / noise kind */

typedef struct {
  int n_det;
  int* dets;
  uint32_t obs;
  double p;
} mech_t;

struct qdo_dem {
  qdo_code code;
  int w, R, K, nq, n_meas, n_det;
  double p;
  op_t* ops;
  int n_ops;
  int* noise_ops; /* op indices of noise locations */
  int n_noise;
  uint8_t* HZ;    /* w x 2w */
  uint8_t* LZ;    /* K x 2w */
  /* merged columns */
  int n_cols;
  int* col_ptr;
  int* col_dets;
  uint32_t* col_obs;
  double* col_p;
  float* col_llr;
};

/* partner of check i under the monomial matrix M (w x w, one 1 per row/col) */
static int row_partner(const uint8_t* M, int w, int i) {
  for (int j = 0; j < w; ++j)
    if (M[(size_t)i * w + j]) return j;
  return -1;
}
static int col_partner(const uint8_t* M, int w, int i) {
  for (int j = 0; j < w; ++j)
    if (M[(size_t)j * w + i]) return j;
  return -1;
}

/* dense x^a y^b (same construction as bbcode.c, repeated to stay local) */
static void mono_dense(int l, int m, int a, int b, uint8_t* out) {
  int w = l * m;
  memset(out, 0, (size_t)w * w);
  for (int i1 = 0; i1 < l; ++i1)
    for (int i2 = 0; i2 < m; ++i2) {
      int j1 = (i1 + a) % l, j2 = (i2 + b) % m;
      out[(size_t)(i1 * m + i2) * w + (j1 * m + j2)] = 1;
    }
}

static void push_op(qdo_dem* d, int cap_hint, int type, int q0, int q1, int aux, double p) {
  (void)cap_hint;
  op_t o = {type, q0, q1, aux, p};
  d->ops[d->n_ops++] = o;
}

static void build_circuit(qdo_dem* d) {
  const qdo_code* c = &d->code;
  int l = c->l, m = c->m, w = l * m, R = d->R;
  double p = d->p;
  uint8_t* Ak[3];
  uint8_t* Bk[3];
  for (int k = 0; k < 3; ++k) {
    Ak[k] = malloc((size_t)w * w);
    Bk[k] = malloc((size_t)w * w);
    mono_dense(l, m, c->ax[k], c->ay[k], Ak[k]);
    mono_dense(l, m, c->bx[k], c->by[k], Bk[k]);
  }
  int XA = 0, LD = w, RD = 2 * w, ZA = 3 * w;
  size_t cap = (size_t)(R + 1) * (64 * (size_t)w + 16);
  d->ops = malloc(sizeof(op_t) * cap);
  d->n_ops = 0;
  int rec = 0;
  /* initialisation: data and Z ancillas to |0>, X flip after reset */
  for (int q = 0; q < 2 * w; ++q) {
    push_op(d, 0, OP_RZ, LD + q, -1, 0, 0);
    push_op(d, 0, OP_NOISE, LD + q, -1, NZ_XERR, p);
  }
  for (int i = 0; i < w; ++i) {
    push_op(d, 0, OP_RZ, ZA + i, -1, 0, 0);
    push_op(d, 0, OP_NOISE, ZA + i, -1, NZ_XERR, p);
  }
  for (int r = 1; r <= R; ++r) {
    /* layer 1 */
    for (int i = 0; i < w; ++i) push_op(d, 0, OP_RX, XA + i, -1, 0, 0);
    for (int i = 0; i < w; ++i) {
      int j = col_partner(Ak[0], w, i);
      push_op(d, 0, OP_CNOT, RD + j, ZA + i, 0, 0);
      push_op(d, 0, OP_NOISE, RD + j, ZA + i, NZ_DEP2, p);
    }
    for (int i = 0; i < w; ++i) push_op(d, 0, OP_NOISE, LD + i, -1, NZ_DEP1, p);
    /* layers 2..7: X-check target, Z-check control */
    struct { int xmat, xk, xside, zmat, zk, zside; } L[6] = {
        {0, 1, 0, 0, 2, 1}, /* 2: X->L[A2], R[A3^T]->Z */
        {1, 1, 1, 1, 0, 0}, /* 3: X->R[B2], L[B1^T]->Z */
        {1, 0, 1, 1, 1, 0}, /* 4: X->R[B1], L[B2^T]->Z */
        {1, 2, 1, 1, 2, 0}, /* 5: X->R[B3], L[B3^T]->Z */
        {0, 0, 0, 0, 1, 1}, /* 6: X->L[A1], R[A2^T]->Z */
        {0, 2, 0, -1, 0, 0} /* 7: X->L[A3] */
    };
    for (int t = 0; t < 6; ++t) {
      for (int i = 0; i < w; ++i) {
        const uint8_t* Mx = L[t].xmat == 0 ? Ak[L[t].xk] : Bk[L[t].xk];
        int j = row_partner(Mx, w, i);
        int tgt = (L[t].xside == 0 ? LD : RD) + j;
        push_op(d, 0, OP_CNOT, XA + i, tgt, 0, 0);
        push_op(d, 0, OP_NOISE, XA + i, tgt, NZ_DEP2, p);
      }
      if (L[t].zmat >= 0) {
        for (int i = 0; i < w; ++i) {
          const uint8_t* Mz = L[t].zmat == 0 ? Ak[L[t].zk] : Bk[L[t].zk];
          int j = col_partner(Mz, w, i);
          int ctl = (L[t].zside == 0 ? LD : RD) + j;
          push_op(d, 0, OP_CNOT, ctl, ZA + i, 0, 0);
          push_op(d, 0, OP_NOISE, ctl, ZA + i, NZ_DEP2, p);
        }
      } else {
        /* layer 7: measure Z ancillas (flip before), R data idle */
        for (int i = 0; i < w; ++i) {
          push_op(d, 0, OP_NOISE, ZA + i, -1, NZ_XERR, p);
          push_op(d, 0, OP_MZ, ZA + i, -1, rec++, 0);
        }
        for (int i = 0; i < w; ++i) push_op(d, 0, OP_NOISE, RD + i, -1, NZ_DEP1, p);
      }
    }
    /* layer 8 */
    for (int i = 0; i < w; ++i) push_op(d, 0, OP_MRX, XA + i, -1, 0, 0);
    if (r < R)
      for (int i = 0; i < w; ++i) {
        push_op(d, 0, OP_RZ, ZA + i, -1, 0, 0);
        push_op(d, 0, OP_NOISE, ZA + i, -1, NZ_XERR, p);
      }
    for (int q = 0; q < 2 * w; ++q) push_op(d, 0, OP_NOISE, LD + q, -1, NZ_DEP1, p);
  }
  d->n_meas = rec;
  d->noise_ops = malloc(sizeof(int) * d->n_ops);
  d->n_noise = 0;
  for (int k = 0; k < d->n_ops; ++k)
    if (d->ops[k].type == OP_NOISE) d->noise_ops[d->n_noise++] = k;
  for (int k = 0; k < 3; ++k) {
    free(Ak[k]);
    free(Bk[k]);
  }
}

/*
 * Forward Pauli-frame simulation of one injected X pattern placed right after
 * op index `start` (a noise location).  Writes the flipped detectors (sorted)
 * and the observable mask.
 */
static int simulate(const qdo_dem* d, int start, const int* xq, int nxq, int* dets, uint32_t* obs) {
  int w = d->w, R = d->R, nq = d->nq;
  uint8_t* fr = calloc(nq, 1);
  uint8_t* mf = calloc(d->n_meas, 1);
  for (int k = 0; k < nxq; ++k) fr[xq[k]] ^= 1;
  for (int k = start + 1; k < d->n_ops; ++k) {
    const op_t* o = &d->ops[k];
    switch (o->type) {
      case OP_CNOT: fr[o->q1] ^= fr[o->q0]; break;   /* X on control spreads to target */
      case OP_MZ: mf[o->aux] ^= fr[o->q0]; break;    /* X flips a Z measurement */
      case OP_RZ: case OP_RX: case OP_MRX: fr[o->q0] = 0; break; /* reset erases it */
      default: break;
    }
  }
  /* final noiseless data readout d = frame on the data qubits */
  const uint8_t* dd = fr + w;
  int nd = 0;
  for (int b = 0; b <= R; ++b)
    for (int i = 0; i < w; ++i) {
      int v;
      if (b == 0) v = mf[i];
      else if (b < R) v = mf[b * w + i] ^ mf[(b - 1) * w + i];
      else {
        v = mf[(R - 1) * w + i];
        for (int q = 0; q < 2 * w; ++q) v ^= d->HZ[(size_t)i * 2 * w + q] & dd[q];
      }
      if (v) dets[nd++] = b * w + i;
    }
  uint32_t om = 0;
  for (int kk = 0; kk < d->K; ++kk) {
    int v = 0;
    for (int q = 0; q < 2 * w; ++q) v ^= d->LZ[(size_t)kk * 2 * w + q] & dd[q];
    if (v) om |= 1u << kk;
  }
  *obs = om;
  free(fr);
  free(mf);
  return nd;
}

static int n_patterns(int kind) { return kind == NZ_DEP2 ? 3 : 1; }
static double pattern_prob(int kind, double p) {
  if (kind == NZ_DEP2) return 4.0 * p / 15.0;
  if (kind == NZ_DEP1) return 2.0 * p / 3.0;
  return p;
}

static int cmp_mech(const mech_t* a, const mech_t* b) {
  int n = a->n_det < b->n_det ? a->n_det : b->n_det;
  for (int k = 0; k < n; ++k)
    if (a->dets[k] != b->dets[k]) return a->dets[k] < b->dets[k] ? -1 : 1;
  if (a->n_det != b->n_det) return a->n_det < b->n_det ? -1 : 1;
  if (a->obs != b->obs) return a->obs < b->obs ? -1 : 1;
  return 0;
}
static int cmp_mech_q(const void* x, const void* y) {
  int c = cmp_mech((const mech_t*)x, (const mech_t*)y);
  if (c) return c;
  double a = ((const mech_t*)x)->p, b = ((const mech_t*)y)->p;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* Sort the mechanisms by (detectors, observables, probability) so equal
 * columns are adjacent with their probabilities ascending, merge them into
 * the DEM's columns (Sec. II-B) and free them. */
static void merge_mechanisms(qdo_dem* d, mech_t* ms, int nm) {
  qsort(ms, nm, sizeof(mech_t), cmp_mech_q);
  d->col_ptr = malloc(sizeof(int) * (nm + 1));
  d->col_obs = malloc(sizeof(uint32_t) * nm);
  d->col_p = malloc(sizeof(double) * nm);
  d->col_llr = malloc(sizeof(float) * nm);
  int tot = 0;
  for (int k = 0; k < nm; ++k) tot += ms[k].n_det;
  d->col_dets = malloc(sizeof(int) * (tot > 0 ? tot : 1));
  int nc = 0, ne = 0;
  d->col_ptr[0] = 0;
  for (int k = 0; k < nm;) {
    int e = k;
    double pm = 0.0;
    while (e < nm && cmp_mech(&ms[k], &ms[e]) == 0) {
      double q = ms[e].p;
      pm = pm * (1.0 - q) + q * (1.0 - pm);
      ++e;
    }
    memcpy(d->col_dets + ne, ms[k].dets, sizeof(int) * ms[k].n_det);
    ne += ms[k].n_det;
    d->col_ptr[nc + 1] = ne;
    d->col_obs[nc] = ms[k].obs;
    d->col_p[nc] = pm;
    d->col_llr[nc] = (float)log((1.0 - pm) / pm);
    ++nc;
    k = e;
  }
  d->n_cols = nc;
  for (int k = 0; k < nm; ++k) free(ms[k].dets);
  free(ms);
}

qdo_dem* qdo_dem_build(const qdo_code* c, double p, int rounds) {
  qdo_dem* d = calloc(1, sizeof(qdo_dem));
  d->code = *c;
  d->w = c->l * c->m;
  d->R = rounds;
  d->p = p;
  d->nq = 4 * d->w;
  int n = 2 * d->w;
  d->HZ = malloc((size_t)d->w * n);
  uint8_t* HX = malloc((size_t)d->w * n);
  qdo_code_matrices(c, HX, d->HZ);
  free(HX);
  d->LZ = malloc((size_t)32 * n);
  d->K = qdo_logical_z(c, d->LZ, 32);
  build_circuit(d);
  d->n_det = (rounds + 1) * d->w;
  /* every fault mechanism, simulated directly */
  int cap = 0;
  for (int k = 0; k < d->n_noise; ++k) cap += n_patterns(d->ops[d->noise_ops[k]].aux);
  mech_t* ms = malloc(sizeof(mech_t) * cap);
  int nm = 0;
  int* tmp = malloc(sizeof(int) * d->n_det);
  for (int k = 0; k < d->n_noise; ++k) {
    const op_t* o = &d->ops[d->noise_ops[k]];
    for (int pat = 1; pat <= n_patterns(o->aux); ++pat) {
      int xq[2], nx = 0;
      if (pat & 1) xq[nx++] = o->q0;
      if (pat & 2) xq[nx++] = o->q1;
      uint32_t om;
      int nd = simulate(d, d->noise_ops[k], xq, nx, tmp, &om);
      if (nd == 0 && om == 0) continue; /* invisible to the Z-basis experiment */
      ms[nm].n_det = nd;
      ms[nm].dets = malloc(sizeof(int) * (nd > 0 ? nd : 1));
      memcpy(ms[nm].dets, tmp, sizeof(int) * nd);
      ms[nm].obs = om;
      ms[nm].p = pattern_prob(o->aux, p);
      ++nm;
    }
  }
  free(tmp);
  merge_mechanisms(d, ms, nm);
  return d;
}

/*
 * Code-capacity models of the appendices, decoded with H_X: every data qubit
 * flips independently with probability pd (appendix "Data qubit noise",
 * BSC(p_d)); block 0 holds the syndrome H_X e.  With ps > 0 every syndrome
 * bit also flips with probability ps, one virtual column per check (appendix
 * "Single shot syndrome noise", [H_X | I]), and a second, noiseless block
 * holds H_X e of the data error alone: a window over block 0 decodes, and the
 * Eq. (11) residue of block 1 after the commit is the appendix's success
 * test (the data estimate must reproduce the true data syndrome).  The
 * observables are the logical operators such errors can flip (kernel of H_Z
 * modulo the row span of H_X).  Columns are merged and ordered like the
 * circuit DEM's.
 */
qdo_dem* qdo_dem_code_capacity(const qdo_code* c, double pd, double ps) {
  qdo_dem* d = calloc(1, sizeof(qdo_dem));
  d->code = *c;
  d->w = c->l * c->m;
  d->R = ps > 0.0 ? 1 : 0;
  d->p = pd;
  d->n_det = (d->R + 1) * d->w;
  int w = d->w, n = 2 * w;
  uint8_t* HX = malloc((size_t)w * n);
  d->HZ = malloc((size_t)w * n);
  qdo_code_matrices(c, HX, d->HZ);
  d->LZ = malloc((size_t)32 * n);
  d->K = qdo_logical_x(c, d->LZ, 32);
  int nm = n + (ps > 0.0 ? w : 0);
  mech_t* ms = malloc(sizeof(mech_t) * nm);
  for (int i = 0; i < n; ++i) {
    ms[i].dets = malloc(sizeof(int) * 2 * w);
    ms[i].n_det = 0;
    for (int b = 0; b <= d->R; ++b)
      for (int j = 0; j < w; ++j)
        if (HX[(size_t)j * n + i]) ms[i].dets[ms[i].n_det++] = b * w + j;
    ms[i].obs = 0;
    for (int k = 0; k < d->K; ++k)
      if (d->LZ[(size_t)k * n + i]) ms[i].obs |= 1u << k;
    ms[i].p = pd;
  }
  for (int j = 0; ps > 0.0 && j < w; ++j) {
    mech_t* m = &ms[n + j];
    m->dets = malloc(sizeof(int));
    m->dets[0] = j;
    m->n_det = 1;
    m->obs = 0;
    m->p = ps;
  }
  free(HX);
  merge_mechanisms(d, ms, nm);
  return d;
}

void qdo_dem_free(qdo_dem* d) {
  if (!d) return;
  free(d->ops);
  free(d->noise_ops);
  free(d->HZ);
  free(d->LZ);
  free(d->col_ptr);
  free(d->col_dets);
  free(d->col_obs);
  free(d->col_p);
  free(d->col_llr);
  free(d);
}

void qdo_dem_info(const qdo_dem* d, int* out) {
  out[0] = d->n_det;
  out[1] = d->n_cols;
  out[2] = d->K;
  out[3] = d->R + 1;
  out[4] = d->w;
  out[5] = d->col_ptr[d->n_cols];
}

void qdo_dem_columns(const qdo_dem* d, int* col_ptr, int* col_dets, uint32_t* obs, double* prob,
                     float* llr) {
  memcpy(col_ptr, d->col_ptr, sizeof(int) * (d->n_cols + 1));
  memcpy(col_dets, d->col_dets, sizeof(int) * d->col_ptr[d->n_cols]);
  memcpy(obs, d->col_obs, sizeof(uint32_t) * d->n_cols);
  memcpy(prob, d->col_p, sizeof(double) * d->n_cols);
  memcpy(llr, d->col_llr, sizeof(float) * d->n_cols);
}

int qdo_n_fault_locations(const qdo_dem* d) { return d->n_noise; }

/* Direct simulation of one fault; n_qubits_out[0..1] = (kind, n patterns). */
int qdo_fault_effect(const qdo_dem* d, int loc, int pattern, int* dets, int max_dets,
                     uint32_t* obs, int* info) {
  const op_t* o = &d->ops[d->noise_ops[loc]];
  int xq[2], nx = 0;
  if (pattern & 1) xq[nx++] = o->q0;
  if ((pattern & 2) && o->q1 >= 0) xq[nx++] = o->q1;
  int* tmp = malloc(sizeof(int) * d->n_det);
  int nd = simulate(d, d->noise_ops[loc], xq, nx, tmp, obs);
  for (int k = 0; k < nd && k < max_dets; ++k) dets[k] = tmp[k];
  free(tmp);
  if (info) {
    info[0] = o->aux;
    info[1] = n_patterns(o->aux);
    info[2] = o->q0;
    info[3] = o->q1;
  }
  return nd;
}

/* The circuit as (type, q0, q1, aux) rows for independent checks in tests. */
int qdo_circuit_ops(const qdo_dem* d, int* out, int max_ops) {
  int n = d->n_ops < max_ops ? d->n_ops : max_ops;
  for (int k = 0; k < n; ++k) {
    out[4 * k + 0] = d->ops[k].type;
    out[4 * k + 1] = d->ops[k].q0;
    out[4 * k + 2] = d->ops[k].q1;
    out[4 * k + 3] = d->ops[k].aux;
  }
  return d->n_ops;
}

int qdo_logical_matrix(const qdo_dem* d, uint8_t* LZ) {
  memcpy(LZ, d->LZ, (size_t)d->K * 2 * d->w);
  return d->K;
}

int qdo_noiseless_detectors(const qdo_dem* d, uint8_t* out) {
  uint32_t om;
  int* tmp = malloc(sizeof(int) * d->n_det);
  int nd = simulate(d, -1, NULL, 0, tmp, &om);
  memset(out, 0, d->n_det);
  for (int k = 0; k < nd; ++k) out[tmp[k]] = 1;
  free(tmp);
  return nd + (om ? 1 : 0);
}

/* ------------------------------------------------------------------------ */
/* Sliding windows (Sec. III, Eq. (8)-(10)).  Blocks b = 0..R.  Window k
 * starts at block r = kF and covers blocks [r, min(r+W, R+1)); it is the last
 * window once r + W >= R + 1.  Its columns are the columns whose first
 * detector lies in the window's blocks (the un-committed columns touching its
 * rows), restricted to its rows.  It commits the columns whose first block is
 * in [r, r+F) -- all of its columns when it is the last window. */

int qdo_n_windows(const qdo_dem* d, int W, int F) {
  int B = d->R + 1, k = 0;
  for (int r = 0;; r += F, ++k)
    if (r + W >= B) return k + 1;
}

static void window_range(const qdo_dem* d, int W, int F, int k, int* r0, int* r1, int* last) {
  int B = d->R + 1;
  *r0 = k * F;
  *last = (*r0 + W >= B);
  *r1 = *last ? B : *r0 + W;
}

int qdo_window_info(const qdo_dem* d, int W, int F, int k, int* out) {
  int r0, r1, last, w = d->w;
  window_range(d, W, F, k, &r0, &r1, &last);
  int nc = 0, ne = 0, ncom = 0;
  for (int c = 0; c < d->n_cols; ++c) {
    int a = d->col_ptr[c], b = d->col_ptr[c + 1];
    if (a == b) continue;
    int fb = d->col_dets[a] / w;
    if (fb < r0 || fb >= r1) continue;
    ++nc;
    for (int e = a; e < b; ++e)
      if (d->col_dets[e] / w < r1) ++ne;
    if (last || fb < r0 + F) ++ncom;
  }
  out[0] = r0;
  out[1] = r1 - r0;
  out[2] = (r1 - r0) * w;
  out[3] = nc;
  out[4] = ne;
  out[5] = ncom;
  out[6] = last;
  return 0;
}

int qdo_window_graph(const qdo_dem* d, int W, int F, int k, int* gcols, int* col_ptr, int* col_rows,
                     uint8_t* commit) {
  int r0, r1, last, w = d->w;
  window_range(d, W, F, k, &r0, &r1, &last);
  int nc = 0, ne = 0;
  col_ptr[0] = 0;
  for (int c = 0; c < d->n_cols; ++c) {
    int a = d->col_ptr[c], b = d->col_ptr[c + 1];
    if (a == b) continue;
    int fb = d->col_dets[a] / w;
    if (fb < r0 || fb >= r1) continue;
    gcols[nc] = c;
    for (int e = a; e < b; ++e)
      if (d->col_dets[e] / w < r1) col_rows[ne++] = d->col_dets[e] - r0 * w;
    commit[nc] = (uint8_t)(last || fb < r0 + F);
    ++nc;
    col_ptr[nc] = ne;
  }
  return nc;
}

/* accessors used by gdg.c */
int qdo__w(const qdo_dem* d) { return d->w; }
int qdo__ncols(const qdo_dem* d) { return d->n_cols; }
int qdo__ndet(const qdo_dem* d) { return d->n_det; }
int qdo__R(const qdo_dem* d) { return d->R; }
const int* qdo__col_ptr(const qdo_dem* d) { return d->col_ptr; }
const int* qdo__col_dets(const qdo_dem* d) { return d->col_dets; }
const uint32_t* qdo__col_obs(const qdo_dem* d) { return d->col_obs; }
const double* qdo__col_p(const qdo_dem* d) { return d->col_p; }
const float* qdo__col_llr(const qdo_dem* d) { return d->col_llr; }
