/*
 * qdo.h -- CPU ORACLE for the sliding-window GDG decoder of
 * "Toward Low-latency Iterative Decoding of QLDPC Codes Under Circuit-Level
 * Noise" (Gong, Cammerer, Renes).
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, slow C implementation exists so that
 * the tests can check the CUDA library against the paper.  Nothing in the
 * product package may include, link or call it; only tests/, the smoke check
 * of __graft_entry__ and the cpu_baseline / reference leg of bench.py use it.
 * It shares no source with the CUDA library.
 *
 * Every function cites the passage of the paper it follows.  All arithmetic on
 * LLRs is IEEE FP32, evaluated in the order the comments state, compiled with
 * -ffp-contract=off so no multiply-add is fused.
 */
#ifndef QDO_H
#define QDO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Bivariate-bicycle code: A = sum_k x^{ax[k]} y^{ay[k]}, B likewise (three
 * monomials each, in the order the polynomial is written). */
typedef struct {
  int l, m;
  int ax[3], ay[3], bx[3], by[3];
} qdo_code;

/* Decoder parameters (Alg. 1-3, Sec. III, Sec. IV). */
typedef struct {
  int W, F;              /* window size and commit size in syndrome rounds     */
  float alpha;           /* min-sum normalisation (Sec. II-A)                  */
  int n_pre;             /* BP iterations on the full window before ranking    */
  int iters_per_step;    /* BP iterations per decimation step (Alg. 2)         */
  int d_max_main;        /* D_max of branch 0                                  */
  int d_max_other;       /* D_max of the other branches                        */
  int k_guess;           /* guessing depths: 2^k branches                      */
  int low_error_mode;    /* 1: Alg. 3 disabled                                 */
  int peel_at_init;      /* peel once before the first BP step                 */
  int shorten;           /* keep only the first 2w' ranked columns             */
  float clip;            /* |VN->CN message| bound (50 in the paper)           */
  float pa_main, pa_other, pb_main, pb_other, pb_d1, pc, pd; /* Alg. 3 */
  int pc_max_depth;      /* P_C test applies for D <= this (4)                 */
  int n_unsat_min;       /* unsatisfied-neighbour count of Alg. 3 (3)          */
  int side_max;          /* side branches of Fig. 2 split off the main branch  */
                         /* at D_split = k .. side_max (0: the 2^k tree only) */
  int reinit_on_split;   /* 1: a path restarts its messages where it splits    */
                         /* off another (appendix, multi-thread snapshots)     */
  int iters_first;       /* BP iterations of step D = 1 (0: iters_per_step)    */
  int merge_h1;          /* Sec. III H_1 merge: 0 off, 1 equal restrictions,   */
                         /* 2 identity with XOR priors (see gdg.c)             */
  int reuse_msgs;        /* Sec. VI: the next window's pre-BP starts from what */
                         /* this window's output path ends with (see gdg.c)    */
  int fallback;          /* output when no path converges (Alg. 2 is silent):  */
                         /* 0 path 0's estimate, 1 fewest unsatisfied checks,  */
                         /* 2 fewest in the committed rows, then in the window */
  /* Learned weighted min-sum (no counterpart in the paper; alpha of Eq. (1)
   * replaced by w[t][e]): wts[k] is window k's array [wT][n_edges] over the
   * full-window edges (CSC order), or NULL for plain alpha.  Iteration t
   * counts from the last message (re)initialisation; t > wT uses row wT. */
  const float* const* wts;
  int wT;
  /* Learned decimation ranker (no counterpart in the paper): NULL for
   * Alg. 1, else 641 raw FP32 parameters W1[64][8], b1[64], W2[64], b2 of
   * score = W2 . relu(W1 x + b1) + b2 over 8 candidate features. */
  const float* ranker;
  /* Candidate dump of path 0 (training data for the ranker; NULL: off): at
   * every selection step, one record per candidate left after Alg. 3, in
   * column order, while *dump_n < dump_cap (*dump_n counts every record). */
  struct qdo_rank_rec* dump;
  int* dump_n;
  int dump_cap;
} qdo_params;

/* One ranker candidate: features x (as the ranker sees them), the window
 * column, the selection depth D and path id; flags bit 0 = [L <= 0] (the
 * value Alg. 1 would give it), bit 1 = the candidate selected at this step. */
typedef struct qdo_rank_rec {
  float x[8];
  int32_t shot, wcol;
  int16_t depth, path;
  int32_t flags;
} qdo_rank_rec;

/* Per-branch summary of one GDG decision path. */
typedef struct {
  int status;      /* 0 converged, 1 reached D_max, 2 contradiction, 3 no candidate */
  int depth;       /* last depth D reached                                   */
  int iters;       /* BP iterations executed on this path                    */
  double pm;       /* path metric Eq. (5); +inf unless converged             */
} qdo_branch_summary;

/* Per-step decision record of one branch. */
typedef struct {
  int g;           /* selected VN (short-column index), -1 if none          */
  int value;       /* value it was decimated to                              */
  int n_agg;       /* VNs fixed by aggressive decimation at this step        */
  int n_peel;      /* VNs fixed by peeling after this step                   */
} qdo_step_record;

typedef struct qdo_dem qdo_dem;

/* ---- code ---- */
int qdo_code_matrices(const qdo_code* c, uint8_t* HX, uint8_t* HZ); /* dense w x 2w each */
int qdo_gf2_rank(const uint8_t* M, int rows, int cols);
int qdo_logical_z(const qdo_code* c, uint8_t* LZ /* K x 2w */, int max_k);
/* Logical operators flipped by errors decoded with H_X: kernel of H_Z modulo
 * the row span of H_X (appendices A and B). */
int qdo_logical_x(const qdo_code* c, uint8_t* LX /* K x 2w */, int max_k);

/* ---- circuit / DEM ---- */
qdo_dem* qdo_dem_build(const qdo_code* c, double p, int rounds);
/* Code-capacity DEM (appendices A, B): BSC(pd) on the data qubits decoded with
 * H_X, and with ps > 0 one virtual column per check ([H_X | I]); one block of
 * w detectors. */
qdo_dem* qdo_dem_code_capacity(const qdo_code* c, double pd, double ps);
void qdo_dem_free(qdo_dem* d);
/* out: n_det, n_cols, n_obs, n_blocks, w, total_col_edges */
void qdo_dem_info(const qdo_dem* d, int* out);
void qdo_dem_columns(const qdo_dem* d, int* col_ptr, int* col_dets, uint32_t* obs,
                     double* prob, float* llr);
/* Simulate one injected X fault at noise location `loc` with pattern bits
 * (bit0 = first qubit, bit1 = second qubit); returns detector list length. */
int qdo_n_fault_locations(const qdo_dem* d);
/* info[4] = (noise kind, n patterns, qubit 0, qubit 1) */
int qdo_fault_effect(const qdo_dem* d, int loc, int pattern, int* dets, int max_dets,
                     uint32_t* obs, int* info);
/* circuit rows (type, q0, q1, aux); returns the number of operations */
int qdo_circuit_ops(const qdo_dem* d, int* out, int max_ops);
int qdo_logical_matrix(const qdo_dem* d, uint8_t* LZ);
int qdo_noiseless_detectors(const qdo_dem* d, uint8_t* dets_out);

/* ---- windows ---- */
int qdo_n_windows(const qdo_dem* d, int W, int F);
/* out: r0, n_blocks_in_window, n_rows, n_cols, n_edges, n_commit, is_last */
int qdo_window_info(const qdo_dem* d, int W, int F, int k, int* out);
int qdo_window_graph(const qdo_dem* d, int W, int F, int k, int* gcols, int* col_ptr,
                     int* col_rows, uint8_t* commit);
/* The window as GDG decodes it, after the H_1 merge `merge` (Sec. III; 0:
 * none): info as qdo_window_info; with gcols != NULL also the columns (DEM
 * column, or a merged class's first member), CSC, commit flags and priors. */
int qdo_window_build(const qdo_dem* d, int W, int F, int k, int merge, int* info, int* gcols, int* col_ptr,
                     int* col_rows, uint8_t* commit, float* llr);

/* ---- sampling (Philox4x32-10, Salmon et al. SC'11) ---- */
void qdo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int qdo_sample(const qdo_dem* d, uint64_t seed, uint64_t shot_offset, int64_t n_shots,
               uint32_t* det_bits, uint32_t* obs_bits);

/* ---- decoding ---- */
/* Min-sum BP on an explicit graph (tests). */
int qdo_bp_run(int n_rows, int n_cols, const int* col_ptr, const int* col_rows,
               const float* llr, const uint8_t* synd, float alpha, float clip,
               int max_iter, int early_stop, uint8_t* e_out, float* post_out);
/* GDG decode of one window: syndrome over the window rows, correction over
 * window columns.  Trace pointers may be NULL. */
int qdo_decode_window(const qdo_dem* d, const qdo_params* P, int k, const uint8_t* synd,
                      uint8_t* corr, int* info /* [4]: prebp_conv, winner, n_short, prebp_iters */,
                      int* short_cols /* 2w' or NULL */, qdo_branch_summary* br /* 2^k or NULL */,
                      qdo_step_record* steps /* 2^k * max(Dmax) or NULL */,
                      int8_t* final_status /* 2^k * n_short or NULL */);
/* qdo_decode_window with message reuse (Sec. VI reading, see gdg.c): init
 * [n_cols] the first VN->CN message of each window column's edges (NaN: its
 * prior; NULL: all priors), keep [n_cols] (may be NULL) receives what the
 * window's output path leaves the next window (NaN: nothing). */
int qdo_decode_window_ex(const qdo_dem* d, const qdo_params* P, int k, const uint8_t* synd, uint8_t* corr,
                         int* info, const float* init, float* keep);
/* qdo_decode_window that also reports every decision path's final estimate:
 * est [n_paths][n_cols] over the window's columns (0 outside the shortened
 * set; untouched when the pre-BP converges).  For tests of the output rule. */
int qdo_decode_window_paths(const qdo_dem* d, const qdo_params* P, int k, const uint8_t* synd, uint8_t* corr,
                            int* info, uint8_t* est);
/* Decode with an explicit graph (column order = index order), no shortening
 * table; for tests on tiny graphs. */
int qdo_gdg_graph(const qdo_params* P, int n_rows, int n_cols, const int* col_ptr,
                  const int* col_rows, const float* llr, const uint8_t* synd,
                  uint8_t* corr, qdo_branch_summary* br);
/* Whole sliding-window memory experiment over n shots.
 * fail[s]: bit0 = Eq. (11) residue, bit1 = Eq. (12) observable mismatch.
 * det_out (may be NULL): detector bits after all commits (residue). */
int qdo_run_shots(const qdo_dem* d, const qdo_params* P, const uint32_t* det_bits,
                  const uint32_t* obs_bits, int64_t n_shots, uint8_t* fail,
                  uint32_t* obs_pred, uint32_t* win_corr_words /* may be NULL */,
                  int corr_words_per_window);

/* Test access to Alg. 3 (one VN: history h[4] oldest first, depth D, main
 * branch flag, unsatisfied-neighbour count): returns 1, 0 or -1. */
int qdo_agg_dec(const qdo_params* P, const float* h, int D, int main_branch, int n_unsat);
/* Test access to one SELECT-VN call (Alg. 1, with Alg. 3 outside the
 * low-error mode) on an explicit graph and path state: hist [4][nc] oldest
 * first (the newest row is the current posterior); status [nc] and synd [nr]
 * (s') are updated with the aggressive decisions.  Returns g or -1. */
int qdo_select_vn(const qdo_params* P, int nr, int nc, const int* col_ptr, const int* col_rows,
                  const float* hist, int8_t* status, uint8_t* synd, int D, int main_branch,
                  int* f_out, int* n_agg);

/* Number of decision paths (2^k tree + side branches) and the largest D_max. */
int qdo_n_paths(const qdo_params* P);
int qdo_path_dmax_all(const qdo_params* P);

/* Ranker scores of n feature rows x [n][8] under raw parameters (641 floats,
 * rounded to the ranker's grids first). */
void qdo_ranker_score(const float* raw, const float* x, int n, float* out);

#ifdef __cplusplus
}
#endif
#endif
