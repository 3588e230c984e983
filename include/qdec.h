/*
 * qdec.h -- C ABI of libqdec: a GB300 (sm_103a) sliding-window decoder for
 * bivariate-bicycle (BB) codes under circuit-level noise, with BP guided
 * decimation guessing (GDG) as the inner decoder (Gong, Cammerer, Renes,
 * "Toward Low-latency Iterative Decoding of QLDPC Codes Under Circuit-Level
 * Noise").
 *
 * Conventions
 *  - Every call returns a qd_status; QD_OK is 0.  On error,
 *    qd_last_error_message() returns a thread-local description.
 *  - Handles (qd_dem, qd_decoder) are owned by the library and released with
 *    the matching *_destroy call.
 *  - Device buffers are owned by the caller.  Pointers marked "device" must
 *    point to GPU memory of the current device; all device work is enqueued
 *    on the given stream and is asynchronous unless stated otherwise.
 *  - Bit vectors are packed little-endian into uint32 words: bit b of a
 *    vector is bit (b mod 32) of word b / 32.  Per-shot arrays are row-major
 *    [n_shots][words].
 *  - Detector d (0 <= d < n_det) belongs to syndrome block d / w, check
 *    d mod w, with w = N/2 checks per round (Fig. 1).
 *  - No entry point allocates device memory after qd_decoder_create.  The
 *    DEM is copied to the device on its first device use (qd_sample_shots
 *    or qd_decoder_create); qd_build_dem itself needs no GPU.
 */
#ifndef QDEC_H
#define QDEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* qd_stream_t; /* a cudaStream_t; NULL = legacy default */

typedef enum {
  QD_OK = 0,
  QD_EINVAL = 1,       /* bad argument (null pointer, size out of range)            */
  QD_ENOMEM = 2,       /* host or device allocation failed                           */
  QD_ECUDA = 3,        /* a CUDA runtime call failed                                 */
  QD_ETIMEOUT = 4,     /* a bounded device wait gave up                              */
  QD_EUNSUPPORTED = 5  /* parameter combination this build does not implement        */
} qd_status;

/* A BB code (appendix "Single shot syndrome noise"): H_X = [A | B],
 * H_Z = [B^T | A^T], A = sum_k x^{a_x[k]} y^{a_y[k]}, B likewise, with
 * x = S_l (x) I_m, y = I_l (x) S_m.  The order of the three terms fixes which
 * term each CNOT layer of the syndrome circuit uses. */
typedef struct {
  int l, m;
  int a_x[3], a_y[3];
  int b_x[3], b_y[3];
} qd_bb_code;

/* Circuit-level depolarizing noise of rate p (Sec. II) on a Z-basis memory
 * experiment of `rounds` noisy syndrome rounds followed by a noiseless data
 * readout (appendix "Stim circuit implementation"). */
typedef struct {
  double p;
  int rounds;
} qd_noise;

/* GDG decoder parameters (Sec. III, Sec. IV, Alg. 1-3, Fig. 2). */
typedef struct {
  int W, F;              /* (W,F) sliding window, in syndrome rounds (Sec. III)   */
  float alpha;           /* normalised min-sum factor (Sec. II-A)                 */
  int n_pre;             /* BP iterations on the full window before ranking       */
  int iters_per_step;    /* BP iterations per decimation step; >= 4 on the GPU    */
  int d_max_main;        /* D_max of path 0 (the main branch)                     */
  int d_max_other;       /* D_max of every other path                             */
  int k_guess;           /* guessing depths: 2^k decision paths, 0 <= k <= 5      */
  int low_error_mode;    /* 1 disables aggressive decimation (Alg. 3)             */
  int peel_at_init;      /* peel degree-one checks once before the first step    */
  int shorten;           /* GDG on the first 2w' ranked columns only (Sec. III)   */
  float clip;            /* bound on |VN->CN| messages (50 in the paper)          */
  float pa_main, pa_other, pb_main, pb_other, pb_d1, pc, pd; /* Alg. 3 thresholds */
  int pc_max_depth;      /* P_C applies while D <= this                           */
  int n_unsat_min;       /* unsatisfied-neighbour count of Alg. 3                 */
  int side_max;          /* side branches of Fig. 2 split off the main branch at  */
                         /* D_split = k .. side_max and run D_split +            */
                         /* (d_max_other - k) steps; 0: the 2^k tree only.       */
                         /* With side branches id 1 (contrary only at D = k) is  */
                         /* the D_split = k side branch; ids 2^k.. the others.   */
  int reinit_on_split;   /* 1: a path that continues from another's status (side  */
                         /* branches at D_split, odd tree ids at D = k) restarts  */
                         /* its messages there, mu = Lambda (the appendix's       */
                         /* multi-thread snapshots); 0: continuous messages.      */
  int iters_first;       /* BP iterations of the first decimation step (D = 1);   */
                         /* 0: iters_per_step.  With n_pre = 0 and shorten = 0    */
                         /* this is the reading in which the initial BP run is    */
                         /* GDG's own first step on the whole window; >= 4 on     */
                         /* the GPU when set.                                     */
  int merge_h1;          /* Sec. III: the window's H_1 columns (those reaching    */
                         /* past its last block) merged toward an identity:       */
                         /* 0 off; 1 columns with equal restrictions to the       */
                         /* window merged (probabilities XOR-combined; the        */
                         /* window's parity-check problem unchanged); 2 replaced  */
                         /* by one column per last-block detector with the XOR    */
                         /* of the H_1 columns holding it.  Not in the last       */
                         /* window, and only with W > F (never committed).        */
  int reuse_msgs;        /* Sec. VI (future work there): 1 = the next window's    */
                         /* pre-BP starts the first VN->CN messages of every      */
                         /* column it shares with this window from what this      */
                         /* window's output path ends with (final posterior;      */
                         /* +-clip for a column decimated to 0 / 1; the pre-BP's  */
                         /* posterior when the pre-BP converged); other columns   */
                         /* start from their prior.  Windows must be decoded in   */
                         /* order, each call on the same shots; window 0 starts   */
                         /* from the priors.  Not in batched steps.               */
  int fallback;          /* the window's output when no decision path converges  */
                         /* (Alg. 2 leaves it open): 0 path 0's estimate; 1 the  */
                         /* estimate with the fewest unsatisfied checks of the    */
                         /* window; 2 the fewest among the checks the window      */
                         /* commits (its first F blocks; all in the last window), */
                         /* then among all.  Ties go to the lowest path id.       */
} qd_gdg_params;

typedef struct qd_dem qd_dem;
typedef struct qd_decoder qd_decoder;

typedef struct {
  int n_det;       /* detectors = (rounds + 1) * w                            */
  int n_cols;      /* fault mechanisms (DEM columns) after merging            */
  int n_obs;       /* logical observables K                                   */
  int n_blocks;    /* rounds + 1                                              */
  int w;           /* checks per round, N/2                                   */
  int det_words;   /* ceil(n_det / 32)                                        */
  int n_edges;     /* nonzeros of the DEM parity-check matrix                 */
} qd_dem_info_t;

typedef struct {
  int r0;          /* first syndrome block of the window                       */
  int n_blocks;    /* blocks covered                                           */
  int n_rows;      /* detectors in the window (n_blocks * w)                   */
  int n_cols;      /* window columns (un-committed faults touching its rows)   */
  int n_edges;     /* nonzeros of the window matrix                            */
  int n_commit;    /* committed columns: window columns [0, n_commit)          */
  int is_last;     /* the last window commits all of its columns               */
  int n_short;     /* columns GDG runs on (2w' or all)                         */
} qd_window_info_t;

const char* qd_last_error_message(void);

/*
 * Build the detector error model of the Z-basis memory experiment
 * (Sec. II-B): every single fault location of the circuit, X part only, is
 * mapped to the detectors and observables it flips; mechanisms with the same
 * detectors and observables merge with p <- p(1-q) + q(1-p), ascending q.
 * Columns are in canonical order (sorted detector lists, then observable
 * mask).  Host-side work; needs no GPU.
 * Errors: QD_EINVAL for l, m < 1, rounds < 1, p outside (0, 0.5).
 */
qd_status qd_build_dem(const qd_bb_code* code, const qd_noise* noise, qd_dem** out);

/*
 * Code-capacity models of the appendices, decoded with H_X = [A|B]:
 *   p_synd = 0: every data qubit flips with probability p_data (appendix
 *     "Data qubit noise", BSC(p_d)); one block of w detectors, H_X e.
 *   p_synd > 0: also every syndrome bit flips with probability p_synd, one
 *     virtual column per check (appendix "Single shot syndrome noise",
 *     [H_X | I]); block 0 holds the noisy syndrome H_X e + s', a noiseless
 *     block 1 holds H_X e.  Decode with W = F = 1: window 0 decides every
 *     column, window 1 has none and its commit's Eq. (11) residue is the
 *     appendix's success test (the data estimate must have the data syndrome).
 * Observables: a basis of the kernel of H_Z independent of the row span of
 * H_X.  Same ownership and errors as qd_build_dem.
 */
qd_status qd_build_dem_code_capacity(const qd_bb_code* code, double p_data, double p_synd, qd_dem** out);
qd_status qd_dem_info(const qd_dem* dem, qd_dem_info_t* out);
/* Host copies of the DEM (CSC over detectors): col_ptr[n_cols+1],
 * col_dets[n_edges], obs[n_cols], prob[n_cols], llr[n_cols] (Lambda_i =
 * log((1-p_i)/p_i), Sec. II-A).  Any pointer may be NULL. */
qd_status qd_dem_columns(const qd_dem* dem, int* col_ptr, int* col_dets, uint32_t* obs,
                         double* prob, float* llr);
/* Window k of the (W,F) schedule as the decoder builds it (Sec. III, Eq. (8);
 * host only, no device call), after the H_1 merge `merge_h1` (see
 * qd_gdg_params; 0: none): info[7] = (first block, blocks, rows, columns,
 * edges, committed columns, last window); with gcols != NULL also gcols[n_cols]
 * (DEM column, or a merged class's first member), col_ptr[n_cols+1],
 * col_rows[n_edges] (window rows, ascending per column) and llr[n_cols]
 * (the priors GDG uses).  QD_EINVAL for a bad window index or a merged prior
 * outside (2^-15, 16). */
qd_status qd_dem_window(const qd_dem* dem, int W, int F, int k, int merge_h1, int info[7], int* gcols,
                        int* col_ptr, int* col_rows, float* llr);
/* Shot mode's decision-path plan for parameters p and `wave` warps (host
 * only; see qd_decoder_set_fork): info = (paths nb, deepest D_max dmx, nodes
 * or -1 when there is no plan: nb <= wave); with order != NULL also the queue
 * order[nb], chain[nb][dmx] (the snapshot node of path q after the BP of step
 * D at chain[q * dmx + D - 1], -1: none), fnode[nb] / fdep[nb] (each path's
 * planned resume node and its depth, -1 / 0: none).  Paths with equal
 * decisions at depths 1..D-1 -- guess value (Alg. 2, Fig. 2), Alg. 3's
 * thresholds, message restart -- share the node of depth D. */
qd_status qd_path_plan(const qd_gdg_params* p, int wave, int info[3], int16_t* order, int16_t* chain, int16_t* fnode,
                       int16_t* fdep);
qd_status qd_dem_destroy(qd_dem* dem);

/*
 * Sample n_shots Monte-Carlo shots of the DEM on the GPU.  Shot s (global
 * index shot_offset + s) fires column c iff u < round(p_c 2^32), where u is
 * word (c mod 4) of Philox4x32-10(counter = (c/4, s_lo, s_hi, 0),
 * key = (seed_lo, seed_hi)); detectors and observables are the XOR of the
 * fired columns (s = H e, l = L e, Sec. III).
 * det_bits: device, [n_shots][det_words]; obs_bits: device, [n_shots] (bit k =
 * observable k).  Errors: QD_EINVAL on null pointers or n_shots < 0.
 */
qd_status qd_sample_shots(const qd_dem* dem, uint64_t seed, uint64_t shot_offset, int64_t n_shots,
                          uint32_t* det_bits, uint32_t* obs_bits, qd_stream_t stream);

/*
 * Prepare the (W,F) window matrices (Eq. (8)) and the GPU launch plan for
 * batches of up to max_shots shots.  Allocates all device scratch (windows
 * whose pre-BP scratch or path slots exceed shared memory get a region in
 * global memory).  Errors: QD_EINVAL for bad parameters or a window with
 * 2^15 or more rows or columns (or 65535 edges); QD_EUNSUPPORTED when
 * iters_per_step < 4, k_guess > 5, or a window whose persistent part alone
 * exceeds shared memory.
 */
qd_status qd_decoder_create(const qd_dem* dem, const qd_gdg_params* params, int64_t max_shots,
                            qd_decoder** out);
qd_status qd_decoder_destroy(qd_decoder* dec);
qd_status qd_decoder_n_windows(const qd_decoder* dec, int* n_windows);
/* Words per shot of the window-correction buffer (max over windows). */
qd_status qd_decoder_corr_words(const qd_decoder* dec, int* corr_words);
/* out = {number of decision paths (2^k + side branches), largest D_max}: the
 * branch and step dimensions of the trace. */
qd_status qd_decoder_path_info(const qd_decoder* dec, int out[2]);
/* Window k's shape and, if gcols != NULL, its DEM column ids [n_cols]. */
qd_status qd_window_info(const qd_decoder* dec, int k, qd_window_info_t* out, int* gcols);
/* Bytes of the optional per-shot trace written by qd_decode_windows. */
qd_status qd_decoder_trace_bytes(const qd_decoder* dec, size_t* bytes_per_shot);

/*
 * Decode window k of every shot (Sec. III + Sec. IV): n_pre flooding
 * min-sum iterations on the window with early stop; if they do not satisfy
 * the window syndrome, rank columns by the sum of the last four posteriors
 * and run GDG (Alg. 2, 2^k paths, Alg. 1 selection, Alg. 3 aggressive
 * decimation, peeling) on the first 2w' columns; the output is the estimate
 * of least path metric (Eq. (5)).  The window syndrome is read from det_bits
 * rows [r0*w, (r0+n_blocks)*w) (call qd_commit_and_slide for windows 0..k-1
 * first).
 *   det_bits       device [n_shots][det_words], read only
 *   win_correction device [n_shots][corr_words], out: bit c = estimate of
 *                  window column c
 *   status         device [n_shots] or NULL, out: winning path id, -1 when
 *                  the pre-BP converged, -2 when no path converged
 *   trace          device, n_shots * trace_bytes, or NULL
 * Errors: QD_EINVAL (k out of range, n_shots > max_shots, null pointers).
 */
qd_status qd_decode_windows(qd_decoder* dec, int k, const uint32_t* det_bits, int64_t n_shots,
                            uint32_t* win_correction, int32_t* status, void* trace,
                            qd_stream_t stream);

/*
 * Commit window k (Sec. III, Eq. (10)): XOR the full detector sets of the
 * committed columns whose estimate is 1 into det_bits (this is
 * s_{r+1}' = s_{r+1} + H_2 e_1), XOR their observable masks into obs_pred,
 * and set bit 0 of residue_fail when a committed block is left non-zero
 * (Eq. (11) fails).
 *   det_bits device [n_shots][det_words], updated in place
 *   obs_pred device [n_shots], updated in place (start from 0)
 *   residue_fail device [n_shots], updated in place (start from 0)
 */
qd_status qd_commit_and_slide(qd_decoder* dec, int k, const uint32_t* win_correction,
                              int64_t n_shots, uint32_t* det_bits, uint32_t* obs_pred,
                              uint32_t* residue_fail, qd_stream_t stream);

/*
 * Success test (Sec. III, appendix "Stim circuit implementation"): a shot
 * fails when Eq. (11) failed in some window (bit 0) or L e differs from the
 * sampled observables, Eq. (12) (bit 1).  fail: device [n_shots] out;
 * n_fail: device int64 counter, incremented by the number of failed shots.
 */
qd_status qd_evaluate(const uint32_t* obs_pred, const uint32_t* obs_true,
                      const uint32_t* residue_fail, int64_t n_shots, uint32_t* fail,
                      long long* n_fail, qd_stream_t stream);

/*
 * Whole sliding-window pass on device buffers: for k = 0..n_windows-1
 * decode window k and commit it, then evaluate.  det_bits is consumed (holds
 * the residues afterwards); obs_pred, fail: device [n_shots] out; n_fail:
 * device int64 accumulator (may be NULL).  Uses the decoder's own scratch
 * for window corrections.
 */
qd_status qd_decode_all(qd_decoder* dec, uint32_t* det_bits, const uint32_t* obs_true,
                        int64_t n_shots, uint32_t* obs_pred, uint32_t* fail, long long* n_fail,
                        qd_stream_t stream);

/*
 * qd_decode_all on HOST buffers: copies det_bits / obs_true to the device,
 * decodes, and copies obs_pred and fail back (pageable or pinned host
 * memory).  Synchronous: returns when the outputs are on the host.
 *   det_bits [n_shots][det_words], obs_true [n_shots] in
 *   obs_pred [n_shots], fail [n_shots] out (either may be NULL)
 * Errors: QD_EINVAL when n_shots exceeds the decoder's max_shots.
 */
qd_status qd_decode_shots_host(qd_decoder* dec, const uint32_t* det_bits, const uint32_t* obs_true,
                               int64_t n_shots, uint32_t* obs_pred, uint32_t* fail,
                               long long* n_fail, qd_stream_t stream);

/*
 * Decode window k and commit it without any device allocation, for callers
 * that cannot call cudaMalloc between decoder set-up and the end of the run:
 * a real-time decoding loop in which an allocation (or the device-wide
 * synchronisation cudaFree implies) would stall the stream, or a host
 * framework that owns all device memory and forbids the runtime allocator.
 * The paper has no counterpart; this is a packaging of qd_decode_windows
 * followed by qd_commit_and_slide, with the same results bit for bit.
 *
 * The window corrections and the work counter, which qd_decode_windows keeps
 * in caller or decoder buffers, live in one fixed array of
 * QD_STATIC_SCRATCH_BYTES compiled into the library (every GPU that loads it
 * holds that memory until the process exits).  Limit: n_shots * corr_words * 4
 * + 256 <= QD_STATIC_SCRATCH_BYTES (30839 shots for [[144,12,12]] with
 * (3,1) windows, 68 correction words per shot); larger batches return QD_EINVAL with the limit in the
 * message.
 *   det_bits     device [n_shots][det_words], updated in place as by
 *                qd_commit_and_slide
 *   obs_pred     device [n_shots], updated in place as by qd_commit_and_slide
 *   residue_fail device [n_shots], updated in place as by qd_commit_and_slide
 * The launch shape follows qd_decoder_set_launch exactly as qd_decode_windows
 * does (path mode for small batches in mode 0 or on request in mode 2, within
 * the same limits; global-memory path state in mode 3 or for windows too large
 * for shared memory), using the buffers the decoder allocated at creation;
 * the work counters add to the decoder's, read by qd_decoder_counters.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  All calls share the array and it
 * keeps the previous call's contents: two calls whose work can overlap on
 * the same GPU (for example calls on two different streams, or on two
 * decoders) race with each other; issue them on one stream per device.
 * Allocates nothing and makes no allocating library call.
 */
#define QD_STATIC_SCRATCH_BYTES (8u << 20)
qd_status qd_decode_commit_static(qd_decoder* dec, int k, uint32_t* det_bits, int64_t n_shots,
                                  uint32_t* obs_pred, uint32_t* residue_fail, qd_stream_t stream);

/*
 * Batched window steps (no counterpart in the paper, which decodes one code
 * and window size at a time): several decoders -- different codes, noise
 * levels or window sizes W -- advance together.  Window step j decodes window
 * j of every member that has one, in ONE persistent launch (shots of all
 * members share the CTAs through one work counter, heavier windows first),
 * then commits all of them in one launch (Eq. (10)-(11)).  Results are
 * identical to qd_decode_windows + qd_commit_and_slide per member.  The batch
 * borrows the members (which must outlive it) and their correction buffers:
 * members of a batch must not run other decodes concurrently.
 */
typedef struct qd_batch qd_batch;
qd_status qd_batch_create(qd_decoder* const* members, int n_members, qd_batch** out); /* 1..16 members */
qd_status qd_batch_destroy(qd_batch* b);
/* number of window steps: the largest member window count */
qd_status qd_batch_n_steps(const qd_batch* b, int* n_steps);
/*
 * One window step.  Host arrays of per-member DEVICE pointers / counts:
 *   det_bits[i]     [n_shots[i]][det_words_i], updated in place by the commit
 *   obs_pred[i]     [n_shots[i]], ^= L e_commit
 *   residue_fail[i] [n_shots[i]], |= the Eq. (11) residue flag
 * Members without window `step`, or with n_shots[i] = 0, are skipped.
 * Asynchronous on `stream`; capturable in a CUDA graph (it launches a memset
 * and two kernels).
 */
qd_status qd_batch_step(qd_batch* b, int step, uint32_t* const* det_bits, const int64_t* n_shots,
                        uint32_t* const* obs_pred, uint32_t* const* residue_fail, qd_stream_t stream);
/*
 * CTA shape of step `step`: `warps` warps per CTA (1..8) and a shared-memory
 * budget that leaves room for `ctas_per_sm` (1 or 2) CTAs per SM.  Every
 * member's layout takes as many decision-path slots (one per warp, at most
 * `warps`) as fit in the budget, so small windows run a path on every warp and
 * large ones on fewer.  Default: 8 warps, two CTAs per SM where every member
 * fits.  QD_EUNSUPPORTED when a member's window does not fit one slot.
 */
qd_status qd_batch_set_shape(qd_batch* b, int step, int warps, int ctas_per_sm);
/* out = {warps, dynamic shared bytes, CTAs per SM, members with this step} */
qd_status qd_batch_info(const qd_batch* b, int step, int out[4]);
/*
 * Autotuner: times the decode launch of step `step` on the given inputs for
 * every shape (4..8 warps x 1 or 2 CTAs per SM) that fits (one warm-up +
 * `reps` timed launches each, CUDA events
 * on `stream`, synchronous), keeps the fastest and returns its mean time in
 * *best_ms (may be NULL).  Writes only the members' correction buffers; the
 * inputs are not modified.  Not capturable.
 */
qd_status qd_batch_autotune(qd_batch* b, int step, uint32_t* const* det_bits, const int64_t* n_shots, int reps,
                            qd_stream_t stream, float* best_ms);

/*
 * Learned weighted min-sum for window k (no counterpart in the paper: the
 * fixed normalisation alpha of Eq. (1) becomes a per-edge, per-iteration
 * weight).  w: device [T][n_edges of window k], FP32, indexed by the window's
 * CSC edge order; iteration t (counted from message initialisation, in the
 * pre-BP and in every decision path) uses row min(t, T) - 1, and an edge of
 * the shortened matrix uses the weights of its full-window edge.  The caller
 * owns w and keeps it valid while the decoder uses it; NULL restores alpha.
 */
qd_status qd_decoder_set_weights(qd_decoder* dec, int k, const float* w, int T);

/*
 * Learned decimation ranker (no counterpart in the paper: it replaces the
 * argmin over the history sums L_i of Alg. 1, SELECT-VN, in every window and
 * decision path; aggressive decimation (Alg. 3), the guess rule of Alg. 2 and
 * f = [L_g <= 0] for the selected VN g stay as they are).
 *   params  HOST pointer to 641 FP32 values, copied: W1[64][8], b1[64],
 *           W2[64], b2 of score = W2 . relu(W1 x + b1) + b2; NULL removes it.
 * The library rounds W1 and W2 to multiples of 2^-6 clamped to [-2, 2] and b1
 * to multiples of 2^-7 within [-512, 512] (round half to even), keeps b2 as given, and selects
 * the candidate with the highest score (ties to the lowest short column).
 * Features of candidate i, in this order: L_i / 4, h_0..h_3 (the last four
 * posteriors, oldest first), each rounded to the 1/2 grid and clamped to
 * +-63.5; the number of unsatisfied neighbour checks (at most 127); the
 * static column degree; the window block of the column's first detector
 * (at most 255).  Installing or removing the ranker re-plans the shared-memory
 * layouts; not to be called while this decoder's launches are in flight.
 * Returns QD_EINVAL on a non-finite parameter, QD_EUNSUPPORTED when a window
 * no longer fits in shared memory.
 */
qd_status qd_decoder_set_ranker(qd_decoder* dec, const float* params);

/*
 * One ranker candidate record (training data; no counterpart in the paper).
 * x: the eight ranker features above, exactly as the ranker sees them;
 * shot: index within the decode call; wcol: window column; depth: the
 * selection depth D of Alg. 2; path: the decision path (0); flags bit 0 =
 * [L <= 0] (the value f Alg. 1 gives the candidate), bit 1 = the candidate the
 * active rule (Alg. 1 or the ranker) selected at this step.
 */
typedef struct {
  float x[8];
  int32_t shot, wcol;
  int16_t depth, path;
  int32_t flags;
} qd_rank_rec_t;

/*
 * Candidate dump: while set, every decode of this decoder appends, for
 * decision path 0 at each selection step, one record per candidate left after
 * Alg. 3.  records: device [capacity] qd_rank_rec_t; count: device int32 that
 * the caller zeroes, incremented once per candidate (records beyond capacity
 * are counted, not written); record order is unspecified.  records = NULL
 * turns the dump off.  Like the ranker it re-plans the shared-memory layouts.
 */
qd_status qd_decoder_set_dump(qd_decoder* dec, void* records, int* count, int capacity);

/*
 * Window-local samples for window k (training data): every column of the
 * window fires independently with its prior p_i (Philox4x32-10, counter
 * (column / 4, shot, 1 + k)), the same draws as qd_wms_sample.
 *   det_bits   device [n][det_words]: the window syndrome H_win e placed at
 *              the window's detector rows, zeros elsewhere (input of
 *              qd_decode_windows for window k)
 *   fault_bits device [n][corr_words] or NULL: e, by window column
 */
qd_status qd_window_sample(qd_decoder* dec, int k, uint64_t seed, uint64_t offset, int64_t n, uint32_t* det_bits,
                           uint32_t* fault_bits, qd_stream_t stream);

/*
 * Ranker forward / backward on n candidate records (device pointers):
 *   params     [641] FP32 W1[64][8], b1[64], W2[64], b2
 *   labels     [n] uint8 0/1 (required for grad and loss)
 *   quantize   1: the forward uses the grid-rounded parameters the decoder
 *              uses and the gradient passes straight through the rounding
 *   score      [n] or NULL: the logit z
 *   loss       [n] or NULL: w_y (softplus(z) - y z), w_1 = pos_weight, w_0 = 1
 *   grad       [641] or NULL: ACCUMULATES grad_scale * d(sum of losses)/d params
 *              (FP32 atomics: the last bits depend on the order of arrival)
 */
qd_status qd_ranker_eval(const float* params, const void* records, const uint8_t* labels, int64_t n, int quantize,
                         float pos_weight, float grad_scale, float* grad, float* loss, float* score,
                         qd_stream_t stream);

/*
 * Training the learned weighted min-sum of window k (no counterpart in the
 * paper).  A training sample is a window syndrome s = H_win e with every
 * window column firing independently with its prior (the syndrome a window
 * sees when every earlier window committed the truth).  The model is T
 * unrolled flooding iterations of weighted min-sum on the full window, from
 * v2c = Lambda, with w[t][e] in place of alpha in Eq. (1); the loss is the
 * soft-syndrome binary cross entropy at t = T: P(check j odd) =
 * (1 - prod_{i in N(j)} tanh(Lambda_i^(T) / 2)) / 2 against s_j, averaged over
 * the window's checks.  Gradients come from a hand-written adjoint of the
 * unrolled iterations, recomputed from message checkpoints every `ckpt`
 * iterations.
 *   qd_wms_create  allocates per-CTA scratch; T, ckpt as above
 *   qd_wms_info    out[6] = rows, columns, edges, T, ckpt, syndrome words
 *   qd_wms_sample  synd: device [n][syndrome words]; counter-based like
 *                  qd_sample_shots, with word 3 of the counter = 1 + k
 *   qd_wms_loss    loss: device [n] per-sample loss; post: device [n][cols]
 *                  posteriors at t = T, or NULL
 *   qd_wms_grad    grad_w: device [T][edges], ACCUMULATES grad_scale * dL/dw
 *                  summed over the n samples (L = per-sample loss); loss as
 *                  above or NULL
 *   qd_adam_step   in-place Adam update of n parameters (bias-corrected,
 *                  step >= 1); g, m1, m2 device arrays of n floats
 * All device pointers are caller-owned; calls are asynchronous on the stream.
 */
typedef struct qd_wms qd_wms;
qd_status qd_wms_create(const qd_decoder* dec, int k, int T, int ckpt, qd_wms** out);
qd_status qd_wms_destroy(qd_wms* m);
qd_status qd_wms_info(const qd_wms* m, int out[6]);
qd_status qd_wms_sample(qd_wms* m, uint64_t seed, uint64_t offset, int64_t n, uint32_t* synd, qd_stream_t stream);
qd_status qd_wms_loss(qd_wms* m, const float* w, const uint32_t* synd, int64_t n, float* loss, float* post,
                      qd_stream_t stream);
qd_status qd_wms_grad(qd_wms* m, const float* w, const uint32_t* synd, int64_t n, float grad_scale, float* grad_w,
                      float* loss, qd_stream_t stream);
qd_status qd_adam_step(float* w, const float* g, float* m1, float* m2, int64_t n, float lr, float beta1, float beta2,
                       float eps, int step, qd_stream_t stream);

/* Launch shape of qd_decode_windows (results are identical in every shape):
 * 0 automatic (default): path mode for batches that leave most SMs idle,
 * otherwise shot mode; 1 shot mode: persistent CTAs, one warp per decision
 * path; 2 path mode: one CTA per (shot, decision path) for the lowest
 * latency, the path CTAs of a shot launched as a thread-block cluster (up to
 * 8 CTAs, padded with idle CTAs to whole clusters) that splits the shot's
 * pre-BP, at most 64 shots per call (larger batches fall back to shot mode);
 * 3 shot mode with every CTA's pre-BP scratch and path states in global
 * memory (L2 / HBM) instead of shared memory -- the shape a window too large
 * for shared memory always uses (chosen at decoder creation, which allocates
 * those regions; mode 3 allocates them for every window here). */
qd_status qd_decoder_set_launch(qd_decoder* dec, int mode);

/* Launch plan of window k: out[0] shared bytes per CTA in shot mode,
 * out[1] its threads, out[2] its CTAs per SM, out[3] shared bytes per CTA in
 * path mode, out[4] its threads, out[5] SM count, out[6] CTAs per cluster in
 * path mode (they split each shot's pre-BP; 1: every path CTA runs it whole),
 * out[7] path-mode CTAs per shot (the paths rounded up to whole clusters). */
qd_status qd_decoder_launch_info(const qd_decoder* dec, int k, int out[8]);

/* Counters summed over every decode since the last reset: out[0] pre-BP
 * edge-iterations, out[1] GDG edge-iterations of every decision path run
 * from the root as Alg. 2 defines it (a path resumed from a shared prefix,
 * see qd_decoder_set_fork, counts the prefix as its own), out[2] windows
 * whose pre-BP converged, out[3] windows that ran GDG, out[4] bulk (TMA)
 * staging copies whose bounded wait ran out (then copied with plain loads;
 * expected 0).  Synchronous. */
qd_status qd_decoder_counters(qd_decoder* dec, long long out[5]);
/* The first n (1..8) counters: out[0..4] as qd_decoder_counters, out[5] GDG
 * edge-iterations the GPU executed (out[1] minus the shared prefixes it did
 * not recompute), out[6..7] 0.  Synchronous. */
qd_status qd_decoder_counters_ex(qd_decoder* dec, long long* out, int n);
qd_status qd_decoder_reset_counters(qd_decoder* dec, qd_stream_t stream);

/* Shot mode's decision-path scheduling (no counterpart in the paper, whose
 * threads snapshot the main branch's status only), for windows with more
 * paths than the CTA has warps.  mode 1: decision paths that made the same
 * decisions at depths 1..D-1 -- the same guess values, the same Alg. 3
 * thresholds and message restarts -- hold the same state after the BP of
 * step D, so the first path to get there leaves a snapshot (in a pool the
 * decoder allocated with its layouts) and paths queued later resume from it
 * instead of recomputing the prefix.  mode 2 (the default) adds preemption:
 * at every step boundary a warp whose path has fewer steps left than a
 * waiting path parks its path (a snapshot of the same kind) and takes the
 * other, longest remaining work first, so that no warp idles at the end of a
 * shot while paths wait.  mode 0: every path from the root, one after
 * another in a fixed order.  Results, traces and out[1] of the counters are
 * the same in every mode. */
qd_status qd_decoder_set_fork(qd_decoder* dec, int mode);

#ifdef __cplusplus
}
#endif
#endif /* QDEC_H */
