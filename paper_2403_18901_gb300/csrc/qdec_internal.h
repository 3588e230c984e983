// qdec_internal.h -- host-side data structures of libqdec (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qdec.h"

namespace qd {

void set_error(const std::string& msg);

// One window of the (W,F) schedule (Sec. III, Eq. (8)), host copy.
struct WindowHost {
  int k = 0, r0 = 0, n_blocks = 0, n_rows = 0, n_cols = 0, n_edges = 0, n_commit = 0, last = 0;
  int n_short = 0;        // columns GDG runs on
  int short_edges_max = 0;  // bound on the edges of the shortened matrix
  int row0 = 0;           // first detector id of the window
  int commit_b1 = 0;      // committed blocks are [r0, commit_b1)
  std::vector<int> gcols;                 // window column -> DEM column
  std::vector<uint16_t> col_ptr, col_rows;  // CSC over window rows (ascending)
  std::vector<uint16_t> row_ptr;            // CSR row pointers
  std::vector<uint32_t> row_ent;            // CSR entries: CSC edge id | (window column << 16)
  std::vector<float> llr;
};

struct DemHost {
  qd_bb_code code{};
  qd_noise noise{};
  int w = 0, R = 0, K = 0, n_det = 0, n_cols = 0;
  std::vector<int> col_ptr, col_dets;
  std::vector<uint32_t> col_obs;
  std::vector<double> col_p;
  std::vector<float> col_llr;
  std::vector<uint32_t> col_thr;  // sampling threshold round(p 2^32)
};

struct KParams;
struct WinDev;
struct Layout;
struct WmsGraph;
struct RankRec;
struct ForkDev;
struct ReuseDev;

// Build the merged DEM (backward sensitivity sweep over the circuit).
bool build_dem_host(const qd_bb_code& code, const qd_noise& noise, DemHost& out);
// Code-capacity models of the appendices (BSC on data qubits; [H_X | I]).
bool build_dem_code_capacity(const qd_bb_code& code, double p_data, double p_synd, DemHost& out);
int n_windows(const DemHost& d, int W, int F);
// merge: the H_1 merge of Sec. III (0 none, 1 equal restrictions, 2 identity)
bool build_window(const DemHost& d, int W, int F, int k, bool shorten, WindowHost& out, int merge = 0);

size_t trace_bytes_per_shot(int nb, int dmx, int ns_max);
cudaError_t set_decode_smem(size_t bytes);
// CTAs per SM of the decode kernel: mode 0 shot mode, 1 path mode, 3 shot
// mode with the union region in global memory.
cudaError_t decode_occupancy(int mode, int threads, size_t smem, int* blocks);
cudaError_t launch_decode(int mode, int grid, int threads, size_t smem, cudaStream_t st, const KParams& P,
                          const WinDev& W, const Layout& L, const uint32_t* det, int det_words, long long n,
                          uint32_t* corr, int corr_words, int32_t* status, char* trace, size_t tr_bytes, int dmx,
                          int ns_max, int* work, long long* counters, char* path_res, int* arrive, int sw_max,
                          char* uglob = nullptr, size_t ubytes = 0, int cps = 1, int cluster = 1,
                          const ForkDev* fork = nullptr, const ReuseDev* reuse = nullptr);
// Clusters of `cluster` path-mode CTAs that can be resident at once (0: none).
cudaError_t path_cluster_occupancy(int threads, size_t smem, int cluster, int* clusters);
// One decoder's share of a batched window step (decode + commit).
struct BatchMember {
  const KParams* P;
  const WinDev* W;
  const Layout* L;
  const uint32_t* det;  // also updated by the commit
  int det_words;
  long long n;
  uint32_t* corr;
  int corr_words, dmx, ns_max, sw_max;
  long long* counters;
  int n_commit;
  const int *cptr, *cdet;
  const uint32_t* cobs;
  uint32_t *obs_pred, *resid;
  int b0, b1;
  const ForkDev* fork;  // the member's path-scheduling plan (nullptr: none)
};
cudaError_t batch_occupancy(int threads, size_t smem, int* blocks);
cudaError_t launch_decode_batch(cudaStream_t st, int grid, int threads, size_t smem, unsigned q_off, int* work,
                                const BatchMember* m, int n);
cudaError_t launch_commit_batch(cudaStream_t st, const BatchMember* m, int n);
cudaError_t launch_sample(cudaStream_t st, int n_cols, const uint32_t* thr, const int* cptr,
                          const int* cdet, const uint32_t* cobs, int det_words,
                          unsigned long long seed, unsigned long long off, long long n, uint32_t* det,
                          uint32_t* obs);
cudaError_t launch_commit(cudaStream_t st, int n_commit, const int* cptr, const int* cdet,
                          const uint32_t* cobs, int corr_words, const uint32_t* corr, long long n,
                          uint32_t* det, int det_words, uint32_t* obs_pred, uint32_t* resid, int b0,
                          int b1);
cudaError_t launch_evaluate(cudaStream_t st, const uint32_t* pred, const uint32_t* obs,
                            const uint32_t* resid, long long n, uint32_t* fail, long long* n_fail);

size_t wms_smem_bytes(int ne, int nc, int rw);
size_t wms_scratch_per_cta(int ne, int T, int ckpt);
cudaError_t wms_set_smem(size_t bytes);
cudaError_t wms_occupancy(size_t smem, int* blocks);
cudaError_t launch_wms(cudaStream_t st, int grid, size_t smem, const WmsGraph& G, const float* w, const uint32_t* synd,
                       long long n, int backward, float grad_scale, float* grad_w, float* loss, float* post,
                       float* scratch, size_t scratch_per_cta, int* work);
cudaError_t launch_wms_sample(cudaStream_t st, const WmsGraph& G, const uint32_t* thr, unsigned long long seed,
                              unsigned long long off, long long n, unsigned domain, uint32_t* synd, uint32_t* det,
                              int det_words, int row0, uint32_t* fault, int cw);
cudaError_t launch_ranker(cudaStream_t st, const float* params, const RankRec* recs, const uint8_t* labels,
                          long long n, int quantize, float pos_weight, float scale, float* grad, float* loss,
                          float* score);
cudaError_t launch_adam(cudaStream_t st, float* w, const float* g, float* m, float* v, long long n, float lr,
                        float b1, float b2, float eps, int step);

}  // namespace qd
