// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "zoom.h"

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------

enum CounterSlot {
  CNT_BUCKET_SUM = 0,   // sum over queries of sum_l |bin_l(q)|
  CNT_BUCKET_MAX = 1,   // max over queries of the same
  CNT_EMPTY = 2,        // queries with no candidate
  CNT_PADDED = 3,       // queries with fewer than K candidates
  CNT_FP64 = 4,         // LLE solves in FP64
  CNT_EXACT = 5,        // exact-match (one-hot) queries
  CNT_FALLBACK = 6,     // statistics: queries the first tensor filter's rerank did not settle
  CNT_FALLBACK2 = 7,    // statistics: queries the second (FP16-split) filter left to the SIMT scan
  CNT_N = 8
};

constexpr int kStageEvents = 10;

struct zoom_ctx_s {
  int device = 0;
  int n_sm = 0;
  zoom_allocator alloc{};
  bool has_alloc = false;
  unsigned int* d_status = nullptr;       // device status word (0 = ok)
  unsigned long long* d_counters = nullptr;  // [CNT_N]
  int64_t last_n_queries = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  bool stage_timing = false;
  // boundaries of the 7 stages (0..7) and of the tensor-core filter kernel (8, 9)
  cudaEvent_t stage_ev[kStageEvents] = {};
  bool stage_rec[kStageEvents] = {};
  void* batch = nullptr;          // recorded batch (graph, workspace, events): zoom_api.cu
  void* tuned = nullptr;          // autotuned search choices: zoom_api.cu
  uint64_t wait_ns = 0;           // bound on the tensor-core filter's waits (0: 2 s)
  int inject = 0;                 // testing aid: zoom_set_fault_injection
};

// Records the boundary event of stage `i` when stage timing is on.
void zoom_stage_mark(zoom_ctx ctx, int i, cudaStream_t st);
// Frees the context's recorded batch and autotuning choices.
void zoom_release_batch(zoom_ctx ctx);

struct zoom_dict_s {
  zoom_ctx ctx = nullptr;
  int64_t n = 0;
  int P = 0, s = 0, d = 0, dpad = 0, PH = 0, ph2 = 0, ph2pad = 0;
  int feature = 0;           // 0: pixels - mu (d = P^2); 1 / 2: first / second-order gradients (d = 2 P^2)
  double blur_sigma = 0.0;
  float* lr_pix = nullptr;   // [N][P^2]
  float* feat = nullptr;     // [N][dpad]  feature, zero padded
  float* mu = nullptr;       // [N]
  float* norm2 = nullptr;    // [N]  ||feat||^2
  float* hr_res = nullptr;   // [N][ph2pad] HR patch - mu
  size_t bytes = 0;
  int index_refs = 0;
};

struct zoom_index_s {
  zoom_dict dict = nullptr;
  int L = 0, k = 0, t = 1, cap = 0;
  float w = 0.f;
  int proj_dist = 0;         // the draws' law and seed when the library drew them
  uint64_t seed = 0;
  float* alpha = nullptr;    // [L*k][d]
  float* beta = nullptr;     // [L*k]
  uint64_t* dkeys = nullptr; // [N][L]
  uint64_t* ukeys = nullptr; // [L][N]  bin keys, ascending (first nuniq[l] valid)
  int32_t* offs = nullptr;   // [L][N+1] CSR offsets into ids
  int32_t* ids = nullptr;    // [L][N]   entry IDs grouped by bin, ascending within a bin
  int32_t* nuniq = nullptr;  // [L]
  // tensor-core operands of the dictionary: 128-row tiles [tile][kc][128][8]
  uint16_t* dop16 = nullptr; // FP16 3-term split, tc_kc(d, 0) chunks of 8 per row
  uint16_t* dopbf = nullptr; // BF16 single term, tc_kc(d, 1) chunks of 8 per row
  uint16_t* dopf1 = nullptr; // FP16 single term, tc_kc(d, 2) chunks of 8 per row
  int64_t nd_rows = 0;       // rows of the operands (N rounded up to 128)
  size_t bytes = 0;
};

// ---------------------------------------------------------------------------
// host helpers (zoom_api.cu)
// ---------------------------------------------------------------------------

void zoom_set_error(const std::string& msg);

// seeded draws (zoom_random.cu): the projections of Eq. 10 (dist 0
// Gaussian, 1 Cauchy by Eq. 11) and the dictionary positions
constexpr double kCauchyEps = 1e-3;
void zoom_draw_projections(int L, int k, int D, float w, int dist, uint64_t seed, float* alpha, float* beta);
int64_t zoom_count_origins(int n_images, const int32_t* lr_h, const int32_t* lr_w, int P);
bool zoom_sample_positions_host(uint64_t seed, int n_images, const int32_t* lr_h, const int32_t* lr_w, int P,
                                int64_t n_pairs, int32_t* positions);
// A dictionary handle of n pairs with its (uninitialised) device arrays in
// one allocation based at lr_pix; nullptr when the allocation fails.
zoom_dict zoom_dict_alloc(zoom_ctx ctx, int64_t n, int P, int s, double blur_sigma, int feature,
                          cudaStream_t st);
void* zoom_alloc(zoom_ctx ctx, size_t bytes, cudaStream_t st);
void zoom_free(zoom_ctx ctx, void* p, size_t bytes, cudaStream_t st);

// ---------------------------------------------------------------------------
// kernel launchers (each returns cudaGetLastError() of its launches)
// ---------------------------------------------------------------------------

// dictionary / index build (kernels_build.cu)
cudaError_t launch_degrade_exact(const float* hr, int H, int W, int s, double sigma, float* lr,
                                 cudaStream_t st);
cudaError_t launch_dict_gather(const float* const* d_lr_images, const int32_t* d_lr_h,
                               const int32_t* d_lr_w, const float* const* d_hr_images,
                               const int32_t* d_hr_w, const int32_t* d_pos, int64_t n, int P, int s,
                               zoom_dict d, cudaStream_t st);
cudaError_t launch_hash(const float* feat, int dpad, int d, int64_t n, const float* alpha,
                        const float* beta, int L, int k, float w, uint64_t* keys, cudaStream_t st);
cudaError_t build_csr_tables(zoom_index ix, void* scratch, size_t scratch_bytes, cudaStream_t st);
size_t csr_scratch_bytes(int64_t n);
// scratch of build_csr_tables: the radix sort's plus the key compaction's
size_t csr_build_scratch_bytes(int64_t n, int L);

// per-query steps (kernels_query.cu)
// F: feature mode (0 pixels minus mean, 1 / 2 first / second-order gradients)
cudaError_t launch_query_features(const float* lr, int h, int w, int P, int F, int dpad, float* feat,
                                  float* mu, float* norm2, cudaStream_t st);
cudaError_t launch_bucket_lookup(zoom_index ix, const uint64_t* qkeys, int64_t nq,
                                 int32_t* bucket_sum, unsigned long long* counters,
                                 cudaStream_t st);
cudaError_t launch_knn_exact(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq,
                             int K, int32_t* nbr, float* dist, unsigned long long* counters,
                             const int32_t* qidx, const unsigned long long* qcount,
                             cudaStream_t st);
// capped candidate walk (index cap > 0): cand = scratch [nq][cap]; queries
// with fewer than K candidates are appended to fb (count *fb_count)
cudaError_t launch_knn_capped(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq, int K,
                              int32_t* nbr, float* dist, int32_t* cand, int32_t* fb,
                              unsigned long long* fb_count, cudaStream_t st);
cudaError_t launch_lle(zoom_dict d, const float* qfeat, int64_t nq, const int32_t* nbr,
                       const float* dist, int K, float reg_rel, double cond_thr, float* wgt,
                       unsigned long long* counters, cudaStream_t st);
// the same three steps for the gradient features, D = 18 or 50 (kernels_query_grad.cu)
cudaError_t launch_knn_exact_grad(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq,
                                  int K, int32_t* nbr, float* dist, unsigned long long* counters,
                                  const int32_t* qidx, const unsigned long long* qcount, cudaStream_t st);
cudaError_t launch_knn_capped_grad(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq,
                                   int K, int32_t* nbr, float* dist, int32_t* cand, int32_t* fb,
                                   unsigned long long* fb_count, cudaStream_t st);
cudaError_t launch_lle_grad(zoom_dict d, const float* qfeat, int64_t nq, const int32_t* nbr,
                            const float* dist, int K, float reg_rel, double cond_thr, float* wgt,
                            unsigned long long* counters, cudaStream_t st);

// tensor-core neighbour search (kernels_tc.cu)
int64_t tc_rows_padded(int64_t n, bool even_tiles);
// n_dev: rows at or past min(*n_dev, n) are padding (a count on the device)
cudaError_t launch_operand(const float* feat, int dpad, int d, int64_t n, int64_t n_rows, int role,
                           int precision, uint16_t* op, float* norm_out, cudaStream_t st,
                           const unsigned long long* n_dev = nullptr);
// operand width in 8-element chunks for feature dimension d: FP16 split
// (precision 0) 10 (K = 80, d <= 25) or 20 (K = 160, d = 50); BF16
// (precision 1) and single-term FP16 (precision 2) 4 or 8
int tc_kc(int d, int precision);
size_t tc_smem_bytes(int KC, int MC);
int tc_list_size(int precision, int K, int rerank_mult);
// tail_split > 0: whole query pairs round robin for the full rounds over the
// grid, the remaining pairs cut into tail_split dictionary parts (nsplit must
// equal tail_split); 0: nsplit round-robin splits of every pair
// The single-term FP16 and BF16 filters (precision 2 and 1, kc 4 or 8) run
// as the wide-step kernel: 256-row dictionary steps, whose operand is laid
// out in 256-row tiles ([tile][kc][256][8]); the dictionary operand needs
// whole 256-row steps (an even number of 128-row tiles).
bool tc_wide_form(int precision, int kc);
// wait_ns: bound on every device wait (0: 2 s); inject: testing aid (1: the
// epilogue withholds its accumulator releases, so a wait runs out)
cudaError_t launch_knn_tc(const uint16_t* qop, const float* qn, int64_t nq, const uint16_t* dop,
                          int64_t nd, int precision, int kc, int MC, int nsplit, int tail_split, int grid,
                          float* out_d, int32_t* out_id, unsigned int* status, cudaStream_t st,
                          const unsigned long long* nq_dev = nullptr, uint64_t wait_ns = 0, int inject = 0);
// ld/li: per split and query the MC best 32-entry chunks (filter minimum d~,
// chunk index), ascending; form 1 for the FP16-split filter, 2 for the
// single-term FP16 filter (both: proof and fallback flags), 0 for the BF16
// filter.  Queries it cannot settle are appended to fb (count *fb_count,
// zeroed by the caller); with qmap, query q of this launch is query qmap[q]
// of the call (outputs and fb use the latter) and only q < *nq_dev run.
cudaError_t launch_rerank(int d, int MC, int K, const float* qfeat, int dpad, const float* qn,
                          const uint64_t* qkeys, int64_t nq, const float* dfeat, const uint64_t* dkeys,
                          int64_t nd, int L, int tmin, const float* ld, const int32_t* li, int nsplit,
                          int form, int32_t* nbr, float* dist, int32_t* fb, unsigned long long* fb_count,
                          cudaStream_t st, const int32_t* qmap = nullptr,
                          const unsigned long long* nq_dev = nullptr);
// The queries idx[0 .. *count) (count <= max_count), compacted: features and
// keys of the first cap into cfeat / ckeys, the rest appended to `over`.
cudaError_t launch_gather_queries(const int32_t* idx, const unsigned long long* count, int64_t max_count,
                                  int64_t cap, const float* feat, int dpad, const uint64_t* keys, int L,
                                  float* cfeat, uint64_t* ckeys, int32_t* over, unsigned long long* over_count,
                                  cudaStream_t st);

// backward / adjoint steps (kernels_backward.cu) and the key sort (kernels_build.cu)
cudaError_t sort_keys_csr(const int32_t* keys32, int64_t n, int32_t* sorted_pos, uint64_t* ukeys,
                          int32_t* offs, int32_t* nuniq, void* scratch, size_t scratch_bytes,
                          cudaStream_t st);
cudaError_t launch_patches(const int32_t* nbr, const float* wgt, const float* mu, const float* hr_res,
                           int ph2pad, int K, int64_t nq, int ph2, float* P, cudaStream_t st);
cudaError_t launch_degrade(const float* x, int H, int W, int s, double sigma, const float* sub, float* y,
                           cudaStream_t st);
cudaError_t launch_degrade_adjoint(const float* r, int h, int w, int H, int W, int s, double sigma,
                                   float alpha, float* g, cudaStream_t st);
cudaError_t launch_patch_grad(const float* gx, const float* P, int h, int w, int s, int Pp, float lambda,
                              float* gP, cudaStream_t st);
cudaError_t launch_dict_grad(const int32_t* sorted_use, const int32_t* offs, const uint64_t* ukeys,
                             const int32_t* nuniq, int64_t max_segments, const float* wgt, const float* gP,
                             int K, int ph2, int ph2pad_out, float* grad, cudaStream_t st);
cudaError_t launch_mu_grad(const float* gP, int64_t nq, int ph2, float* gmu, cudaStream_t st);
cudaError_t launch_energy_partials(const float* r, int64_t n_r, const float* P, int h, int w, int s, int Pp,
                                   double* part, int nblocks, cudaStream_t st);
cudaError_t launch_nbr_dist(const float* qfeat, int dpad, int d, int64_t nq, const float* dfeat,
                            const int32_t* nbr, int K, float* dist, cudaStream_t st);

// image steps (kernels_image.cu)
cudaError_t launch_overlap_add(const int32_t* nbr, const float* wgt, const float* mu,
                               const float* hr_res, int ph2pad, int K, int h, int w, int s, int P,
                               float* hr, cudaStream_t st);
// the same average through nq * (s P)^2 floats of scratch (two passes, the
// same bits; falls back to the one-pass form where the scratch is NULL)
cudaError_t launch_overlap_add_staged(const int32_t* nbr, const float* wgt, const float* mu,
                                      const float* hr_res, int ph2pad, int K, int h, int w, int s, int P,
                                      float* patches, float* hr, cudaStream_t st);
cudaError_t launch_bp_iteration(const float* x, float* x_out, const float* lr, float* err, int h,
                                int w, int s, double blur_sigma, float sigma_sp, float sigma_r,
                                int radius, cudaStream_t st);
