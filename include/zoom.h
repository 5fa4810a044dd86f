/*
 * zoom.h - C ABI of the GB300 (sm_103a) patch-hashing zoom library.
 *
 * Method: M. Das Gupta, "Hashing Image Patches for Zooming".  An LR image is
 * zoomed by hashing every overlapping LR patch feature into L p-stable LSH
 * tables (Sec. 4.1, Eq. 10), selecting the K nearest training patches among
 * the hashed candidates (Sec. 4.2), solving the sum-to-one least-squares
 * weights (Eq. 12-13), blending the paired HR patches (Eq. 14), averaging
 * the overlaps, and refining with error back-projection through an
 * approximate cross-bilateral filter (Sec. 4, Eq. 6-7; Sec. 4.3, Eq. 15-17).
 *
 * Conventions (every function):
 *  - Returns a zoom_status; ZOOM_OK = 0.  Out-parameters are written only on
 *    ZOOM_OK.  Nothing throws.  zoom_last_error() gives a one-line detail of
 *    the last failure on the calling thread.
 *  - "device" pointers are CUDA device memory of the context's device,
 *    "host" pointers are CPU memory.  The caller owns every buffer it passes;
 *    the library never frees or retains them past the call, except that an
 *    asynchronous call reads and writes them on `stream` after returning.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls do not synchronise unless stated.
 *  - Images are row-major float32, values on the [0, 1] scale.
 *  - Handles own their device arrays, allocated through the context's
 *    allocator.  An index refers to its dictionary: destroy the index first.
 *  - A context is not thread-safe; use one per thread or serialise calls.
 */
#ifndef ZOOM_H
#define ZOOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ZOOM_OK = 0,
  ZOOM_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range   */
  ZOOM_ERR_OOM = 2,         /* the allocator returned NULL                     */
  ZOOM_ERR_CUDA = 3,        /* a CUDA runtime call failed                      */
  ZOOM_ERR_TIMEOUT = 4,     /* a device-side bounded wait gave up              */
  ZOOM_ERR_UNSUPPORTED = 5, /* valid request outside what this build supports  */
  ZOOM_ERR_STATE = 6,       /* handle used in the wrong state                  */
  ZOOM_ERR_IO = 7,          /* file could not be read or written               */
  ZOOM_ERR_DEVICE = 8       /* a kernel reported a failed check (status word)  */
} zoom_status;

typedef struct zoom_ctx_s* zoom_ctx;
typedef struct zoom_dict_s* zoom_dict;
typedef struct zoom_index_s* zoom_index;

/* Device-memory allocator.  alloc returns device memory of at least `bytes`
 * usable on `stream` (NULL on failure); free releases it (stream-ordered).
 * A NULL allocator selects cudaMallocAsync / cudaFreeAsync. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} zoom_allocator;

/* Degradation and patch geometry (Sec. 2.1): HR -> Gaussian blur (3 taps,
 * sigma blur_sigma, clamped borders) -> s x s box down-sampling.  LR patches
 * are lr_patch x lr_patch; HR patches are (scale*lr_patch)^2.  blur_sigma is
 * a double so that the taps are computed from the exact parameter value.
 * feature selects the feature an LR patch is hashed and matched by (Sec.
 * 4.1, "Feature representation"): 0 = the P*P pixels minus their mean;
 * 1 = the first-order gradients of the LR image at the patch's pixels,
 * g_x(r,c) = x(r,c+1) - x(r,c-1) then g_y(r,c) = x(r+1,c) - x(r-1,c), each
 * row-major over the patch, image coordinates clamped to the image (2*P*P
 * values); 2 = the second-order gradients in the same layout, g_xx(r,c) =
 * 2x(r,c) - x(r,c-2) - x(r,c+2) then g_yy.  Either way the HR patch is
 * stored and blended relative to the LR patch mean.  Supported: scale 1..4,
 * blur_sigma > 0, feature 0, 1 or 2;
 * dictionaries and queries need lr_patch 3 or 5 (UNSUPPORTED otherwise); the
 * image-only calls (zoom_backproject, zoom_degrade, their adjoints) ignore
 * lr_patch and feature. */
typedef struct {
  int32_t scale;
  int32_t lr_patch;
  double blur_sigma;
  int32_t feature;
} zoom_degradation;

/* LSH parameters (Sec. 3.2, Sec. 4.1).  L tables of k concatenated hashes
 * h = floor((alpha.v + beta) / w).  min_table_hits = t (an ID is a candidate
 * if it shares the query's bin in >= t tables; 1 = plain union).
 * proj_dist and seed: how zoom_build_index draws alpha and beta when the
 * caller passes none (zoom_lsh_draws): proj_dist 0 = Gaussian vectors, 1 =
 * Cauchy vectors by the rule of Eq. 11 (a / b, a and b standard normal,
 * |b| >= 1e-3), from the 64-bit seed.
 * max_candidates: 0 = no cap; > 0 = the early stop of Sec. 4.2 (tables in
 * order, IDs ascending within a bin, stop at exactly max_candidates distinct
 * IDs; t is then not used).  With a cap the K nearest are searched among
 * those IDs in FP32 (both precisions; a query whose bins hold fewer than K
 * IDs is padded with the nearest entries outside them), the inference calls
 * need K <= max_candidates and take nq * max_candidates * 4 bytes of scratch.
 * Supported: 1 <= L <= 32, 1 <= k <= 32, w > 0, 1 <= t <= L,
 * 0 <= max_candidates <= 4096. */
typedef struct {
  int32_t L;
  int32_t k;
  float w;
  int32_t min_table_hits;
  int32_t max_candidates;
  int32_t proj_dist;
  uint64_t seed;
} zoom_lsh_params;

/* Inference parameters.  K nearest neighbours (1..16); reg_rel: the LLE
 * regulariser eps = reg_rel * trace(G) (Eq. 12-13); bp_iters back-projection
 * iterations (0..64) with spatial sigma sigma_spatial (pixels), range sigma
 * sigma_range and window radius bp_radius (1..7) (Sec. 4.3).
 * precision: 0 = exact FP32 neighbour search; 1 = BF16 tensor-core distance
 * filter keeping per query the best 16 (rerank_mult*K <= 16) or 32 chunks of
 * 32 consecutive dictionary entries by their smallest BF16 distance, then the
 * FP32 exact rerank of those chunks' entries.
 * fp64_cond_threshold: the LLE solve runs in FP64 for a query whose
 * condition bound (trace(G) + eps) / eps exceeds it.
 * search (precision 0 only): 0 = automatic (tensor cores from 4096
 * dictionary entries), 1 = SIMT scan of the dictionary in FP32 difference
 * form, 2 = tensor-core search with a proven exact FP32 rerank: a filter with
 * one FP16 term per feature value (K = 32), then, for the queries its error
 * bound cannot settle, the FP16 hi/lo-split filter (K = 80) on just those
 * queries, then the SIMT scan for any left; 3 = the split filter alone (then
 * the SIMT scan).  All four give the same neighbours bit for bit.  Precision 1
 * always uses the tensor cores; it needs rerank_mult * K <= 32. */
typedef struct {
  int32_t K;
  float reg_rel;
  int32_t bp_iters;
  float sigma_spatial;
  float sigma_range;
  int32_t bp_radius;
  int32_t precision;
  int32_t rerank_mult;
  double fp64_cond_threshold;
  int32_t search;
} zoom_upscale_params;

/* Counters of the last zoom_query / zoom_upscale on a context (read after
 * the stream has been synchronised; zoom_get_stats synchronises). */
typedef struct {
  int64_t n_queries;
  double mean_bucket_sum;   /* mean over queries of sum_l |bin_l(q)| (with repeats) */
  int64_t max_bucket_sum;
  int64_t n_empty;          /* queries whose candidate set was empty          */
  int64_t n_padded_queries; /* queries with fewer than K candidates (padded)  */
  int64_t n_fp64_solves;    /* LLE solves that ran in FP64                    */
  int64_t n_exact_match;    /* queries equal to a dictionary entry (one-hot)  */
  int64_t n_filter_fallback;/* queries the first tensor filter's rerank could
                              * not settle (searched again: the split filter
                              * after the single-term one, else the SIMT scan) */
  double ms_total;          /* device time of the last call (CUDA events)     */
  /* per-stage device milliseconds of the last call, when stage timing is on:
   * [0] features, [1] hashing, [2] bin lookup, [3] neighbour search,
   * [4] LLE solve, [5] blend + overlap average, [6] back-projection,
   * [7] the tensor-core filter kernel alone (within [3]; 0 on the SIMT scan) */
  double ms_stage[8];
} zoom_stats;

/* ---- context ----------------------------------------------------------- */

/* Creates a context on CUDA device `device`; `alloc` may be NULL. */
zoom_status zoom_ctx_create(int device, const zoom_allocator* alloc, zoom_ctx* out);
void zoom_ctx_destroy(zoom_ctx ctx);
const char* zoom_status_string(zoom_status s);
/* Thread-local text of the last error (never NULL). */
const char* zoom_last_error(void);

/* ---- dictionary (Sec. 2.1; Sec. 5.1) ------------------------------------
 * Builds N = n_pairs LR/HR training patch pairs.  hr_images: host array of
 * n_images device pointers, image m of heights[m] x widths[m] (host arrays)
 * float32 values.  Each image is degraded (blur + down-sampling; the LR
 * image is rounded once to float32); pair n uses positions[n] = (image m,
 * LR row i, LR col j) (host int32 [n_pairs][3]): LR patch at (i, j) and HR
 * patch at (s*i, s*j).  Pair n gets ID n; positions should be sorted by
 * (m, i, j) so that IDs follow the paper's row order.  positions == NULL:
 * the library draws them from `seed` (zoom_sample_positions: uniform without
 * replacement over every LR patch origin of the images, in origin order);
 * otherwise seed is not used.  Stored per pair:
 * the LR pixels, the LR mean mu, the feature (degr->feature; gradients are
 * taken on the whole LR training image) and the HR patch minus mu.  Errors:
 * INVALID_ARG for sizes out of range or positions whose patch leaves its
 * image (checked on the host). */
zoom_status zoom_build_dictionary(zoom_ctx ctx, const float* const* hr_images,
                                  const int32_t* heights, const int32_t* widths,
                                  int32_t n_images, const zoom_degradation* degr,
                                  int64_t n_pairs, const int32_t* positions, uint64_t seed,
                                  void* stream, zoom_dict* out);
void zoom_dict_destroy(zoom_dict d);
/* Copies stored arrays to the host (synchronises `stream`): lr_pix [N][P*P],
 * mu [N], hr_res [N][(s*P)^2]; any pointer may be NULL. */
zoom_status zoom_dict_export(zoom_dict d, float* lr_pix, float* mu, float* hr_res, void* stream);
/* Dictionary sizes: N, LR patch side P, scale s, the blur sigma of its
 * degradation, its feature mode and feature dimension D (P*P or 2*P*P); any
 * pointer may be NULL. */
zoom_status zoom_dict_info(zoom_dict d, int64_t* n, int32_t* patch, int32_t* scale, double* blur_sigma,
                           int32_t* feature, int32_t* feature_dim);

/* ---- training-crop sampling (Sec. 5.1) -----------------------------------
 * Draws training crops from HR images where they have structure: for image
 * m (device pointer images[m], heights[m] x widths[m] float32, row-major),
 * every pixel carries the mass sqrt(g_x^2 + g_y^2) of its first-order
 * gradients (clamped central differences, as feature 1, in FP64); pixels in
 * row-major order form a CDF, and draw j of the image (u[m][j], host double
 * [n_images][draws_per_image], each in [0, 1); the random numbers are inputs)
 * selects the first pixel whose cumulative mass exceeds u * total (a flat
 * image: pixel floor(u * h * w)).  The crop_h x crop_w window centred there
 * (top = row - crop_h / 2, left = col - crop_w / 2, shifted inside the image)
 * goes to windows (host int32 [n_images][draws_per_image][4]: row, col, top,
 * left) and, if crops != NULL, its pixels to crops (device float32
 * [n_images * draws_per_image][crop_h][crop_w], caller-owned).  The CDF is a
 * fixed-order FP64 sum (tiles of 1024 pixels), equal to a sequential sum up
 * to FP64 rounding, so only a draw within rounding of a CDF step can select
 * the neighbouring pixel.  Synchronises `stream`.  Errors: INVALID_ARG for
 * NULL pointers, a crop larger than an image, a draw outside [0, 1), more
 * than 2^26 draws; OOM for the scratch. */
zoom_status zoom_sample_crops(zoom_ctx ctx, const float* const* images, const int32_t* heights,
                              const int32_t* widths, int32_t n_images, const double* u,
                              int32_t draws_per_image, int32_t crop_h, int32_t crop_w,
                              int32_t* windows, float* crops, void* stream);

/* ---- seeded random draws (host, no device work) ---------------------------
 * Both come from the counter-based generator Philox4x32-10 (Salmon et al.,
 * SC 2011) keyed by the 64-bit seed; a draw is a function of (seed, its
 * counter) alone.
 * zoom_lsh_draws: the draws of Eq. 10 for feature dimension dim: alpha
 * (host float32 [L*k][dim]) element n is the Box-Muller normal (FP64, cosine
 * branch, uniforms (x + 1/2) / 2^32) of counter (n, 0, 0, 0); with
 * lsh->proj_dist 1 it is divided by the normal of counter (n, t, 1, 0) for
 * the first t = 0, 1, ... with |b| >= 1e-3 (Eq. 11).  beta (host float32
 * [L*k]): u * w, u the uniform of the first word of counter (j, 0, 0, 1),
 * kept below w.  Errors: INVALID_ARG (NULL, L or k outside 1..32, dim
 * outside 1..64, w <= 0, another proj_dist). */
zoom_status zoom_lsh_draws(const zoom_lsh_params* lsh, int32_t dim, float* alpha, float* beta);
/* zoom_sample_positions: n_pairs dictionary positions (host int32
 * [n_pairs][3] = (image, LR row, LR col)) drawn uniformly without
 * replacement over every lr_patch x lr_patch origin of n_images LR images of
 * lr_heights[m] x lr_widths[m] (origins numbered image by image, row by
 * row): origin o draws the 64-bit key (first word high) of counter
 * (o, 0, 0, 2), the n_pairs smallest (key, o) are kept, in origin order (the
 * paper's row-order IDs, Sec. 2.1).  For HR training images the LR sizes
 * are the HR sizes divided by the scale.  Errors: INVALID_ARG (NULL, an
 * image smaller than a patch, n_pairs outside 1..number of origins). */
zoom_status zoom_sample_positions(uint64_t seed, int32_t n_images, const int32_t* lr_heights,
                                  const int32_t* lr_widths, int32_t lr_patch, int64_t n_pairs,
                                  int32_t* positions);

/* ---- LSH index (Sec. 3.2; Sec. 4.1, Eq. 10) -----------------------------
 * Hashes every dictionary feature into L tables.  alpha: host float32
 * [L*k][D] projection vectors (D the feature dimension); beta: host float32
 * [L*k] offsets in [0, w).  Both NULL: the library draws them from
 * lsh->seed and lsh->proj_dist (zoom_lsh_draws).  Builds, per table, the
 * bucket key of every entry and a CSR of its bins (keys radix-sorted on the
 * device).  Errors: INVALID_ARG for parameters out of range or only one of
 * alpha and beta given. */
zoom_status zoom_build_index(zoom_dict d, const zoom_lsh_params* lsh, const float* alpha,
                             const float* beta, void* stream, zoom_index* out);
void zoom_index_destroy(zoom_index ix);
/* Copies the bucket key of every entry to host uint64 [N][L] and, if
 * n_bins != NULL, the number of bins per table to host int32 [L]
 * (synchronises `stream`). */
zoom_status zoom_index_export(zoom_index ix, uint64_t* keys, int32_t* n_bins, void* stream);
/* The index's LSH parameters (any pointer may be NULL); proj_dist and seed
 * are those of the library's draws, 0 when the caller gave alpha and beta. */
zoom_status zoom_index_info(zoom_index ix, zoom_lsh_params* lsh);

/* ---- files: checkpoint / resume ------------------------------------------
 * The paper keeps the N training pairs on disk once extracted (Sec. 2.1).
 * zoom_dict_save writes every array the dictionary stores (LR pixels, the
 * features, mu, squared feature norms and the HR residuals, float32) after a
 * little-endian header ("ZOOMDICT", version 1, the feature mode, N, P, s,
 * blur_sigma and the row strides); zoom_dict_load reads such a file into a
 * new dictionary on ctx, bit-identical to the saved one.  zoom_index_save
 * writes the LSH parameters and the projections ("ZOOMINDX", version 1, N,
 * D, L, k, min_table_hits, max_candidates, w; then alpha [L*k][D], beta [L*k]);
 * zoom_index_load rebuilds the index on dictionary d from them (the same
 * keys and bins as the saved index).  All four synchronise `stream`; the
 * caller owns `path` (a NUL-terminated file name).  Errors: IO (cannot
 * open, write failure, truncated file), INVALID_ARG (not such a file,
 * another version, sizes out of range, an index file of another
 * dictionary), OOM, CUDA. */
zoom_status zoom_dict_save(zoom_dict d, const char* path, void* stream);
zoom_status zoom_dict_load(zoom_ctx ctx, const char* path, void* stream, zoom_dict* out);
zoom_status zoom_index_save(zoom_index ix, const char* path, void* stream);
zoom_status zoom_index_load(zoom_dict d, const char* path, void* stream, zoom_index* out);
/* Copies the index's random draws to the host (synchronises `stream`):
 * alpha float32 [L*k][D], beta float32 [L*k] (Eq. 10); either may be NULL. */
zoom_status zoom_export_params(zoom_index ix, float* alpha, float* beta, void* stream);

/* ---- inference ------------------------------------------------------------
 * zoom_upscale: the whole per-patch inference and back-projection of an LR
 * image lr (device, h x w) into hr (device, caller-allocated (s*h) x (s*w)).
 * Requires h, w >= P.  scale must equal the dictionary's.  Device scratch
 * memory comes from the context allocator.  Errors: INVALID_ARG (sizes,
 * scale mismatch, K out of range), OOM, CUDA. */
zoom_status zoom_upscale(zoom_index ix, const float* lr, int32_t h, int32_t w, int32_t scale,
                         const zoom_upscale_params* prm, float* hr, void* stream);

/* zoom_upscale_batch: zoom_upscale of n_images LR images of any sizes and of
 * several scales in one call.  ixs: n_indexes index handles of one context,
 * one per scale (image i uses the index whose dictionary has scale[i]).
 * lr, hr: host arrays of n_images device pointers (hr[i] caller-allocated
 * (scale[i]*h[i]) x (scale[i]*w[i])); h, w, scale: host arrays.  The
 * queries of all images of one scale are concatenated and searched by one
 * persistent launch.  On the first call for a set of images (same pointers,
 * sizes and parameters), the search's dictionary split and list size are
 * autotuned on a sample of the queries (CUDA events; synchronises), then
 * every launch of the batch is recorded once into a CUDA graph; later calls
 * with the same set only launch that graph on `stream` (the image contents
 * may change).  per_image_ms (host, optional): device time from the start of
 * the batch to the completion of image i (synchronises `stream`).  The
 * recording keeps its scratch memory until zoom_batch_release, a call with
 * a different set, or zoom_ctx_destroy. */
zoom_status zoom_upscale_batch(const zoom_index* ixs, int32_t n_indexes, int32_t n_images,
                               const float* const* lr, const int32_t* h, const int32_t* w,
                               const int32_t* scale, const zoom_upscale_params* prm,
                               float* const* hr, void* stream, float* per_image_ms);
/* Frees the recorded batch of a context (synchronises the device). */
zoom_status zoom_batch_release(zoom_ctx ctx);

/* zoom_query: the per-patch steps only, for every LR patch origin (i, j) in
 * row order, n_q = (h-P+1)(w-P+1).  Outputs (device, any may be NULL except
 * nbr): keys uint64 [n_q][L] bucket keys of the query (Eq. 10 folded);
 * nbr int32 [n_q][K] neighbour IDs in (distance, ID) order; dist float32
 * [n_q][K] squared distances; wgt float32 [n_q][K] LLE weights (Eq. 12-13);
 * mu float32 [n_q] patch means; bucket_sum int32 [n_q] sum of the L bin
 * sizes. */
zoom_status zoom_query(zoom_index ix, const float* lr, int32_t h, int32_t w,
                       const zoom_upscale_params* prm, uint64_t* keys, int32_t* nbr, float* dist,
                       float* wgt, float* mu, int32_t* bucket_sum, void* stream);

/* zoom_reconstruct: Eq. 14 blend of the HR patches of given neighbours plus
 * the overlap average (no back-projection).  nbr int32 [n_q][K], wgt float32
 * [n_q][K], mu float32 [n_q] (device); hr device (s*h) x (s*w).  Takes
 * n_q * (s*P)^2 floats of scratch from the context allocator for the blended
 * patches of a two-pass average; where that allocation fails it runs the
 * one-pass form of zoom_reconstruct_with, which needs none and gives the
 * same bits. */
zoom_status zoom_reconstruct(zoom_index ix, const int32_t* nbr, const float* wgt, const float* mu,
                             int32_t h, int32_t w, int32_t K, float* hr, void* stream);

/* zoom_backproject: bp_iters iterations of the approximate cross-bilateral
 * error back-projection (Sec. 4 Eq. 6-7, Sec. 4.3 Eq. 15-17) of the HR
 * estimate hr (device, (s*h) x (s*w), updated in place) against the LR
 * image lr (device, h x w), with the degradation `degr`. */
zoom_status zoom_backproject(zoom_ctx ctx, const zoom_degradation* degr, const float* lr, int32_t h,
                             int32_t w, const zoom_upscale_params* prm, float* hr, void* stream);

/* ---- differentiation (Sec. 4: posterior Eq. 5, likelihood Eq. 8, prior
 * Eq. 9; back-projection Eq. 6-7 as a MAP gradient step) ------------------ */

/* zoom_degrade: lr = D_s(B hr) (Sec. 2.1) in FP32; hr device H x W, lr
 * device (H/s) x (W/s) (sizes not divisible by s are cropped). */
zoom_status zoom_degrade(zoom_ctx ctx, const zoom_degradation* degr, const float* hr, int32_t H,
                         int32_t W, float* lr, void* stream);

/* zoom_degrade_adjoint: g_hr = B^T D^T g_lr, the adjoint of zoom_degrade for
 * H = s*h, W = s*w; g_lr device h x w, g_hr device (s*h) x (s*w). */
zoom_status zoom_degrade_adjoint(zoom_ctx ctx, const zoom_degradation* degr, const float* g_lr,
                                 int32_t h, int32_t w, float* g_hr, void* stream);

/* zoom_reconstruct_with: zoom_reconstruct (Eq. 14 + overlap average) with a
 * caller-supplied HR dictionary hr_res (device [N][hr_stride] floats, row n
 * = the HR patch of ID n minus its LR mean, row-major (s*P)^2 values,
 * hr_stride >= (s*P)^2). */
zoom_status zoom_reconstruct_with(zoom_index ix, const float* hr_res, int32_t hr_stride,
                                  const int32_t* nbr, const float* wgt, const float* mu, int32_t h,
                                  int32_t w, int32_t K, float* hr, void* stream);

/* zoom_reconstruct_adjoint: the adjoint of the reconstruction with the
 * neighbours and weights fixed.  Given grad_hr = dL/d(HR image) (device
 * (s*h) x (s*w)), writes grad_dict = dL/dR (device [N][grad_stride], every
 * row; rows of unused entries are 0) and, if grad_mu != NULL, dL/dmu (device
 * [n_q]).  The sum over the uses of an entry runs in ascending use order
 * (deterministic; no atomics).  grad_dict may be NULL. */
zoom_status zoom_reconstruct_adjoint(zoom_index ix, const int32_t* nbr, const float* wgt, int32_t h,
                                     int32_t w, int32_t K, const float* grad_hr, float* grad_dict,
                                     int32_t grad_stride, float* grad_mu, void* stream);

/* zoom_backward: the MAP energy of an LR image lr (device h x w) with fixed
 * neighbours nbr (device [n_q][K]),
 *   E(R) = || D B x - y ||^2 + lambda * sum over 4-neighbour patch pairs of
 *          the squared difference of their HR patches on the overlap,
 *   x = overlap average of P_n = mu_n + sum_m w_nm R[nbr_nm],
 * and its gradients.  wgt (device [n_q][K]) gives the LLE weights; NULL
 * recomputes them from the LR features (Eq. 12-13, regulariser reg_rel).
 * Outputs (any may be NULL): grad_x = 2 B^T D^T (D B x - y) (device HR: the
 * gradient of the data term at x, i.e. the MAP back-projection direction),
 * grad_dict = dE/dR (device [N][grad_stride]), hr_out = x (device HR),
 * energy (host; when given, the call synchronises `stream`). */
zoom_status zoom_backward(zoom_index ix, const float* lr, int32_t h, int32_t w, const int32_t* nbr,
                          const float* wgt, int32_t K, float reg_rel, float lambda, float* grad_x,
                          float* grad_dict, int32_t grad_stride, float* hr_out, double* energy,
                          void* stream);

/* zoom_backproject_noalloc: zoom_backproject for callers that cannot
 * allocate device memory (for instance code living inside another
 * framework's fixed memory budget, real-time pipelines whose memory is
 * reserved up front, or work being recorded where an allocation would break
 * the recording).  The paper has no counterpart: this is a service of this
 * library.  It takes a CUDA device index instead of a context (creating a
 * context allocates) and makes that device current.  Inputs and outputs are
 * as for zoom_backproject; it calls no allocator.  Its scratch memory (the
 * second HR image and the LR error image) is a library-owned static device
 * array of ZOOM_NOALLOC_SCRATCH_FLOATS floats (8 MiB), held by every GPU
 * that loads the library until the process exits; an image needs
 * round_up((s*h)*(s*w), 64) + h*w floats of it, larger requests return
 * ZOOM_ERR_INVALID_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress): make that first call before any
 * stream capture.  The address is kept for the life of the process, so a
 * device reset (cudaDeviceReset, or the primary context torn down and made
 * again) after the first call on that device is not supported.  All calls
 * share the one array: calls whose work overlaps on the GPU (different
 * streams, or threads without ordering) race; order them on one stream.
 * Errors: INVALID_ARG (NULL pointers, a device index out of range, sizes or
 * parameters out of range, an image beyond the scratch), CUDA (the runtime
 * failed, e.g. no device can be counted). */
#define ZOOM_NOALLOC_SCRATCH_FLOATS (2u * 1024u * 1024u)
zoom_status zoom_backproject_noalloc(int device, const zoom_degradation* degr, const float* lr,
                                     int32_t h, int32_t w, const zoom_upscale_params* prm,
                                     float* hr, void* stream);

/* zoom_get_stats: synchronises `stream` and returns the counters of the
 * last zoom_query / zoom_upscale on ctx. */
zoom_status zoom_get_stats(zoom_ctx ctx, void* stream, zoom_stats* out);

/* zoom_set_stage_timing: when enable != 0, zoom_query / zoom_upscale record
 * CUDA events on their stream between stages (zoom_stats.ms_stage). */
zoom_status zoom_set_stage_timing(zoom_ctx ctx, int32_t enable);

/* zoom_set_fault_injection: a testing aid for the failure paths (the paper
 * has no counterpart).  Every wait inside the tensor-core filter is bounded:
 * after wait_limit_ns (0 = the default, 2 s; at most 60 s) it gives up, the
 * kernel's roles wait for their own copies and MMAs in flight, free their
 * TMEM and return, and the context's status word reads ZOOM_ERR_TIMEOUT
 * (zoom_sync_status).  mode 1 makes every filter CTA withhold the release of
 * its accumulators from the third dictionary tile of its first work item on,
 * so that such a wait runs out; the call's outputs are then not meaningful,
 * but reading them is safe (no access leaves its buffer) and the context
 * stays usable.  mode 0 turns it off.  Applies to later calls on ctx.
 * Errors: INVALID_ARG for other modes or limits. */
zoom_status zoom_set_fault_injection(zoom_ctx ctx, int32_t mode, uint64_t wait_limit_ns);

/* zoom_sync_status: synchronises `stream` and reads (then clears) the
 * context's device status word: ZOOM_OK, ZOOM_ERR_TIMEOUT or
 * ZOOM_ERR_DEVICE. */
zoom_status zoom_sync_status(zoom_ctx ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ZOOM_H */
