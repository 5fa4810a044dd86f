// C ABI of the zoom library: argument checks, handles, orchestration.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "zoom_internal.h"

namespace {
thread_local std::string g_last_error = "";

zoom_status fail(zoom_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define ZCHECK_CUDA(expr)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ZOOM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Scratch {
  zoom_ctx ctx;
  cudaStream_t st;
  void* p = nullptr;
  size_t bytes = 0;
  Scratch(zoom_ctx c, cudaStream_t s) : ctx(c), st(s) {}
  bool get(size_t b) {
    bytes = b;
    p = zoom_alloc(ctx, b, st);
    return p != nullptr || b == 0;
  }
  ~Scratch() {
    if (p) zoom_free(ctx, p, bytes, st);
  }
};

// Carves aligned sub-buffers out of one allocation.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* r = (T*)(base ? base + off : nullptr);
    off += count * sizeof(T);
    return r;
  }
};

}  // namespace

zoom_dict zoom_dict_alloc(zoom_ctx ctx, int64_t n, int P, int s, double blur_sigma, int feature,
                          cudaStream_t st) {
  zoom_dict d = new zoom_dict_s();
  d->ctx = ctx;
  d->n = n;
  d->P = P;
  d->s = s;
  d->feature = feature;
  d->d = feature ? 2 * P * P : P * P;
  d->dpad = (d->d + 3) / 4 * 4;
  d->PH = s * P;
  d->ph2 = d->PH * d->PH;
  d->ph2pad = (d->ph2 + 3) / 4 * 4;
  d->blur_sigma = blur_sigma;
  Carver c0(nullptr);
  c0.take<float>(n * P * P);
  c0.take<float>(n * d->dpad);
  c0.take<float>(n);
  c0.take<float>(n);
  c0.take<float>(n * d->ph2pad);
  d->bytes = c0.off + 256;
  void* mem = zoom_alloc(ctx, d->bytes, st);
  if (!mem) {
    delete d;
    return nullptr;
  }
  Carver c(mem);
  d->lr_pix = c.take<float>(n * P * P);   // first: the allocation's base
  d->feat = c.take<float>(n * d->dpad);
  d->mu = c.take<float>(n);
  d->norm2 = c.take<float>(n);
  d->hr_res = c.take<float>(n * d->ph2pad);
  return d;
}

namespace {

bool check_upscale_params(const zoom_upscale_params* p, zoom_dict d, std::string& why) {
  if (!p) { why = "params is NULL"; return false; }
  if (p->K < 1 || p->K > 16) { why = "K must be in 1..16"; return false; }
  if (p->K > d->n) { why = "K exceeds the dictionary size"; return false; }
  if (!(p->reg_rel >= 0.f) || !isfinite(p->reg_rel)) { why = "reg_rel must be >= 0"; return false; }
  if (p->bp_iters < 0 || p->bp_iters > 64) { why = "bp_iters must be in 0..64"; return false; }
  if (p->bp_iters > 0) {
    if (p->bp_radius < 1 || p->bp_radius > 7) { why = "bp_radius must be in 1..7"; return false; }
    if (!(p->sigma_spatial > 0.f) || !(p->sigma_range > 0.f)) { why = "sigmas must be > 0"; return false; }
  }
  if (p->precision != 0 && p->precision != 1) { why = "precision must be 0 or 1"; return false; }
  if (p->precision == 1 && (p->rerank_mult < 1 || p->rerank_mult * p->K > 32)) {
    why = "rerank_mult * K must be in K..32"; return false;
  }
  if (p->search < 0 || p->search > 3) { why = "search must be 0, 1, 2 or 3"; return false; }
  return true;
}

}  // namespace

void zoom_set_error(const std::string& msg) { g_last_error = msg; }

void zoom_stage_mark(zoom_ctx ctx, int i, cudaStream_t st) {
  if (!ctx->stage_timing || i < 0 || i >= kStageEvents) return;
  if (cudaEventRecord(ctx->stage_ev[i], st) == cudaSuccess) ctx->stage_rec[i] = true;
}

void* zoom_alloc(zoom_ctx ctx, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return nullptr;
  if (ctx->has_alloc) return ctx->alloc.alloc(bytes, (void*)st, ctx->alloc.user);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void zoom_free(zoom_ctx ctx, void* p, size_t bytes, cudaStream_t st) {
  if (!p) return;
  if (ctx->has_alloc) {
    ctx->alloc.free(p, bytes, (void*)st, ctx->alloc.user);
    return;
  }
  cudaFreeAsync(p, st);
}

extern "C" {

const char* zoom_status_string(zoom_status s) {
  switch (s) {
    case ZOOM_OK: return "ok";
    case ZOOM_ERR_INVALID_ARG: return "invalid argument";
    case ZOOM_ERR_OOM: return "out of device memory";
    case ZOOM_ERR_CUDA: return "CUDA error";
    case ZOOM_ERR_TIMEOUT: return "device wait timed out";
    case ZOOM_ERR_UNSUPPORTED: return "unsupported";
    case ZOOM_ERR_STATE: return "invalid handle state";
    case ZOOM_ERR_IO: return "I/O error";
    case ZOOM_ERR_DEVICE: return "device-side check failed";
  }
  return "unknown status";
}

const char* zoom_last_error(void) { return g_last_error.c_str(); }

zoom_status zoom_ctx_create(int device, const zoom_allocator* alloc, zoom_ctx* out) {
  if (!out) return fail(ZOOM_ERR_INVALID_ARG, "out is NULL");
  int n = 0;
  ZCHECK_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(ZOOM_ERR_INVALID_ARG, "no such device");
  if (alloc && (!alloc->alloc || !alloc->free))
    return fail(ZOOM_ERR_INVALID_ARG, "allocator needs both alloc and free");
  ZCHECK_CUDA(cudaSetDevice(device));
  zoom_ctx c = new zoom_ctx_s();
  c->device = device;
  cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (alloc) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  if (cudaMalloc(&c->d_status, 64) != cudaSuccess ||
      cudaMalloc(&c->d_counters, CNT_N * sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(c->d_status);
    delete c;
    return fail(ZOOM_ERR_OOM, "context buffers");
  }
  cudaMemset(c->d_status, 0, 64);
  cudaMemset(c->d_counters, 0, CNT_N * sizeof(unsigned long long));
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  for (int i = 0; i < kStageEvents; ++i) cudaEventCreate(&c->stage_ev[i]);
  *out = c;
  return ZOOM_OK;
}

void zoom_ctx_destroy(zoom_ctx c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  zoom_release_batch(c);
  cudaFree(c->d_status);
  cudaFree(c->d_counters);
  cudaEventDestroy(c->ev0);
  cudaEventDestroy(c->ev1);
  for (int i = 0; i < kStageEvents; ++i) cudaEventDestroy(c->stage_ev[i]);
  delete c;
}

// ---------------------------------------------------------------------------
// dictionary
// ---------------------------------------------------------------------------

zoom_status zoom_build_dictionary(zoom_ctx ctx, const float* const* hr_images,
                                  const int32_t* heights, const int32_t* widths,
                                  int32_t n_images, const zoom_degradation* degr,
                                  int64_t n_pairs, const int32_t* positions, uint64_t seed, void* stream,
                                  zoom_dict* out) {
  if (!ctx || !hr_images || !heights || !widths || !degr || !out)
    return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  const int s = degr->scale, P = degr->lr_patch;
  if (s < 1 || s > 4) return fail(ZOOM_ERR_INVALID_ARG, "scale must be in 1..4");
  if (P != 3 && P != 5) return fail(ZOOM_ERR_UNSUPPORTED, "lr_patch must be 3 or 5");
  if (!(degr->blur_sigma > 0.f)) return fail(ZOOM_ERR_INVALID_ARG, "blur_sigma must be > 0");
  if (degr->feature < 0 || degr->feature > 2) return fail(ZOOM_ERR_INVALID_ARG, "feature must be 0, 1 or 2");
  if (n_images < 1 || n_pairs < 1 || n_pairs > (1LL << 30))
    return fail(ZOOM_ERR_INVALID_ARG, "n_images and n_pairs must be positive");
  for (int m = 0; m < n_images; ++m) {
    if (!hr_images[m]) return fail(ZOOM_ERR_INVALID_ARG, "NULL image pointer");
    if (heights[m] / s < P || widths[m] / s < P)
      return fail(ZOOM_ERR_INVALID_ARG, "training image smaller than one patch");
  }
  // no positions given: draw them from the seed (uniform without
  // replacement over the LR patch origins, in origin order)
  std::vector<int32_t> drawn;
  if (!positions) {
    std::vector<int32_t> lh(n_images), lw(n_images);
    for (int m = 0; m < n_images; ++m) {
      lh[m] = heights[m] / s;
      lw[m] = widths[m] / s;
    }
    if (n_pairs > zoom_count_origins(n_images, lh.data(), lw.data(), P))
      return fail(ZOOM_ERR_INVALID_ARG, "n_pairs exceeds the LR patch origins of the images");
    drawn.resize((size_t)n_pairs * 3);
    zoom_sample_positions_host(seed, n_images, lh.data(), lw.data(), P, n_pairs, drawn.data());
    positions = drawn.data();
  }
  for (int64_t e = 0; e < n_pairs; ++e) {
    int m = positions[3 * e], i = positions[3 * e + 1], j = positions[3 * e + 2];
    if (m < 0 || m >= n_images || i < 0 || j < 0 || i + P > heights[m] / s ||
        j + P > widths[m] / s)
      return fail(ZOOM_ERR_INVALID_ARG, "position " + std::to_string(e) + " leaves its image");
  }
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  zoom_dict d = zoom_dict_alloc(ctx, n_pairs, P, s, degr->blur_sigma, degr->feature, st);
  if (!d) return fail(ZOOM_ERR_OOM, "dictionary arrays");
  void* mem = d->lr_pix;

  // scratch: LR images, pointer/width tables, positions
  size_t lr_total = 0;
  std::vector<size_t> lr_off(n_images);
  for (int m = 0; m < n_images; ++m) {
    lr_off[m] = lr_total;
    lr_total += (size_t)(heights[m] / s) * (widths[m] / s);
    lr_total = (lr_total + 63) / 64 * 64;
  }
  Carver sc(nullptr);
  sc.take<float>(lr_total);
  sc.take<const float*>(n_images);
  sc.take<const float*>(n_images);
  sc.take<int32_t>(n_images);
  sc.take<int32_t>(n_images);
  sc.take<int32_t>(n_images);
  sc.take<int32_t>(n_pairs * 3);
  Scratch scr(ctx, st);
  if (!scr.get(sc.off + 256)) {
    zoom_free(ctx, mem, d->bytes, st);
    delete d;
    return fail(ZOOM_ERR_OOM, "dictionary build scratch");
  }
  Carver s2(scr.p);
  float* lr_all = s2.take<float>(lr_total);
  const float** d_lr_ptr = s2.take<const float*>(n_images);
  const float** d_hr_ptr = s2.take<const float*>(n_images);
  int32_t* d_lr_h = s2.take<int32_t>(n_images);
  int32_t* d_lr_w = s2.take<int32_t>(n_images);
  int32_t* d_hr_w = s2.take<int32_t>(n_images);
  int32_t* d_pos = s2.take<int32_t>(n_pairs * 3);
  std::vector<const float*> h_lr_ptr(n_images), h_hr_ptr(n_images);
  std::vector<int32_t> h_lr_h(n_images), h_lr_w(n_images), h_hr_w(n_images);
  zoom_status rc = ZOOM_OK;
  for (int m = 0; m < n_images && rc == ZOOM_OK; ++m) {
    float* lr = lr_all + lr_off[m];
    h_lr_ptr[m] = lr;
    h_hr_ptr[m] = hr_images[m];
    h_lr_h[m] = heights[m] / s;
    h_lr_w[m] = widths[m] / s;
    h_hr_w[m] = widths[m];
    cudaError_t e = launch_degrade_exact(hr_images[m], heights[m], widths[m], s, degr->blur_sigma,
                                         lr, st);
    if (e != cudaSuccess) rc = fail(ZOOM_ERR_CUDA, std::string("degrade: ") + cudaGetErrorString(e));
  }
  if (rc == ZOOM_OK) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_lr_ptr, h_lr_ptr.data(), n_images * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_hr_ptr, h_hr_ptr.data(), n_images * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_lr_h, h_lr_h.data(), n_images * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_lr_w, h_lr_w.data(), n_images * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_hr_w, h_hr_w.data(), n_images * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_pos, positions, n_pairs * 12, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = launch_dict_gather(d_lr_ptr, d_lr_h, d_lr_w, d_hr_ptr, d_hr_w, d_pos, n_pairs, P, s, d, st);
    // the host vectors must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = fail(ZOOM_ERR_CUDA, std::string("dictionary: ") + cudaGetErrorString(e));
  }
  if (rc != ZOOM_OK) {
    zoom_free(ctx, mem, d->bytes, st);
    delete d;
    return rc;
  }
  *out = d;
  return ZOOM_OK;
}

void zoom_dict_destroy(zoom_dict d) {
  if (!d) return;
  cudaSetDevice(d->ctx->device);
  zoom_free(d->ctx, d->lr_pix, d->bytes, nullptr);
  delete d;
}

zoom_status zoom_dict_info(zoom_dict d, int64_t* n, int32_t* patch, int32_t* scale, double* blur_sigma,
                           int32_t* feature, int32_t* feature_dim) {
  if (!d) return fail(ZOOM_ERR_INVALID_ARG, "NULL dictionary");
  if (n) *n = d->n;
  if (patch) *patch = d->P;
  if (scale) *scale = d->s;
  if (blur_sigma) *blur_sigma = d->blur_sigma;
  if (feature) *feature = d->feature;
  if (feature_dim) *feature_dim = d->d;
  return ZOOM_OK;
}

zoom_status zoom_index_info(zoom_index ix, zoom_lsh_params* lsh) {
  if (!ix) return fail(ZOOM_ERR_INVALID_ARG, "NULL index");
  if (lsh) {
    lsh->L = ix->L;
    lsh->k = ix->k;
    lsh->w = ix->w;
    lsh->min_table_hits = ix->t;
    lsh->max_candidates = ix->cap;
    lsh->proj_dist = ix->proj_dist;
    lsh->seed = ix->seed;
  }
  return ZOOM_OK;
}

zoom_status zoom_dict_export(zoom_dict d, float* lr_pix, float* mu, float* hr_res, void* stream) {
  if (!d) return fail(ZOOM_ERR_INVALID_ARG, "NULL dictionary");
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(d->ctx->device));
  if (lr_pix)
    ZCHECK_CUDA(cudaMemcpyAsync(lr_pix, d->lr_pix, d->n * d->P * d->P * 4, cudaMemcpyDeviceToHost, st));
  if (mu) ZCHECK_CUDA(cudaMemcpyAsync(mu, d->mu, d->n * 4, cudaMemcpyDeviceToHost, st));
  if (hr_res)
    ZCHECK_CUDA(cudaMemcpy2DAsync(hr_res, d->ph2 * 4, d->hr_res, d->ph2pad * 4, d->ph2 * 4, d->n,
                                  cudaMemcpyDeviceToHost, st));
  ZCHECK_CUDA(cudaStreamSynchronize(st));
  return ZOOM_OK;
}

// ---------------------------------------------------------------------------
// index
// ---------------------------------------------------------------------------

zoom_status zoom_build_index(zoom_dict d, const zoom_lsh_params* lsh, const float* alpha,
                             const float* beta, void* stream, zoom_index* out) {
  if (!d || !lsh || !out) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  if (!alpha != !beta) return fail(ZOOM_ERR_INVALID_ARG, "give both alpha and beta, or neither");
  if (lsh->proj_dist < 0 || lsh->proj_dist > 1) return fail(ZOOM_ERR_INVALID_ARG, "proj_dist must be 0 or 1");
  if (lsh->L < 1 || lsh->L > 32 || lsh->k < 1 || lsh->k > 32)
    return fail(ZOOM_ERR_INVALID_ARG, "L and k must be in 1..32");
  if (!(lsh->w > 0.f) || !isfinite(lsh->w)) return fail(ZOOM_ERR_INVALID_ARG, "w must be > 0");
  if (lsh->min_table_hits < 1 || lsh->min_table_hits > lsh->L)
    return fail(ZOOM_ERR_INVALID_ARG, "min_table_hits must be in 1..L");
  if (lsh->max_candidates < 0 || lsh->max_candidates > 4096)
    return fail(ZOOM_ERR_INVALID_ARG, "max_candidates must be in 0..4096");
  const size_t smem = (size_t)lsh->L * lsh->k * ((d->d + 3) / 4 * 4 + 1) * 4;
  if (smem > 200 * 1024) return fail(ZOOM_ERR_INVALID_ARG, "L*k*(d+1) too large");
  zoom_ctx ctx = d->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  const int64_t N = d->n;
  const int L = lsh->L, k = lsh->k;
  // no draws given: the library's own, from the seed (zoom_lsh_draws)
  std::vector<float> drawn_a, drawn_b;
  if (!alpha) {
    drawn_a.resize((size_t)L * k * d->d);
    drawn_b.resize((size_t)L * k);
    zoom_draw_projections(L, k, d->d, lsh->w, lsh->proj_dist, lsh->seed, drawn_a.data(), drawn_b.data());
    alpha = drawn_a.data();
    beta = drawn_b.data();
  }
  zoom_index ix = new zoom_index_s();
  ix->dict = d;
  ix->L = L;
  ix->k = k;
  ix->w = lsh->w;
  ix->t = lsh->min_table_hits;
  ix->cap = lsh->max_candidates;
  ix->proj_dist = drawn_a.empty() ? 0 : lsh->proj_dist;
  ix->seed = drawn_a.empty() ? 0 : lsh->seed;
  ix->nd_rows = tc_rows_padded(N, true);   // whole 256-row steps for the wide-step filter
  {
    Carver c(nullptr);
    c.take<float>((size_t)L * k * d->d);
    c.take<float>((size_t)L * k);
    c.take<uint64_t>(N * L);
    c.take<uint64_t>(N * L);
    c.take<int32_t>((N + 1) * L);
    c.take<int32_t>(N * L);
    c.take<int32_t>(L);
    c.take<uint16_t>(ix->nd_rows * tc_kc(d->d, 0) * 8);
    c.take<uint16_t>(ix->nd_rows * tc_kc(d->d, 1) * 8);
    c.take<uint16_t>(ix->nd_rows * tc_kc(d->d, 2) * 8);
    ix->bytes = c.off + 256;
  }
  void* mem = zoom_alloc(ctx, ix->bytes, st);
  if (!mem) {
    delete ix;
    return fail(ZOOM_ERR_OOM, "index arrays");
  }
  Carver c(mem);
  ix->alpha = c.take<float>((size_t)L * k * d->d);
  ix->beta = c.take<float>((size_t)L * k);
  ix->dkeys = c.take<uint64_t>(N * L);
  ix->ukeys = c.take<uint64_t>(N * L);
  ix->offs = c.take<int32_t>((N + 1) * L);
  ix->ids = c.take<int32_t>(N * L);
  ix->nuniq = c.take<int32_t>(L);
  ix->dop16 = c.take<uint16_t>(ix->nd_rows * tc_kc(d->d, 0) * 8);
  ix->dopbf = c.take<uint16_t>(ix->nd_rows * tc_kc(d->d, 1) * 8);
  ix->dopf1 = c.take<uint16_t>(ix->nd_rows * tc_kc(d->d, 2) * 8);
  zoom_status rc = ZOOM_OK;
  cudaError_t e = cudaMemcpyAsync(ix->alpha, alpha, (size_t)L * k * d->d * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ix->beta, beta, (size_t)L * k * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_hash(d->feat, d->dpad, d->d, N, ix->alpha, ix->beta, L, k, ix->w, ix->dkeys, st);
  if (e == cudaSuccess)
    e = launch_operand(d->feat, d->dpad, d->d, N, ix->nd_rows, 1, 0, ix->dop16, nullptr, st);
  if (e == cudaSuccess)
    e = launch_operand(d->feat, d->dpad, d->d, N, ix->nd_rows, 1, 1, ix->dopbf, nullptr, st);
  if (e == cudaSuccess)
    e = launch_operand(d->feat, d->dpad, d->d, N, ix->nd_rows, 1, 2, ix->dopf1, nullptr, st);
  if (e == cudaSuccess) {
    Scratch scr(ctx, st);
    size_t sb = csr_build_scratch_bytes(N, L);
    if (!scr.get(sb)) {
      rc = fail(ZOOM_ERR_OOM, "index build scratch");
    } else {
      e = build_csr_tables(ix, scr.p, sb, st);
    }
    if (e == cudaSuccess && rc == ZOOM_OK) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess && rc == ZOOM_OK) rc = fail(ZOOM_ERR_CUDA, std::string("index: ") + cudaGetErrorString(e));
  if (rc != ZOOM_OK) {
    zoom_free(ctx, mem, ix->bytes, st);
    delete ix;
    return rc;
  }
  d->index_refs++;
  *out = ix;
  return ZOOM_OK;
}

void zoom_index_destroy(zoom_index ix) {
  if (!ix) return;
  cudaSetDevice(ix->dict->ctx->device);
  ix->dict->index_refs--;
  zoom_free(ix->dict->ctx, ix->alpha, ix->bytes, nullptr);
  delete ix;
}

zoom_status zoom_index_export(zoom_index ix, uint64_t* keys, int32_t* n_bins, void* stream) {
  if (!ix || !keys) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(ix->dict->ctx->device));
  ZCHECK_CUDA(cudaMemcpyAsync(keys, ix->dkeys, ix->dict->n * ix->L * 8, cudaMemcpyDeviceToHost, st));
  if (n_bins) ZCHECK_CUDA(cudaMemcpyAsync(n_bins, ix->nuniq, ix->L * 4, cudaMemcpyDeviceToHost, st));
  ZCHECK_CUDA(cudaStreamSynchronize(st));
  return ZOOM_OK;
}

// ---------------------------------------------------------------------------
// inference
// ---------------------------------------------------------------------------

namespace {

struct QueryBufs {
  float* feat;
  float* mu;
  float* norm2;
  uint64_t* keys;
  int32_t* nbr;
  float* dist;
  float* wgt;
  int32_t* bucket_sum;
};

// How one neighbour search runs: the SIMT scan, or the tensor-core filter
// with MC-entry lists over nsplit dictionary splits, and its scratch size.
struct SearchPlan {
  bool tc = false;
  bool capped = false;   // the index caps the candidate set (Sec. 4.2 early stop)
  int tail_split = 0;     // > 0: whole pairs, then the last round's pairs cut in parts
  int prec = 0, MC = 16, nsplit = 1, KCH = 80;
  int64_t q_rows = 0;
  // precision 2: the queries the single-term filter cannot settle (at most
  // cap2) run again through the FP16-split filter, nsplit2 dictionary parts
  int64_t cap2 = 0, q_rows2 = 0;
  int MC2 = 16, nsplit2 = 1;
  size_t bytes = 0;
};

SearchPlan plan_search(zoom_index ix, const zoom_upscale_params* prm, int64_t nq, int nsplit_override,
                       int mc_override) {
  zoom_dict d = ix->dict;
  SearchPlan p;
  if (ix->cap > 0) {
    p.capped = true;
    Carver c(nullptr);
    c.take<unsigned long long>(2);
    c.take<int32_t>((size_t)nq * ix->cap);
    c.take<int32_t>(nq);
    p.bytes = c.off + 256;
    return p;
  }
  p.tc = prm->precision == 1 || prm->search >= 2 || (prm->search == 0 && d->n >= 4096);
  if (!p.tc) return p;
  // the exact form: the single-term FP16 filter with the split-filter second
  // stage (internal precision 2), or the split filter alone (search 3)
  p.prec = prm->precision == 1 ? 1 : (prm->search == 3 ? 0 : 2);
  p.MC = mc_override > 0 ? mc_override : tc_list_size(p.prec, prm->K, prm->rerank_mult);
  p.KCH = tc_kc(d->d, p.prec) * 8;
  // the narrow forms step through the dictionary 256 rows at a time
  const int64_t unit_rows = tc_wide_form(p.prec, p.KCH / 8) ? 256 : 128;
  const int64_t nd_tiles = ix->nd_rows / unit_rows;
  const int64_t nq_pairs = (nq + 255) / 256;
  // Every CTA streams the dictionary tiles in the same order at about the
  // same pace, so L2 serves nearly all of them whatever the dictionary size.
  // The persistent CTAs take (query pair, split) items in turn, so the last
  // round decides the run time: the split count minimises the tiles of the
  // busiest CTA, each item charged a restart of its best chunk lists (about
  // MC*(1 + ln(N/32/MC)) merged chunks per query, most in the first tiles),
  // measured at about 768 128-row tiles (98,304 rows).
  const int64_t kRestartTiles = 98304 / unit_rows;
  int64_t nsplit = nsplit_override;
  if (nsplit <= 0 && nq_pairs >= d->ctx->n_sm) {
    // whole pairs in step over all SMs (every CTA streams the dictionary from
    // tile 0 together, so L2 serves it), then the pairs of the last, partial
    // round cut into S dictionary parts so that it ends sooner: S minimises
    // the tail's rounds * (tiles per part + list restart)
    const int64_t grid = d->ctx->n_sm;
    const int64_t tail = nq_pairs % grid;
    int64_t best = INT64_MAX;
    nsplit = 1;
    for (int64_t sp = 1; tail > 0 && sp <= std::min<int64_t>(8, nd_tiles); ++sp) {
      const int64_t tps = (nd_tiles + sp - 1) / sp;
      if ((sp - 1) * tps >= nd_tiles) continue;
      const int64_t cost = (tail * sp + grid - 1) / grid * (tps + kRestartTiles);
      if (cost < best) {
        best = cost;
        nsplit = sp;
      }
    }
    p.tail_split = (int)nsplit;
  } else if (nsplit <= 0) {
    int64_t best_cost = INT64_MAX;
    const int64_t grid = std::max(1, d->ctx->n_sm);
    for (int64_t ns = 1; ns <= std::min<int64_t>(8, nd_tiles); ++ns) {
      const int64_t tps = (nd_tiles + ns - 1) / ns;
      if ((ns - 1) * tps >= nd_tiles) continue;   // the last split would be empty
      const int64_t rounds = (nq_pairs * ns + grid - 1) / grid;
      const int64_t cost = rounds * (tps + kRestartTiles);
      if (cost < best_cost) {
        best_cost = cost;
        nsplit = ns;
      }
    }
  }
  p.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(nsplit, std::min<int64_t>(8, nd_tiles)));
  p.q_rows = tc_rows_padded(nq, true);
  if (p.prec == 2) {
    // room for 4x the unsettled share measured on the 1M-pair workload
    // (0.4 %): queries past it go straight to the (slow) SIMT scan
    p.cap2 = std::min<int64_t>(nq, std::max<int64_t>(8192, nq / 64));
    p.q_rows2 = tc_rows_padded(p.cap2, true);
    p.MC2 = tc_list_size(0, prm->K, prm->rerank_mult);
    p.nsplit2 = (int)std::min<int64_t>(8, nd_tiles);
  }
  Carver c(nullptr);
  c.take<unsigned long long>(2);
  c.take<uint16_t>(p.q_rows * p.KCH);
  c.take<float>(nq);
  c.take<float>((size_t)p.nsplit * nq * p.MC);
  c.take<int32_t>((size_t)p.nsplit * nq * p.MC);
  c.take<int32_t>(nq);
  if (p.prec == 2) {
    c.take<float>((size_t)p.cap2 * d->dpad);
    c.take<uint64_t>((size_t)p.cap2 * ix->L);
    c.take<uint16_t>((size_t)p.q_rows2 * tc_kc(d->d, 0) * 8);
    c.take<float>(p.cap2);
    c.take<float>((size_t)p.nsplit2 * p.cap2 * p.MC2);
    c.take<int32_t>((size_t)p.nsplit2 * p.cap2 * p.MC2);
    c.take<int32_t>(nq);
  }
  p.bytes = c.off + 256;
  return p;
}

// Adds a search's fallback counts to the context's statistics.
__global__ void k_add_fallback_counts(const unsigned long long* __restrict__ cnt,
                                      unsigned long long* __restrict__ counters) {
  counters[CNT_FALLBACK] += cnt[0];
  counters[CNT_FALLBACK2] += cnt[1];
}

// Neighbour search with a caller-provided workspace of plan.bytes: SIMT
// scan, or the capped walk, or the tensor-core search in its stages (the
// queries a stage leaves go to the next one, the lists counted in the
// workspace's own two counters, zeroed here: the workspace may serve many
// searches of one call or of a recorded batch).  Allocates nothing.
cudaError_t run_search_ws(zoom_index ix, const zoom_upscale_params* prm, const QueryBufs& b, int64_t nq,
                          const SearchPlan& pl, void* ws, cudaStream_t st) {
  zoom_dict d = ix->dict;
  zoom_ctx ctx = d->ctx;
  const int K = prm->K;
  if (!pl.tc && !pl.capped)
    return launch_knn_exact(ix, b.feat, b.keys, nq, K, b.nbr, b.dist, ctx->d_counters, nullptr,
                            nullptr, st);
  Carver s2(ws);
  unsigned long long* cnt = s2.take<unsigned long long>(2);   // [0] first list, [1] second
  cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (pl.capped) {
    int32_t* cand = s2.take<int32_t>((size_t)nq * ix->cap);
    int32_t* fb = s2.take<int32_t>(nq);
    e = launch_knn_capped(ix, b.feat, b.keys, nq, K, b.nbr, b.dist, cand, fb, cnt, st);
    if (e == cudaSuccess)
      e = launch_knn_exact(ix, b.feat, b.keys, nq, K, b.nbr, b.dist, ctx->d_counters, fb, cnt, st);
    if (e == cudaSuccess) {
      k_add_fallback_counts<<<1, 1, 0, st>>>(cnt, ctx->d_counters);
      e = cudaGetLastError();
    }
    return e;
  }
  uint16_t* qop = s2.take<uint16_t>(pl.q_rows * pl.KCH);
  float* qn = s2.take<float>(nq);
  float* ld = s2.take<float>((size_t)pl.nsplit * nq * pl.MC);
  int32_t* li = s2.take<int32_t>((size_t)pl.nsplit * nq * pl.MC);
  int32_t* fb = s2.take<int32_t>(nq);
  e = launch_operand(b.feat, d->dpad, d->d, nq, pl.q_rows, 0, pl.prec, qop, qn, st);
  zoom_stage_mark(ctx, 8, st);   // start of the tensor-core filter kernel
  if (e == cudaSuccess)
    e = launch_knn_tc(qop, qn, nq, pl.prec == 0 ? ix->dop16 : pl.prec == 1 ? ix->dopbf : ix->dopf1, d->n, pl.prec,
                      pl.KCH / 8, pl.MC, pl.nsplit, pl.tail_split, ctx->n_sm, ld, li, ctx->d_status, st, nullptr,
                      ctx->wait_ns, ctx->inject);
  zoom_stage_mark(ctx, 9, st);   // end of the filter kernel
  if (e == cudaSuccess)
    e = launch_rerank(d->d, pl.MC, K, b.feat, d->dpad, qn, b.keys, nq, d->feat, ix->dkeys, d->n, ix->L,
                      ix->t, ld, li, pl.nsplit, pl.prec == 0 ? 1 : (pl.prec == 1 ? 0 : 2), b.nbr, b.dist, fb,
                      cnt, st);
  if (pl.prec == 2) {
    // second stage, on the device's count of unsettled queries: compact
    // them, FP16-split operands, the split filter over nsplit2 parts, its
    // rerank (results written at the original query indices); what it
    // cannot settle joins fb2 for the SIMT scan
    float* cfeat = s2.take<float>((size_t)pl.cap2 * d->dpad);
    uint64_t* ckeys = s2.take<uint64_t>((size_t)pl.cap2 * ix->L);
    uint16_t* cqop = s2.take<uint16_t>((size_t)pl.q_rows2 * tc_kc(d->d, 0) * 8);
    float* cqn = s2.take<float>(pl.cap2);
    float* ld2 = s2.take<float>((size_t)pl.nsplit2 * pl.cap2 * pl.MC2);
    int32_t* li2 = s2.take<int32_t>((size_t)pl.nsplit2 * pl.cap2 * pl.MC2);
    int32_t* fb2 = s2.take<int32_t>(nq);
    if (e == cudaSuccess)
      e = launch_gather_queries(fb, cnt, nq, pl.cap2, b.feat, d->dpad, b.keys, ix->L, cfeat, ckeys, fb2, cnt + 1, st);
    if (e == cudaSuccess)
      e = launch_operand(cfeat, d->dpad, d->d, pl.cap2, pl.q_rows2, 0, 0, cqop, cqn, st, cnt);
    if (e == cudaSuccess)
      e = launch_knn_tc(cqop, cqn, pl.cap2, ix->dop16, d->n, 0, tc_kc(d->d, 0), pl.MC2, pl.nsplit2, 0, ctx->n_sm,
                        ld2, li2, ctx->d_status, st, cnt, ctx->wait_ns, ctx->inject);
    if (e == cudaSuccess)
      e = launch_rerank(d->d, pl.MC2, K, cfeat, d->dpad, cqn, ckeys, pl.cap2, d->feat, ix->dkeys, d->n, ix->L,
                        ix->t, ld2, li2, pl.nsplit2, 1, b.nbr, b.dist, fb2, cnt + 1, st, fb, cnt);
    if (e == cudaSuccess)
      e = launch_knn_exact(ix, b.feat, b.keys, nq, K, b.nbr, b.dist, ctx->d_counters, fb2, cnt + 1, st);
  } else if (e == cudaSuccess) {
    e = launch_knn_exact(ix, b.feat, b.keys, nq, K, b.nbr, b.dist, ctx->d_counters, fb, cnt, st);
  }
  if (e == cudaSuccess) {
    k_add_fallback_counts<<<1, 1, 0, st>>>(cnt, ctx->d_counters);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t run_search(zoom_index ix, const zoom_upscale_params* prm, const QueryBufs& b, int64_t nq,
                       cudaStream_t st, bool& oom) {
  const SearchPlan pl = plan_search(ix, prm, nq, 0, 0);
  if (!pl.tc && !pl.capped) return run_search_ws(ix, prm, b, nq, pl, nullptr, st);
  Scratch scr(ix->dict->ctx, st);
  if (!scr.get(pl.bytes)) {
    oom = true;
    return cudaSuccess;
  }
  return run_search_ws(ix, prm, b, nq, pl, scr.p, st);
}

zoom_status run_query_steps(zoom_index ix, const float* lr, int h, int w,
                            const zoom_upscale_params* prm, const QueryBufs& b, cudaStream_t st) {
  zoom_dict d = ix->dict;
  zoom_ctx ctx = d->ctx;
  const int64_t nq = (int64_t)(h - d->P + 1) * (w - d->P + 1);
  zoom_stage_mark(ctx, 0, st);
  cudaError_t e = launch_query_features(lr, h, w, d->P, d->feature, d->dpad, b.feat, b.mu, b.norm2, st);
  zoom_stage_mark(ctx, 1, st);
  if (e == cudaSuccess)
    e = launch_hash(b.feat, d->dpad, d->d, nq, ix->alpha, ix->beta, ix->L, ix->k, ix->w, b.keys, st);
  zoom_stage_mark(ctx, 2, st);
  if (e == cudaSuccess) e = launch_bucket_lookup(ix, b.keys, nq, b.bucket_sum, ctx->d_counters, st);
  zoom_stage_mark(ctx, 3, st);
  bool oom = false;
  if (e == cudaSuccess) e = run_search(ix, prm, b, nq, st, oom);
  if (oom) return fail(ZOOM_ERR_OOM, "neighbour search scratch");
  zoom_stage_mark(ctx, 4, st);
  if (e == cudaSuccess)
    e = launch_lle(d, b.feat, nq, b.nbr, b.dist, prm->K, prm->reg_rel, prm->fp64_cond_threshold,
                   b.wgt, ctx->d_counters, st);
  zoom_stage_mark(ctx, 5, st);
  if (e != cudaSuccess) return fail(ZOOM_ERR_CUDA, std::string("query: ") + cudaGetErrorString(e));
  return ZOOM_OK;
}

zoom_status begin_call(zoom_ctx ctx, int64_t nq, cudaStream_t st) {
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  for (int i = 0; i < kStageEvents; ++i) ctx->stage_rec[i] = false;
  ZCHECK_CUDA(cudaMemsetAsync(ctx->d_counters, 0, CNT_N * sizeof(unsigned long long), st));
  ZCHECK_CUDA(cudaEventRecord(ctx->ev0, st));
  ctx->last_n_queries = nq;
  ctx->timed = false;
  return ZOOM_OK;
}

zoom_status end_call(zoom_ctx ctx, cudaStream_t st) {
  ZCHECK_CUDA(cudaEventRecord(ctx->ev1, st));
  ctx->timed = true;
  return ZOOM_OK;
}

}  // namespace

zoom_status zoom_query(zoom_index ix, const float* lr, int32_t h, int32_t w,
                       const zoom_upscale_params* prm, uint64_t* keys, int32_t* nbr, float* dist,
                       float* wgt, float* mu, int32_t* bucket_sum, void* stream) {
  if (!ix || !lr || !nbr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  zoom_dict d = ix->dict;
  std::string why;
  if (!check_upscale_params(prm, d, why)) return fail(ZOOM_ERR_INVALID_ARG, why);
  if (ix->cap > 0 && prm->K > ix->cap) return fail(ZOOM_ERR_INVALID_ARG, "K exceeds max_candidates");
  if (h < d->P || w < d->P) return fail(ZOOM_ERR_INVALID_ARG, "image smaller than one patch");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nq = (int64_t)(h - d->P + 1) * (w - d->P + 1);
  const int K = prm->K;
  zoom_status rc = begin_call(d->ctx, nq, st);
  if (rc != ZOOM_OK) return rc;
  Carver c(nullptr);
  c.take<float>(nq * d->dpad);
  if (!mu) c.take<float>(nq);
  if (!keys) c.take<uint64_t>(nq * ix->L);
  if (!dist) c.take<float>(nq * K);
  if (!wgt) c.take<float>(nq * K);
  Scratch scr(d->ctx, st);
  if (!scr.get(c.off + 256)) return fail(ZOOM_ERR_OOM, "query scratch");
  Carver s2(scr.p);
  QueryBufs b;
  b.feat = s2.take<float>(nq * d->dpad);
  b.mu = mu ? mu : s2.take<float>(nq);
  b.norm2 = nullptr;
  b.keys = keys ? keys : s2.take<uint64_t>(nq * ix->L);
  b.dist = dist ? dist : s2.take<float>(nq * K);
  b.wgt = wgt ? wgt : s2.take<float>(nq * K);
  b.nbr = nbr;
  b.bucket_sum = bucket_sum;
  rc = run_query_steps(ix, lr, h, w, prm, b, st);
  if (rc != ZOOM_OK) return rc;
  return end_call(d->ctx, st);
}

zoom_status zoom_reconstruct(zoom_index ix, const int32_t* nbr, const float* wgt, const float* mu,
                             int32_t h, int32_t w, int32_t K, float* hr, void* stream) {
  if (!ix || !nbr || !wgt || !mu || !hr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  zoom_dict d = ix->dict;
  if (h < d->P || w < d->P) return fail(ZOOM_ERR_INVALID_ARG, "image smaller than one patch");
  if (K < 1 || K > 64) return fail(ZOOM_ERR_INVALID_ARG, "K must be in 1..64");
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(d->ctx->device));
  // the blended patches of the two-pass form; without room for them the
  // one-pass form (the same bits)
  Scratch scr(d->ctx, st);
  float* patches = scr.get((size_t)(h - d->P + 1) * (w - d->P + 1) * d->ph2 * 4) ? (float*)scr.p : nullptr;
  cudaError_t e = launch_overlap_add_staged(nbr, wgt, mu, d->hr_res, d->ph2pad, K, h, w, d->s, d->P, patches,
                                            hr, st);
  if (e != cudaSuccess) return fail(ZOOM_ERR_CUDA, std::string("reconstruct: ") + cudaGetErrorString(e));
  return ZOOM_OK;
}

static zoom_status run_backproject(zoom_ctx ctx, int s, double blur_sigma, const float* lr, int h,
                                   int w, const zoom_upscale_params* prm, float* hr, float* tmp,
                                   float* err, cudaStream_t st) {
  // ping-pong between hr and tmp; an odd count ends with a copy back
  float* a = hr;
  float* b = tmp;
  for (int it = 0; it < prm->bp_iters; ++it) {
    cudaError_t e = launch_bp_iteration(a, b, lr, err, h, w, s, blur_sigma, prm->sigma_spatial,
                                        prm->sigma_range, prm->bp_radius, st);
    if (e != cudaSuccess) return fail(ZOOM_ERR_CUDA, std::string("backproject: ") + cudaGetErrorString(e));
    std::swap(a, b);
  }
  if (a != hr)
    ZCHECK_CUDA(cudaMemcpyAsync(hr, a, (size_t)s * h * s * w * 4, cudaMemcpyDeviceToDevice, st));
  (void)ctx;
  return ZOOM_OK;
}

zoom_status zoom_backproject(zoom_ctx ctx, const zoom_degradation* degr, const float* lr, int32_t h,
                             int32_t w, const zoom_upscale_params* prm, float* hr, void* stream) {
  if (!ctx || !degr || !lr || !prm || !hr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  if (degr->scale < 1 || degr->scale > 4 || !(degr->blur_sigma > 0.f))
    return fail(ZOOM_ERR_INVALID_ARG, "bad degradation");
  if (h < 1 || w < 1) return fail(ZOOM_ERR_INVALID_ARG, "empty image");
  if (prm->bp_iters < 0 || prm->bp_iters > 64 || prm->bp_radius < 1 || prm->bp_radius > 7 ||
      !(prm->sigma_spatial > 0.f) || !(prm->sigma_range > 0.f))
    return fail(ZOOM_ERR_INVALID_ARG, "bad back-projection parameters");
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  const int s = degr->scale;
  Scratch scr(ctx, st);
  Carver c(nullptr);
  c.take<float>((size_t)s * h * s * w);
  c.take<float>((size_t)h * w);
  if (!scr.get(c.off + 256)) return fail(ZOOM_ERR_OOM, "backproject scratch");
  Carver s2(scr.p);
  float* tmp = s2.take<float>((size_t)s * h * s * w);
  float* err = s2.take<float>((size_t)h * w);
  return run_backproject(ctx, s, degr->blur_sigma, lr, h, w, prm, hr, tmp, err, st);
}

zoom_status zoom_upscale(zoom_index ix, const float* lr, int32_t h, int32_t w, int32_t scale,
                         const zoom_upscale_params* prm, float* hr, void* stream) {
  if (!ix || !lr || !hr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  zoom_dict d = ix->dict;
  std::string why;
  if (!check_upscale_params(prm, d, why)) return fail(ZOOM_ERR_INVALID_ARG, why);
  if (ix->cap > 0 && prm->K > ix->cap) return fail(ZOOM_ERR_INVALID_ARG, "K exceeds max_candidates");
  if (scale != d->s) return fail(ZOOM_ERR_INVALID_ARG, "scale differs from the dictionary's");
  if (h < d->P || w < d->P) return fail(ZOOM_ERR_INVALID_ARG, "image smaller than one patch");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nq = (int64_t)(h - d->P + 1) * (w - d->P + 1);
  const int K = prm->K, s = d->s;
  zoom_status rc = begin_call(d->ctx, nq, st);
  if (rc != ZOOM_OK) return rc;
  Carver c(nullptr);
  c.take<float>(nq * d->dpad);
  c.take<float>(nq);
  c.take<uint64_t>(nq * ix->L);
  c.take<int32_t>(nq * K);
  c.take<float>(nq * K);
  c.take<float>(nq * K);
  c.take<float>((size_t)s * h * s * w);
  c.take<float>((size_t)h * w);
  Scratch scr(d->ctx, st);
  if (!scr.get(c.off + 256)) return fail(ZOOM_ERR_OOM, "upscale scratch");
  Carver s2(scr.p);
  QueryBufs b;
  b.feat = s2.take<float>(nq * d->dpad);
  b.mu = s2.take<float>(nq);
  b.norm2 = nullptr;
  b.keys = s2.take<uint64_t>(nq * ix->L);
  b.nbr = s2.take<int32_t>(nq * K);
  b.dist = s2.take<float>(nq * K);
  b.wgt = s2.take<float>(nq * K);
  b.bucket_sum = nullptr;
  float* tmp = s2.take<float>((size_t)s * h * s * w);
  float* err = s2.take<float>((size_t)h * w);
  rc = run_query_steps(ix, lr, h, w, prm, b, st);
  if (rc != ZOOM_OK) return rc;
  // the blended patches of the two-pass overlap average; without room for
  // them the one-pass form (the same bits)
  Scratch pscr(d->ctx, st);
  float* patches = pscr.get((size_t)nq * d->ph2 * 4) ? (float*)pscr.p : nullptr;
  cudaError_t e =
      launch_overlap_add_staged(b.nbr, b.wgt, b.mu, d->hr_res, d->ph2pad, K, h, w, s, d->P, patches, hr, st);
  if (e != cudaSuccess) return fail(ZOOM_ERR_CUDA, std::string("overlap-add: ") + cudaGetErrorString(e));
  zoom_stage_mark(d->ctx, 6, st);
  rc = run_backproject(d->ctx, s, d->blur_sigma, lr, h, w, prm, hr, tmp, err, st);
  if (rc != ZOOM_OK) return rc;
  zoom_stage_mark(d->ctx, 7, st);
  return end_call(d->ctx, st);
}

zoom_status zoom_get_stats(zoom_ctx ctx, void* stream, zoom_stats* out) {
  if (!ctx || !out) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  unsigned long long c[CNT_N];
  ZCHECK_CUDA(cudaMemcpyAsync(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost, st));
  ZCHECK_CUDA(cudaStreamSynchronize(st));
  memset(out, 0, sizeof(*out));
  out->n_queries = ctx->last_n_queries;
  out->mean_bucket_sum = ctx->last_n_queries ? (double)c[CNT_BUCKET_SUM] / ctx->last_n_queries : 0.0;
  out->max_bucket_sum = (int64_t)c[CNT_BUCKET_MAX];
  out->n_empty = (int64_t)c[CNT_EMPTY];
  out->n_padded_queries = (int64_t)c[CNT_PADDED];
  out->n_fp64_solves = (int64_t)c[CNT_FP64];
  out->n_exact_match = (int64_t)c[CNT_EXACT];
  out->n_filter_fallback = (int64_t)c[CNT_FALLBACK];
  out->ms_total = 0.0;
  for (int i = 0; i < 7; ++i) {
    float ms = 0.f;
    if (ctx->stage_rec[i] && ctx->stage_rec[i + 1] &&
        cudaEventElapsedTime(&ms, ctx->stage_ev[i], ctx->stage_ev[i + 1]) == cudaSuccess)
      out->ms_stage[i] = ms;
    else
      cudaGetLastError();
  }
  {
    float ms = 0.f;   // the tensor-core filter kernel alone
    if (ctx->stage_rec[8] && ctx->stage_rec[9] &&
        cudaEventElapsedTime(&ms, ctx->stage_ev[8], ctx->stage_ev[9]) == cudaSuccess)
      out->ms_stage[7] = ms;
    else
      cudaGetLastError();
  }
  if (ctx->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) out->ms_total = ms;
    else cudaGetLastError();
  }
  return ZOOM_OK;
}

zoom_status zoom_set_stage_timing(zoom_ctx ctx, int32_t enable) {
  if (!ctx) return fail(ZOOM_ERR_INVALID_ARG, "NULL context");
  ctx->stage_timing = enable != 0;
  return ZOOM_OK;
}

zoom_status zoom_set_fault_injection(zoom_ctx ctx, int32_t mode, uint64_t wait_limit_ns) {
  if (!ctx) return fail(ZOOM_ERR_INVALID_ARG, "NULL context");
  if (mode < 0 || mode > 1) return fail(ZOOM_ERR_INVALID_ARG, "mode must be 0 or 1");
  if (wait_limit_ns > 60000000000ull) return fail(ZOOM_ERR_INVALID_ARG, "wait_limit_ns above 60 s");
  ctx->inject = mode;
  ctx->wait_ns = wait_limit_ns;
  return ZOOM_OK;
}

zoom_status zoom_sync_status(zoom_ctx ctx, void* stream) {
  if (!ctx) return fail(ZOOM_ERR_INVALID_ARG, "NULL context");
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  unsigned int v = 0;
  ZCHECK_CUDA(cudaMemcpyAsync(&v, ctx->d_status, 4, cudaMemcpyDeviceToHost, st));
  ZCHECK_CUDA(cudaStreamSynchronize(st));
  if (v == 0) return ZOOM_OK;
  ZCHECK_CUDA(cudaMemsetAsync(ctx->d_status, 0, 4, st));
  if (v == 1) return fail(ZOOM_ERR_TIMEOUT, "a device wait gave up");
  return fail(ZOOM_ERR_DEVICE, "device status word " + std::to_string(v));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batched zoom: one call for many LR images, recorded into a CUDA graph
// ---------------------------------------------------------------------------

namespace {

// Search choices picked by the autotuner, per (index, query count bucket,
// precision, K).
struct TuneKey {
  const void* ix;
  int64_t qbucket;
  int prec, K;
  bool operator<(const TuneKey& o) const {
    if (ix != o.ix) return ix < o.ix;
    if (qbucket != o.qbucket) return qbucket < o.qbucket;
    if (prec != o.prec) return prec < o.prec;
    return K < o.K;
  }
};
struct TuneChoice {
  int nsplit = 0, mc = 0;
  float ms = 0.f;
};
using TuneMap = std::map<TuneKey, TuneChoice>;

struct Group {
  zoom_index ix = nullptr;
  std::vector<int> images;
  std::vector<int64_t> q_off;   // query offset of each image in the group
  int64_t nq = 0;
  SearchPlan plan;
  QueryBufs b{};
  void* ws = nullptr;
};

struct BatchRecord {
  std::vector<int64_t> key;
  void* mem = nullptr;           // query buffers and back-projection scratch
  size_t bytes = 0;
  void* ws = nullptr;            // search scratch of every group
  size_t ws_bytes = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cudaEvent_t> ev;   // [0] start, [1 + i] end of image i
  std::vector<Group> groups;
};

void free_record(zoom_ctx ctx, BatchRecord* r) {
  if (r->exec) cudaGraphExecDestroy(r->exec);
  for (cudaEvent_t e : r->ev) cudaEventDestroy(e);
  if (r->cap) cudaStreamDestroy(r->cap);
  if (r->mem) zoom_free(ctx, r->mem, r->bytes, nullptr);
  if (r->ws) zoom_free(ctx, r->ws, r->ws_bytes, nullptr);
  delete r;
}

}  // namespace

void zoom_release_batch(zoom_ctx ctx) {
  if (ctx->batch) {
    cudaDeviceSynchronize();
    free_record(ctx, (BatchRecord*)ctx->batch);
    ctx->batch = nullptr;
  }
  delete (TuneMap*)ctx->tuned;
  ctx->tuned = nullptr;
}

namespace {

void release_batch(zoom_ctx ctx) {
  BatchRecord* r = (BatchRecord*)ctx->batch;
  if (!r) return;
  cudaDeviceSynchronize();   // the recorded graph may still run on the caller's stream
  free_record(ctx, r);
  ctx->batch = nullptr;
}

int64_t qbucket(int64_t nq) {
  int64_t b = 1;
  while (b < nq) b <<= 1;
  return b;
}

// Times each candidate (splits x list size) of one group's search on a
// sample of its queries and remembers the fastest.
zoom_status autotune_group(Group& g, const zoom_upscale_params* prm, cudaStream_t st) {
  zoom_ctx ctx = g.ix->dict->ctx;
  if (g.ix->cap > 0) return ZOOM_OK;   // the capped walk has nothing to tune
  TuneMap& tm = *(TuneMap*)ctx->tuned;
  const TuneKey key{g.ix, qbucket(g.nq), prm->precision, prm->K};
  if (tm.count(key)) return ZOOM_OK;
  const int64_t ns = std::min<int64_t>(g.nq, 131072);
  std::vector<std::pair<int, int>> cands;
  const int mc0 = tc_list_size(prm->precision, prm->K, prm->rerank_mult);
  for (int s : {0, 1, 2, 4}) {
    cands.push_back({s, mc0});
    if (prm->precision != 1 && mc0 == 16) cands.push_back({s, 32});
  }
  TuneChoice best;
  best.ms = 1e30f;
  cudaEvent_t e0, e1;
  ZCHECK_CUDA(cudaEventCreate(&e0));
  ZCHECK_CUDA(cudaEventCreate(&e1));
  for (auto& c : cands) {
    const SearchPlan pl = plan_search(g.ix, prm, ns, c.first, c.second);
    Scratch scr(ctx, st);
    if (!scr.get(pl.bytes)) continue;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // first run warms up
      cudaEventRecord(e0, st);
      cudaError_t e = run_search_ws(g.ix, prm, g.b, ns, pl, scr.p, st);
      cudaEventRecord(e1, st);
      if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(ZOOM_ERR_CUDA, "autotune search failed");
      }
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (ms < best.ms) {
      best.ms = ms;
      best.nsplit = c.first;
      best.mc = c.second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tm[key] = best;
  return ZOOM_OK;
}

}  // namespace

extern "C" {

zoom_status zoom_upscale_batch(const zoom_index* ixs, int32_t n_indexes, int32_t n_images,
                               const float* const* lr, const int32_t* h, const int32_t* w,
                               const int32_t* scale, const zoom_upscale_params* prm,
                               float* const* hr, void* stream, float* per_image_ms) {
  if (!ixs || n_indexes < 1 || n_images < 1 || !lr || !h || !w || !scale || !prm || !hr)
    return fail(ZOOM_ERR_INVALID_ARG, "NULL or empty argument");
  zoom_ctx ctx = ixs[0] ? ixs[0]->dict->ctx : nullptr;
  if (!ctx) return fail(ZOOM_ERR_INVALID_ARG, "NULL index");
  for (int j = 0; j < n_indexes; ++j) {
    if (!ixs[j]) return fail(ZOOM_ERR_INVALID_ARG, "NULL index");
    if (ixs[j]->dict->ctx != ctx) return fail(ZOOM_ERR_INVALID_ARG, "indexes of different contexts");
    std::string why;
    if (!check_upscale_params(prm, ixs[j]->dict, why)) return fail(ZOOM_ERR_INVALID_ARG, why);
    if (ixs[j]->cap > 0 && prm->K > ixs[j]->cap)
      return fail(ZOOM_ERR_INVALID_ARG, "K exceeds max_candidates");
  }
  cudaStream_t st = (cudaStream_t)stream;
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  cudaGetLastError();   // launch checks below read the runtime's last error
  // group the images by the index whose dictionary has their scale
  std::vector<Group> groups(n_indexes);
  std::vector<int64_t> key;
  key.push_back(n_images);
  for (int j = 0; j < n_indexes; ++j) {
    groups[j].ix = ixs[j];
    key.push_back((int64_t)(uintptr_t)ixs[j]);
  }
  for (int i = 0; i < n_images; ++i) {
    int g = -1;
    for (int j = 0; j < n_indexes; ++j)
      if (ixs[j]->dict->s == scale[i]) g = j;
    if (g < 0) return fail(ZOOM_ERR_INVALID_ARG, "no index for the scale of image " + std::to_string(i));
    zoom_dict d = ixs[g]->dict;
    if (!lr[i] || !hr[i] || h[i] < d->P || w[i] < d->P)
      return fail(ZOOM_ERR_INVALID_ARG, "bad image " + std::to_string(i));
    groups[g].images.push_back(i);
    groups[g].q_off.push_back(groups[g].nq);
    groups[g].nq += (int64_t)(h[i] - d->P + 1) * (w[i] - d->P + 1);
    for (int64_t v : {(int64_t)(uintptr_t)lr[i], (int64_t)(uintptr_t)hr[i], (int64_t)h[i], (int64_t)w[i],
                      (int64_t)scale[i]})
      key.push_back(v);
  }
  for (int64_t v : {(int64_t)prm->K, (int64_t)prm->bp_iters, (int64_t)prm->precision,
                    (int64_t)prm->rerank_mult, (int64_t)prm->search, (int64_t)prm->bp_radius,
                    (int64_t)(prm->reg_rel * 1e9f), (int64_t)(prm->sigma_spatial * 1e6f),
                    (int64_t)(prm->sigma_range * 1e6f)})
    key.push_back(v);
  if (!ctx->tuned) ctx->tuned = new TuneMap();
  BatchRecord* rec = (BatchRecord*)ctx->batch;
  if (!rec || rec->key != key) {
    release_batch(ctx);
    rec = new BatchRecord();
    rec->key = key;
    // workspace: per group the query buffers and the search scratch, per
    // image the back-projection scratch
    int64_t max_hw = 0;
    for (int i = 0; i < n_images; ++i) max_hw = std::max<int64_t>(max_hw, (int64_t)h[i] * w[i] * scale[i] * scale[i]);
    Carver c(nullptr);
    for (auto& g : groups) {
      if (g.images.empty()) continue;
      zoom_dict d = g.ix->dict;
      c.take<float>(g.nq * d->dpad);
      c.take<float>(g.nq);
      c.take<uint64_t>(g.nq * g.ix->L);
      c.take<int32_t>(g.nq * prm->K);
      c.take<float>(g.nq * prm->K);
      c.take<float>(g.nq * prm->K);
      c.take<char>(0);
    }
    // one buffer of blended patches, reused image after image
    int64_t max_patch = 0;
    for (auto& g : groups)
      for (int i : g.images) {
        zoom_dict d = g.ix->dict;
        max_patch = std::max<int64_t>(max_patch, (int64_t)(h[i] - d->P + 1) * (w[i] - d->P + 1) * d->ph2);
      }
    for (int i = 0; i < n_images; ++i) {
      c.take<float>((size_t)h[i] * w[i] * scale[i] * scale[i]);
      c.take<float>((size_t)h[i] * w[i]);
    }
    c.take<float>(max_patch);
    const size_t base_bytes = c.off + 256;
    // the query buffers first (the autotuner needs features and keys)
    rec->bytes = base_bytes;
    rec->mem = zoom_alloc(ctx, rec->bytes, st);
    if (!rec->mem) {
      delete rec;
      return fail(ZOOM_ERR_OOM, "batch workspace");
    }
    Carver m(rec->mem);
    for (auto& g : groups) {
      if (g.images.empty()) continue;
      zoom_dict d = g.ix->dict;
      g.b.feat = m.take<float>(g.nq * d->dpad);
      g.b.mu = m.take<float>(g.nq);
      g.b.norm2 = nullptr;
      g.b.keys = m.take<uint64_t>(g.nq * g.ix->L);
      g.b.nbr = m.take<int32_t>(g.nq * prm->K);
      g.b.dist = m.take<float>(g.nq * prm->K);
      g.b.wgt = m.take<float>(g.nq * prm->K);
      g.b.bucket_sum = nullptr;
      m.take<char>(0);
    }
    std::vector<float*> tmp(n_images), err(n_images);
    for (int i = 0; i < n_images; ++i) {
      tmp[i] = m.take<float>((size_t)h[i] * w[i] * scale[i] * scale[i]);
      err[i] = m.take<float>((size_t)h[i] * w[i]);
    }
    float* patches = m.take<float>(max_patch);
    // features and keys of every image, then one autotuning pass per group
    for (auto& g : groups) {
      zoom_dict d = g.ix->dict;
      for (size_t k = 0; k < g.images.size(); ++k) {
        const int i = g.images[k];
        const int64_t o = g.q_off[k];
        cudaError_t e = launch_query_features(lr[i], h[i], w[i], d->P, d->feature, d->dpad, g.b.feat + o * d->dpad,
                                              g.b.mu + o, nullptr, st);
        const int64_t nqi = (int64_t)(h[i] - d->P + 1) * (w[i] - d->P + 1);
        if (e == cudaSuccess)
          e = launch_hash(g.b.feat + o * d->dpad, d->dpad, d->d, nqi, g.ix->alpha, g.ix->beta, g.ix->L,
                          g.ix->k, g.ix->w, g.b.keys + o * g.ix->L, st);
        if (e != cudaSuccess) {
          free_record(ctx, rec);
          return fail(ZOOM_ERR_CUDA, std::string("batch features: ") + cudaGetErrorString(e));
        }
      }
      if (!g.images.empty() && plan_search(g.ix, prm, g.nq, 0, 0).tc) {
        zoom_status rs = autotune_group(g, prm, st);
        if (rs != ZOOM_OK) {
          free_record(ctx, rec);
          return rs;
        }
      }
    }
    // search scratch per group, with the tuned plan
    size_t extra = 0;
    TuneMap& tm = *(TuneMap*)ctx->tuned;
    for (auto& g : groups) {
      if (g.images.empty()) continue;
      const TuneKey tk{g.ix, qbucket(g.nq), prm->precision, prm->K};
      const TuneChoice ch = tm.count(tk) ? tm[tk] : TuneChoice();
      g.plan = plan_search(g.ix, prm, g.nq, ch.nsplit, ch.mc);
      extra += (g.plan.bytes + 255) / 256 * 256;
    }
    void* ws = extra ? zoom_alloc(ctx, extra, st) : nullptr;
    if (extra && !ws) {
      free_record(ctx, rec);
      return fail(ZOOM_ERR_OOM, "batch search workspace");
    }
    rec->ws = ws;
    rec->ws_bytes = extra;
    {
      char* p = (char*)ws;
      for (auto& g : groups) {
        if (g.images.empty()) continue;
        g.ws = p;
        p += (g.plan.bytes + 255) / 256 * 256;
      }
    }
    // record the whole batch on a private stream into a graph
    ZCHECK_CUDA(cudaStreamCreateWithFlags(&rec->cap, cudaStreamNonBlocking));
    rec->ev.resize(n_images + 1);
    for (auto& e : rec->ev) ZCHECK_CUDA(cudaEventCreate(&e));
    cudaStream_t cs = rec->cap;
    ZCHECK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    // external records become event nodes of the graph (readable timings)
    cudaError_t e = cudaEventRecordWithFlags(rec->ev[0], cs, cudaEventRecordExternal);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_counters, 0, CNT_N * sizeof(unsigned long long), cs);
    for (auto& g : groups) {
      if (g.images.empty() || e != cudaSuccess) continue;
      zoom_dict d = g.ix->dict;
      for (size_t k = 0; k < g.images.size() && e == cudaSuccess; ++k) {
        const int i = g.images[k];
        const int64_t o = g.q_off[k];
        const int64_t nqi = (int64_t)(h[i] - d->P + 1) * (w[i] - d->P + 1);
        e = launch_query_features(lr[i], h[i], w[i], d->P, d->feature, d->dpad, g.b.feat + o * d->dpad, g.b.mu + o,
                                  nullptr, cs);
        if (e == cudaSuccess)
          e = launch_hash(g.b.feat + o * d->dpad, d->dpad, d->d, nqi, g.ix->alpha, g.ix->beta, g.ix->L,
                          g.ix->k, g.ix->w, g.b.keys + o * g.ix->L, cs);
      }
      // one search over the concatenated queries of every image of this scale
      if (e == cudaSuccess) e = run_search_ws(g.ix, prm, g.b, g.nq, g.plan, g.ws, cs);
      if (e == cudaSuccess)
        e = launch_lle(d, g.b.feat, g.nq, g.b.nbr, g.b.dist, prm->K, prm->reg_rel, prm->fp64_cond_threshold,
                       g.b.wgt, ctx->d_counters, cs);
      for (size_t k = 0; k < g.images.size() && e == cudaSuccess; ++k) {
        const int i = g.images[k];
        const int64_t o = g.q_off[k];
        e = launch_overlap_add_staged(g.b.nbr + o * prm->K, g.b.wgt + o * prm->K, g.b.mu + o, d->hr_res,
                                      d->ph2pad, prm->K, h[i], w[i], d->s, d->P, patches, hr[i], cs);
        float* a = hr[i];
        float* bb = tmp[i];
        for (int it = 0; it < prm->bp_iters && e == cudaSuccess; ++it) {
          e = launch_bp_iteration(a, bb, lr[i], err[i], h[i], w[i], d->s, d->blur_sigma, prm->sigma_spatial,
                                  prm->sigma_range, prm->bp_radius, cs);
          std::swap(a, bb);
        }
        if (e == cudaSuccess && a != hr[i])
          e = cudaMemcpyAsync(hr[i], a, (size_t)h[i] * w[i] * d->s * d->s * 4, cudaMemcpyDeviceToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(rec->ev[1 + i], cs, cudaEventRecordExternal);
      }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&rec->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    rec->groups = groups;
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_record(ctx, rec);
      return fail(ZOOM_ERR_CUDA, std::string("batch recording: ") + cudaGetErrorString(e));
    }
    ctx->batch = rec;
  }
  ZCHECK_CUDA(cudaGraphLaunch(rec->exec, st));
  ctx->last_n_queries = 0;
  for (auto& g : rec->groups)
    if (g.ix) ctx->last_n_queries += g.nq;
  if (per_image_ms) {
    ZCHECK_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < n_images; ++i) {
      float ms = 0.f;
      ZCHECK_CUDA(cudaEventElapsedTime(&ms, rec->ev[0], rec->ev[1 + i]));
      per_image_ms[i] = ms;
    }
  }
  return ZOOM_OK;
}

zoom_status zoom_batch_release(zoom_ctx ctx) {
  if (!ctx) return fail(ZOOM_ERR_INVALID_ARG, "NULL context");
  ZCHECK_CUDA(cudaSetDevice(ctx->device));
  zoom_release_batch(ctx);
  return ZOOM_OK;
}

}  // extern "C"
