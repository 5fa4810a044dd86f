// C ABI of the differentiation entry points: degradation and its adjoint,
// reconstruction with a caller-supplied HR dictionary and its adjoint, and
// the MAP energy with its gradients (Sec. 4, Eq. 5-9).
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "zoom_internal.h"

namespace {

zoom_status fail(zoom_status s, const std::string& m) {
  zoom_set_error(m);
  return s;
}

#define ZB_CUDA(expr)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) return fail(ZOOM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Buf {
  zoom_ctx ctx;
  cudaStream_t st;
  void* p = nullptr;
  size_t bytes = 0;
  Buf(zoom_ctx c, cudaStream_t s) : ctx(c), st(s) {}
  ~Buf() {
    if (p) zoom_free(ctx, p, bytes, st);
  }
  bool get(size_t b) {
    bytes = b;
    p = zoom_alloc(ctx, b, st);
    return p != nullptr || b == 0;
  }
};

struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* r = base ? (T*)(base + off) : nullptr;
    off += n * sizeof(T);
    return r;
  }
};

bool bad_image(zoom_dict d, int h, int w) { return h < d->P || w < d->P; }

// Gradient of the reconstruction with respect to the HR dictionary (and mu)
// given the per-patch gradients gP [nq][ph2]: grad_R[id] = sum over uses of
// w * gP, via the uses sorted by entry ID (deterministic, no atomics).
zoom_status dict_grad_from_patches(zoom_dict d, const int32_t* nbr, const float* wgt, int64_t nq, int K,
                                   const float* gP, float* grad_dict, int grad_stride, char* scratch,
                                   size_t scratch_bytes, cudaStream_t st) {
  const int64_t nu = nq * K;
  Carve c(scratch);
  int32_t* sorted = c.take<int32_t>(nu);
  uint64_t* ukeys = c.take<uint64_t>(nu);
  int32_t* offs = c.take<int32_t>(nu + 1);
  int32_t* nuniq = c.take<int32_t>(1);
  char* rest = c.take<char>(0);
  const size_t used = (size_t)(rest - scratch);
  if (used > scratch_bytes) return fail(ZOOM_ERR_OOM, "dictionary-gradient scratch");
  ZB_CUDA(cudaMemsetAsync(grad_dict, 0, (size_t)d->n * grad_stride * sizeof(float), st));
  ZB_CUDA(sort_keys_csr(nbr, nu, sorted, ukeys, offs, nuniq, rest, scratch_bytes - used, st));
  ZB_CUDA(launch_dict_grad(sorted, offs, ukeys, nuniq, std::min<int64_t>(nu, d->n), wgt, gP, K, d->ph2,
                           grad_stride, grad_dict, st));
  return ZOOM_OK;
}

size_t dict_grad_scratch(int64_t nu) {
  return (size_t)nu * 4 + (size_t)nu * 8 + (size_t)(nu + 1) * 4 + 4 + 4 * 256 + csr_scratch_bytes(nu);
}

}  // namespace

extern "C" {

zoom_status zoom_degrade(zoom_ctx ctx, const zoom_degradation* degr, const float* hr, int32_t H, int32_t W,
                         float* lr, void* stream) {
  if (!ctx || !degr || !hr || !lr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  if (degr->scale < 1 || degr->scale > 4 || !(degr->blur_sigma > 0.0))
    return fail(ZOOM_ERR_INVALID_ARG, "bad degradation");
  if (H < degr->scale || W < degr->scale) return fail(ZOOM_ERR_INVALID_ARG, "image smaller than one LR pixel");
  ZB_CUDA(cudaSetDevice(ctx->device));
  ZB_CUDA(launch_degrade(hr, H, W, degr->scale, degr->blur_sigma, nullptr, lr, (cudaStream_t)stream));
  return ZOOM_OK;
}

zoom_status zoom_degrade_adjoint(zoom_ctx ctx, const zoom_degradation* degr, const float* g_lr, int32_t h,
                                 int32_t w, float* g_hr, void* stream) {
  if (!ctx || !degr || !g_lr || !g_hr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  if (degr->scale < 1 || degr->scale > 4 || !(degr->blur_sigma > 0.0))
    return fail(ZOOM_ERR_INVALID_ARG, "bad degradation");
  if (h < 1 || w < 1) return fail(ZOOM_ERR_INVALID_ARG, "empty image");
  ZB_CUDA(cudaSetDevice(ctx->device));
  const int s = degr->scale;
  ZB_CUDA(launch_degrade_adjoint(g_lr, h, w, s * h, s * w, s, degr->blur_sigma, 1.f, g_hr,
                                 (cudaStream_t)stream));
  return ZOOM_OK;
}

zoom_status zoom_reconstruct_with(zoom_index ix, const float* hr_res, int32_t hr_stride, const int32_t* nbr,
                                  const float* wgt, const float* mu, int32_t h, int32_t w, int32_t K,
                                  float* hr, void* stream) {
  if (!ix || !hr_res || !nbr || !wgt || !mu || !hr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  zoom_dict d = ix->dict;
  if (bad_image(d, h, w)) return fail(ZOOM_ERR_INVALID_ARG, "image smaller than one patch");
  if (K < 1 || K > 64) return fail(ZOOM_ERR_INVALID_ARG, "K must be in 1..64");
  if (hr_stride < d->ph2) return fail(ZOOM_ERR_INVALID_ARG, "hr_stride smaller than the HR patch size");
  ZB_CUDA(cudaSetDevice(d->ctx->device));
  ZB_CUDA(launch_overlap_add(nbr, wgt, mu, hr_res, hr_stride, K, h, w, d->s, d->P, hr, (cudaStream_t)stream));
  return ZOOM_OK;
}

zoom_status zoom_reconstruct_adjoint(zoom_index ix, const int32_t* nbr, const float* wgt, int32_t h, int32_t w,
                                     int32_t K, const float* grad_hr, float* grad_dict, int32_t grad_stride,
                                     float* grad_mu, void* stream) {
  if (!ix || !nbr || !wgt || !grad_hr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  zoom_dict d = ix->dict;
  if (bad_image(d, h, w)) return fail(ZOOM_ERR_INVALID_ARG, "image smaller than one patch");
  if (K < 1 || K > 64) return fail(ZOOM_ERR_INVALID_ARG, "K must be in 1..64");
  if (grad_dict && grad_stride < d->ph2) return fail(ZOOM_ERR_INVALID_ARG, "grad_stride too small");
  cudaStream_t st = (cudaStream_t)stream;
  ZB_CUDA(cudaSetDevice(d->ctx->device));
  const int64_t nq = (int64_t)(h - d->P + 1) * (w - d->P + 1);
  Buf b(d->ctx, st);
  const size_t gpb = (size_t)nq * d->ph2 * 4 + 256;
  const size_t dgs = grad_dict ? dict_grad_scratch(nq * K) : 0;
  if (!b.get(gpb + dgs + 256)) return fail(ZOOM_ERR_OOM, "adjoint scratch");
  Carve c(b.p);
  float* gP = c.take<float>((size_t)nq * d->ph2);
  char* rest = c.take<char>(0);
  ZB_CUDA(launch_patch_grad(grad_hr, nullptr, h, w, d->s, d->P, 0.f, gP, st));
  if (grad_dict) {
    zoom_status rc = dict_grad_from_patches(d, nbr, wgt, nq, K, gP, grad_dict, grad_stride, rest,
                                            b.bytes - (size_t)(rest - (char*)b.p), st);
    if (rc != ZOOM_OK) return rc;
  }
  if (grad_mu) ZB_CUDA(launch_mu_grad(gP, nq, d->ph2, grad_mu, st));
  return ZOOM_OK;
}

zoom_status zoom_backward(zoom_index ix, const float* lr, int32_t h, int32_t w, const int32_t* nbr,
                          const float* wgt, int32_t K, float reg_rel, float lambda, float* grad_x,
                          float* grad_dict, int32_t grad_stride, float* hr_out, double* energy,
                          void* stream) {
  if (!ix || !lr || !nbr) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  zoom_dict d = ix->dict;
  if (bad_image(d, h, w)) return fail(ZOOM_ERR_INVALID_ARG, "image smaller than one patch");
  if (K < 1 || K > 16) return fail(ZOOM_ERR_INVALID_ARG, "K must be in 1..16");
  if (!(lambda >= 0.f) || !(reg_rel >= 0.f)) return fail(ZOOM_ERR_INVALID_ARG, "lambda and reg_rel must be >= 0");
  if (grad_dict && grad_stride < d->ph2) return fail(ZOOM_ERR_INVALID_ARG, "grad_stride too small");
  cudaStream_t st = (cudaStream_t)stream;
  zoom_ctx ctx = d->ctx;
  ZB_CUDA(cudaSetDevice(ctx->device));
  const int s = d->s;
  const int64_t nq = (int64_t)(h - d->P + 1) * (w - d->P + 1);
  const int64_t hr_n = (int64_t)s * h * s * w;
  const int nblocks = 256;
  Carve sz(nullptr);
  sz.take<float>(nq * d->dpad);
  sz.take<float>(nq);
  sz.take<float>(nq * K);
  sz.take<float>(nq * K);
  sz.take<float>(nq * d->ph2);
  sz.take<float>(hr_n);
  sz.take<float>((size_t)h * w);
  sz.take<float>(hr_n);
  sz.take<float>(nq * d->ph2);
  sz.take<double>(2 * nblocks);
  const size_t dgs = grad_dict ? dict_grad_scratch(nq * K) : 0;
  Buf b(ctx, st);
  if (!b.get(sz.off + dgs + 512)) return fail(ZOOM_ERR_OOM, "backward scratch");
  Carve c(b.p);
  float* qfeat = c.take<float>(nq * d->dpad);
  float* mu = c.take<float>(nq);
  float* dist = c.take<float>(nq * K);
  float* wloc = c.take<float>(nq * K);
  float* P = c.take<float>(nq * d->ph2);
  float* x = hr_out ? (c.take<float>(hr_n), hr_out) : c.take<float>(hr_n);
  float* r = c.take<float>((size_t)h * w);
  float* gx = grad_x ? (c.take<float>(hr_n), grad_x) : c.take<float>(hr_n);
  float* gP = c.take<float>(nq * d->ph2);
  double* part = c.take<double>(2 * nblocks);
  char* rest = c.take<char>(0);
  // weights: given, or recomputed from the neighbours (Eq. 12-13)
  ZB_CUDA(launch_query_features(lr, h, w, d->P, d->feature, d->dpad, qfeat, mu, nullptr, st));
  const float* wv = wgt;
  if (!wv) {
    ZB_CUDA(launch_nbr_dist(qfeat, d->dpad, d->d, nq, d->feat, nbr, K, dist, st));
    ZB_CUDA(launch_lle(d, qfeat, nq, nbr, dist, K, reg_rel, 1e6, wloc, ctx->d_counters, st));
    wv = wloc;
  }
  // forward: patches, overlap average, residual of the data term
  ZB_CUDA(launch_patches(nbr, wv, mu, d->hr_res, d->ph2pad, K, nq, d->ph2, P, st));
  ZB_CUDA(launch_overlap_add(nbr, wv, mu, d->hr_res, d->ph2pad, K, h, w, s, d->P, x, st));
  ZB_CUDA(launch_degrade(x, s * h, s * w, s, d->blur_sigma, lr, r, st));
  // d/dx of ||D B x - y||^2
  ZB_CUDA(launch_degrade_adjoint(r, h, w, s * h, s * w, s, d->blur_sigma, 2.f, gx, st));
  if (grad_dict) {
    ZB_CUDA(launch_patch_grad(gx, P, h, w, s, d->P, lambda, gP, st));
    zoom_status rc = dict_grad_from_patches(d, nbr, wv, nq, K, gP, grad_dict, grad_stride, rest,
                                            b.bytes - (size_t)(rest - (char*)b.p), st);
    if (rc != ZOOM_OK) return rc;
  }
  if (energy) {
    ZB_CUDA(launch_energy_partials(r, (int64_t)h * w, P, h, w, s, d->P, part, nblocks, st));
    std::vector<double> hp(2 * nblocks);
    ZB_CUDA(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ZB_CUDA(cudaStreamSynchronize(st));
    double e_data = 0.0, e_prior = 0.0;
    for (int i = 0; i < nblocks; ++i) e_data += hp[i];
    for (int i = 0; i < nblocks; ++i) e_prior += hp[nblocks + i];
    *energy = e_data + (double)lambda * e_prior;
  }
  return ZOOM_OK;
}

}  // extern "C"
