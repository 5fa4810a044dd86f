// Per-patch inference steps (Sec. 4.1-4.2): query features, bin lookup,
// exact K-nearest selection over the hashed candidate set, LLE weights.
#include <float.h>
#include <limits.h>

#include "device_common.cuh"
#include "knn_kernels.cuh"
#include "zoom_internal.h"

namespace {

// ---------------------------------------------------------------------------
// query features: every P x P patch of the LR image at stride 1, row order;
// F = 0 pixels minus their mean, F = 1, 2 first- or second-order gradients
// (Sec. 4.1)
// ---------------------------------------------------------------------------
template <int P, int F>
__global__ void k_query_features(const float* __restrict__ lr, int h, int w, int dpad,
                                 float* __restrict__ feat, float* __restrict__ mu,
                                 float* __restrict__ norm2) {
  constexpr int P2 = P * P;
  constexpr int D = zoom_feature_dim(P, F);
  const int nw = w - P + 1;
  const int64_t nq = (int64_t)(h - P + 1) * nw;
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  int i = (int)(q / nw), j = (int)(q % nw);
  float px[P2], v[P2], m, n2;
#pragma unroll
  for (int a = 0; a < P; ++a)
#pragma unroll
    for (int b = 0; b < P; ++b) px[a * P + b] = lr[(size_t)(i + a) * w + j + b];
  zoom_patch_feature<P2>(px, v, m, n2);
  if constexpr (F == 0) {
    for (int t = 0; t < dpad; ++t) feat[q * dpad + t] = t < D ? v[t] : 0.f;
  } else {
    float g[D];
    zoom_gradient_feature<P, F>(lr, h, w, (size_t)w, i, j, g, n2);
    for (int t = 0; t < dpad; ++t) feat[q * dpad + t] = t < D ? g[t] : 0.f;
  }
  mu[q] = m;
  if (norm2) norm2[q] = n2;
}

// ---------------------------------------------------------------------------
// bin lookup: binary search of each table's query key among its bin keys
// ---------------------------------------------------------------------------
__global__ void k_bucket_lookup(const uint64_t* __restrict__ qkeys, int64_t nq, int L,
                                const uint64_t* __restrict__ ukeys, const int32_t* __restrict__ offs,
                                const int32_t* __restrict__ nuniq, int64_t N,
                                int32_t* __restrict__ bucket_sum,
                                unsigned long long* __restrict__ counters) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = 0;
  if (q < nq) {
    for (int l = 0; l < L; ++l) {
      const uint64_t key = qkeys[q * L + l];
      const uint64_t* uk = ukeys + (int64_t)l * N;
      int lo = 0, hi = nuniq[l];
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (uk[mid] < key) lo = mid + 1; else hi = mid;
      }
      if (lo < nuniq[l] && uk[lo] == key) {
        const int32_t* of = offs + (int64_t)l * (N + 1);
        tot += of[lo + 1] - of[lo];
      }
    }
    if (bucket_sum) bucket_sum[q] = (int32_t)tot;
  }
  // one atomic per warp (a per-query atomic on one address serialised the
  // kernel): a query's sum is below L * 2^30, a warp's sum below 2^64
  const unsigned long long s = (unsigned long long)tot;
  unsigned long long ws = s, wm = s;
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    ws += __shfl_xor_sync(0xffffffffu, ws, off);
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, wm, off);
    wm = o > wm ? o : wm;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&counters[CNT_BUCKET_SUM], ws);
    atomicMax(&counters[CNT_BUCKET_MAX], wm);
  }
}

}  // namespace

cudaError_t launch_query_features(const float* lr, int h, int w, int P, int F, int dpad, float* feat,
                                  float* mu, float* norm2, cudaStream_t st) {
  int64_t nq = (int64_t)(h - P + 1) * (w - P + 1);
  int blocks = (int)((nq + 127) / 128);
  if (P == 3 && F == 0)
    k_query_features<3, 0><<<blocks, 128, 0, st>>>(lr, h, w, dpad, feat, mu, norm2);
  else if (P == 5 && F == 0)
    k_query_features<5, 0><<<blocks, 128, 0, st>>>(lr, h, w, dpad, feat, mu, norm2);
  else if (P == 3 && F == 1)
    k_query_features<3, 1><<<blocks, 128, 0, st>>>(lr, h, w, dpad, feat, mu, norm2);
  else if (P == 5 && F == 1)
    k_query_features<5, 1><<<blocks, 128, 0, st>>>(lr, h, w, dpad, feat, mu, norm2);
  else if (P == 3 && F == 2)
    k_query_features<3, 2><<<blocks, 128, 0, st>>>(lr, h, w, dpad, feat, mu, norm2);
  else if (P == 5 && F == 2)
    k_query_features<5, 2><<<blocks, 128, 0, st>>>(lr, h, w, dpad, feat, mu, norm2);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_bucket_lookup(zoom_index ix, const uint64_t* qkeys, int64_t nq,
                                 int32_t* bucket_sum, unsigned long long* counters,
                                 cudaStream_t st) {
  int blocks = (int)((nq + 127) / 128);
  k_bucket_lookup<<<blocks, 128, 0, st>>>(qkeys, nq, ix->L, ix->ukeys, ix->offs, ix->nuniq,
                                          ix->dict->n, bucket_sum, counters);
  return cudaGetLastError();
}

cudaError_t launch_knn_exact(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq,
                             int K, int32_t* nbr, float* dist, unsigned long long* counters,
                             const int32_t* qidx, const unsigned long long* qcount,
                             cudaStream_t st) {
  if (ix->dict->d == 9)
    return knn_dispatch_k<9>(ix, qfeat, qkeys, nq, K, nbr, dist, counters, qidx, qcount, st);
  if (ix->dict->d == 25)
    return knn_dispatch_k<25>(ix, qfeat, qkeys, nq, K, nbr, dist, counters, qidx, qcount, st);
  return launch_knn_exact_grad(ix, qfeat, qkeys, nq, K, nbr, dist, counters, qidx, qcount, st);
}

cudaError_t launch_knn_capped(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq, int K,
                              int32_t* nbr, float* dist, int32_t* cand, int32_t* fb,
                              unsigned long long* fb_count, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  if (ix->dict->d == 9) return capped_dispatch_k<9>(ix, qfeat, qkeys, nq, K, nbr, dist, cand, fb, fb_count, st);
  if (ix->dict->d == 25)
    return capped_dispatch_k<25>(ix, qfeat, qkeys, nq, K, nbr, dist, cand, fb, fb_count, st);
  return launch_knn_capped_grad(ix, qfeat, qkeys, nq, K, nbr, dist, cand, fb, fb_count, st);
}

cudaError_t launch_lle(zoom_dict d, const float* qfeat, int64_t nq, const int32_t* nbr,
                       const float* dist, int K, float reg_rel, double cond_thr, float* wgt,
                       unsigned long long* counters, cudaStream_t st) {
  if (d->d == 9)
    return lle_dispatch_k<9>(d, qfeat, nq, nbr, dist, K, reg_rel, cond_thr, wgt, counters, st);
  if (d->d == 25)
    return lle_dispatch_k<25>(d, qfeat, nq, nbr, dist, K, reg_rel, cond_thr, wgt, counters, st);
  return launch_lle_grad(d, qfeat, nq, nbr, dist, K, reg_rel, cond_thr, wgt, counters, st);
}
