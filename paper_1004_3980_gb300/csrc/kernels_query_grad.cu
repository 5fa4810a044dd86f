// Exact neighbour search and LLE weights for the gradient features of
// Sec. 4.1 (D = 2 P^2: 18 for 3 x 3 patches, 50 for 5 x 5), in a translation
// unit of their own so that the build compiles them in parallel with the
// pixel-feature instantiations.
#include "knn_kernels.cuh"

cudaError_t launch_knn_exact_grad(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq,
                                  int K, int32_t* nbr, float* dist, unsigned long long* counters,
                                  const int32_t* qidx, const unsigned long long* qcount, cudaStream_t st) {
  if (ix->dict->d == 18)
    return knn_dispatch_k<18>(ix, qfeat, qkeys, nq, K, nbr, dist, counters, qidx, qcount, st);
  if (ix->dict->d == 50)
    return knn_dispatch_k<50>(ix, qfeat, qkeys, nq, K, nbr, dist, counters, qidx, qcount, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_knn_capped_grad(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq,
                                   int K, int32_t* nbr, float* dist, int32_t* cand, int32_t* fb,
                                   unsigned long long* fb_count, cudaStream_t st) {
  if (ix->dict->d == 18)
    return capped_dispatch_k<18>(ix, qfeat, qkeys, nq, K, nbr, dist, cand, fb, fb_count, st);
  if (ix->dict->d == 50)
    return capped_dispatch_k<50>(ix, qfeat, qkeys, nq, K, nbr, dist, cand, fb, fb_count, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_lle_grad(zoom_dict d, const float* qfeat, int64_t nq, const int32_t* nbr,
                            const float* dist, int K, float reg_rel, double cond_thr, float* wgt,
                            unsigned long long* counters, cudaStream_t st) {
  if (d->d == 18) return lle_dispatch_k<18>(d, qfeat, nq, nbr, dist, K, reg_rel, cond_thr, wgt, counters, st);
  if (d->d == 50) return lle_dispatch_k<50>(d, qfeat, nq, nbr, dist, K, reg_rel, cond_thr, wgt, counters, st);
  return cudaErrorInvalidValue;
}
