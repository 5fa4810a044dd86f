// Per-D templates of the exact neighbour search (plain and capped candidate
// walks) and the LLE solve (Sec. 4.2, Eq. 12-13).  Included by the two
// translation units that instantiate them: kernels_query.cu (pixel features,
// D = 9, 25) and kernels_query_grad.cu (gradient features, D = 18, 50).
#pragma once
#include <float.h>
#include <limits.h>

#include "device_common.cuh"
#include "zoom_internal.h"

namespace {

// ---------------------------------------------------------------------------
// Exact K nearest in the candidate set (Sec. 4.2), SIMT FP32.
//
// The candidate set C(q) (entries sharing the query's bin in >= t of the L
// tables) is nearly the whole dictionary at the workloads' bin widths, so
// the dictionary is streamed densely through shared memory and membership
// is tested only for entries that would enter the list.  Order key:
// (not a member, squared distance in FP32 difference form, ID); members thus
// precede every non-member, which pads queries with fewer than K candidates
// by their nearest non-members.  Entries arrive in ascending ID, so a tie in
// distance never displaces an earlier entry.
// ---------------------------------------------------------------------------
struct Cand {
  float d;
  int id;
  int flag;  // 0 member, 1 non-member, 2 empty slot
};

__device__ __forceinline__ bool cand_less(const Cand& a, const Cand& b) {
  if (a.flag != b.flag) return a.flag < b.flag;
  if (a.d != b.d) return a.d < b.d;
  return a.id < b.id;
}

template <int KMAX>
__device__ __forceinline__ void list_insert(Cand (&bl)[KMAX], int K, const Cand& c) {
  bool done = false;
#pragma unroll
  for (int j = KMAX - 1; j > 0; --j) {
    if (j < K && !done) {
      if (cand_less(c, bl[j - 1])) {
        bl[j] = bl[j - 1];
      } else {
        bl[j] = c;
        done = true;
      }
    }
  }
  if (!done) bl[0] = c;
}

template <int KMAX>
__device__ __forceinline__ Cand list_worst(const Cand (&bl)[KMAX], int K) {
  Cand w = bl[0];
#pragma unroll
  for (int j = 1; j < KMAX; ++j)
    if (j == K - 1) w = bl[j];
  return w;
}

constexpr int KNN_THREADS = 128;
constexpr int KNN_TN = 64;

template <int D, int KMAX>
__global__ __launch_bounds__(KNN_THREADS) void k_knn_exact(
    const float* __restrict__ qfeat, int dpad, int64_t nq, const uint64_t* __restrict__ qkeys,
    const float* __restrict__ dfeat, int64_t N, const uint64_t* __restrict__ dkeys, int L, int tmin,
    int K, int32_t* __restrict__ nbr, float* __restrict__ dist,
    unsigned long long* __restrict__ counters, const int32_t* __restrict__ qidx,
    const unsigned long long* __restrict__ qcount) {
  constexpr int DP = (D + 3) / 4 * 4;
  __shared__ __align__(16) float tile[KNN_TN * DP];
  // with qidx, thread i handles query qidx[i] for i < *qcount (queries that
  // another search path could not settle)
  const int64_t slot = (int64_t)blockIdx.x * KNN_THREADS + threadIdx.x;
  int64_t q = slot;
  bool active = q < nq;
  if (qidx) {
    const int64_t cnt = (int64_t)*qcount;
    if ((int64_t)blockIdx.x * KNN_THREADS >= cnt) return;   // whole block idle
    active = slot < cnt;
    q = active ? qidx[slot] : 0;
  }
  float qv[D];
#pragma unroll
  for (int i = 0; i < D; ++i) qv[i] = active ? qfeat[q * dpad + i] : 0.f;
  Cand bl[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) bl[j] = Cand{FLT_MAX, INT_MAX, 2};
  float thr = FLT_MAX;  // fast-path bound: only d < thr can enter the list
  bool thr_inf = true;

  for (int64_t base = 0; base < N; base += KNN_TN) {
    const int nt = (int)((N - base) < KNN_TN ? (N - base) : KNN_TN);
    __syncthreads();
    for (int t = threadIdx.x; t < nt * (DP / 4); t += KNN_THREADS) {
      int r = t / (DP / 4), c4 = t % (DP / 4);
      reinterpret_cast<float4*>(tile)[t] =
          reinterpret_cast<const float4*>(dfeat + (base + r) * dpad)[c4];
    }
    __syncthreads();
    if (!active) continue;
    for (int c = 0; c < nt; ++c) {
      const float* cv = tile + c * DP;
      float dd = 0.f;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        float df = qv[i] - cv[i];
        dd = fmaf(df, df, dd);
      }
      if (thr_inf || dd < thr) {
        const int64_t id = base + c;
        int hits = 0;
        for (int l = 0; l < L; ++l) hits += (qkeys[q * L + l] == dkeys[id * L + l]) ? 1 : 0;
        Cand cd{dd, (int)id, hits >= tmin ? 0 : 1};
        Cand wst = list_worst<KMAX>(bl, K);
        if (cand_less(cd, wst)) {
          list_insert<KMAX>(bl, K, cd);
          wst = list_worst<KMAX>(bl, K);
          thr_inf = wst.flag != 0;
          thr = wst.d;
        }
      }
    }
  }
  if (!active) return;
  int npad = 0;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < K) {
      nbr[q * K + j] = bl[j].id;
      dist[q * K + j] = bl[j].d;
      npad += bl[j].flag != 0 ? 1 : 0;
    }
  }
  if (npad > 0) atomicAdd(&counters[CNT_PADDED], 1ull);
  if (npad == K) atomicAdd(&counters[CNT_EMPTY], 1ull);
}

// ---------------------------------------------------------------------------
// Candidate set under the cap (the early stop of Sec. 4.2): the tables are
// visited in order l = 0..L-1, each bin in ascending ID, and the first `cap`
// distinct IDs form C(q); the K nearest of them in FP32 difference form,
// ties by ID.  One thread per query; the collected IDs live in global
// scratch [nq][cap].  A query with fewer than K candidates (its bins hold
// fewer than K distinct IDs, cap >= K) is flagged: the SIMT scan then pads
// it with the nearest entries outside its bins.
// ---------------------------------------------------------------------------
template <int D, int KMAX>
__global__ __launch_bounds__(128) void k_knn_capped(
    const float* __restrict__ qfeat, int dpad, int64_t nq, const uint64_t* __restrict__ qkeys,
    const float* __restrict__ dfeat, int64_t N, int L, const uint64_t* __restrict__ ukeys,
    const int32_t* __restrict__ offs, const int32_t* __restrict__ ids, const int32_t* __restrict__ nuniq,
    int cap, int K, int32_t* __restrict__ nbr, float* __restrict__ dist, int32_t* __restrict__ cand,
    int32_t* __restrict__ fb_list, unsigned long long* __restrict__ fb_count) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  int32_t* cs = cand + q * cap;
  int nc = 0;
  for (int l = 0; l < L && nc < cap; ++l) {
    const uint64_t key = qkeys[q * L + l];
    const uint64_t* uk = ukeys + (int64_t)l * N;
    int lo = 0, hi = nuniq[l];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (uk[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= nuniq[l] || uk[lo] != key) continue;
    const int32_t* off = offs + (int64_t)l * (N + 1);
    const int32_t* bin = ids + (int64_t)l * N;
    const int nprev = nc;   // IDs of earlier tables; a bin holds distinct IDs
    for (int p = off[lo]; p < off[lo + 1] && nc < cap; ++p) {
      const int id = bin[p];
      bool seen = false;
      for (int j = 0; j < nprev && !seen; ++j) seen = cs[j] == id;
      if (!seen) cs[nc++] = id;
    }
  }
  if (nc < K) {
    const unsigned long long slot = atomicAdd(fb_count, 1ull);
    fb_list[slot] = (int32_t)q;
    return;
  }
  float qv[D];
#pragma unroll
  for (int i = 0; i < D; ++i) qv[i] = qfeat[q * dpad + i];
  Cand bl[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) bl[j] = Cand{FLT_MAX, INT_MAX, 2};
  for (int j = 0; j < nc; ++j) {
    const int id = cs[j];
    float dd = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float df = qv[i] - dfeat[(int64_t)id * dpad + i];
      dd = fmaf(df, df, dd);
    }
    const Cand cd{dd, id, 0};
    if (cand_less(cd, list_worst<KMAX>(bl, K))) list_insert<KMAX>(bl, K, cd);
  }
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < K) {
      nbr[q * K + j] = bl[j].id;
      dist[q * K + j] = bl[j].d;
    }
}

// ---------------------------------------------------------------------------
// LLE weights (Eq. 12-13): G = Z Z^T over the K neighbours, C = G + eps I,
// eps = reg_rel * trace(G), Cholesky, C z = 1, w = z / sum(z).  One thread
// per query.  FP64 when the condition bound (trace + eps) / eps exceeds the
// threshold or an FP32 pivot is not positive.  A query at distance exactly 0
// from its first neighbour gets the one-hot weight.
// ---------------------------------------------------------------------------
template <typename T, int KMAX>
__device__ __forceinline__ bool chol_solve(T (&C)[KMAX][KMAX], int K, T (&z)[KMAX]) {
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < K) {
      T s = C[j][j];
#pragma unroll
      for (int m = 0; m < j; ++m) s -= C[j][m] * C[j][m];
      if (!(s > T(0))) return false;
      T ljj = sqrt(s);
      C[j][j] = ljj;
#pragma unroll
      for (int i = j + 1; i < KMAX; ++i) {
        if (i < K) {
          T t = C[i][j];
#pragma unroll
          for (int m = 0; m < j; ++m) t -= C[i][m] * C[j][m];
          C[i][j] = t / ljj;
        }
      }
    }
  }
  T u[KMAX];
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    if (i < K) {
      T t = T(1);
#pragma unroll
      for (int m = 0; m < i; ++m) t -= C[i][m] * u[m];
      u[i] = t / C[i][i];
    }
  }
#pragma unroll
  for (int i = KMAX - 1; i >= 0; --i) {
    if (i < K) {
      T t = u[i];
#pragma unroll
      for (int m = i + 1; m < KMAX; ++m)
        if (m < K) t -= C[m][i] * z[m];
      z[i] = t / C[i][i];
    }
  }
  return true;
}

template <int D, int KMAX>
__global__ __launch_bounds__(128) void k_lle(const float* __restrict__ qfeat, int dpad, int64_t nq,
                                             const float* __restrict__ dfeat,
                                             const int32_t* __restrict__ nbr,
                                             const float* __restrict__ dist, int K, float reg_rel,
                                             double cond_thr, float* __restrict__ wgt,
                                             unsigned long long* __restrict__ counters) {
  int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  if (dist[q * K] == 0.f) {
    for (int j = 0; j < K; ++j) wgt[q * K + j] = j == 0 ? 1.f : 0.f;
    atomicAdd(&counters[CNT_EXACT], 1ull);
    return;
  }
  int id[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) id[j] = j < K ? nbr[q * K + j] : 0;
  float G[KMAX][KMAX];
#pragma unroll
  for (int a = 0; a < KMAX; ++a)
#pragma unroll
    for (int b = 0; b < KMAX; ++b) G[a][b] = 0.f;
  for (int i = 0; i < D; ++i) {
    float qi = qfeat[q * dpad + i];
    float z[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) z[j] = j < K ? qi - dfeat[(int64_t)id[j] * dpad + i] : 0.f;
#pragma unroll
    for (int a = 0; a < KMAX; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b) G[a][b] = fmaf(z[a], z[b], G[a][b]);
  }
  float tr = 0.f;
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < K) tr += G[j][j];
  const float eps = reg_rel * tr;
  const double cond = ((double)tr + (double)eps) / (double)eps;
  float w[KMAX];
  bool ok = false;
  if (cond <= cond_thr) {
    float C[KMAX][KMAX];
#pragma unroll
    for (int a = 0; a < KMAX; ++a)
#pragma unroll
      for (int b = 0; b < KMAX; ++b) C[a][b] = (b <= a ? G[a][b] : G[b][a]) + (a == b ? eps : 0.f);
    float z[KMAX];
    ok = chol_solve<float, KMAX>(C, K, z);
    if (ok) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < K) s += z[j];
#pragma unroll
      for (int j = 0; j < KMAX; ++j) w[j] = z[j] / s;
    }
  }
  if (!ok) {
    // FP64 Gram and Cholesky from the FP32 features
    double Gd[KMAX][KMAX];
#pragma unroll
    for (int a = 0; a < KMAX; ++a)
#pragma unroll
      for (int b = 0; b < KMAX; ++b) Gd[a][b] = 0.0;
    for (int i = 0; i < D; ++i) {
      double qi = qfeat[q * dpad + i];
      double z[KMAX];
#pragma unroll
      for (int j = 0; j < KMAX; ++j) z[j] = j < K ? qi - (double)dfeat[(int64_t)id[j] * dpad + i] : 0.0;
#pragma unroll
      for (int a = 0; a < KMAX; ++a)
#pragma unroll
        for (int b = 0; b < KMAX; ++b) Gd[a][b] += z[a] * z[b];
    }
    double trd = 0.0;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < K) trd += Gd[j][j];
    const double epsd = (double)reg_rel * trd;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) Gd[j][j] += epsd;
    double zd[KMAX];
    bool okd = chol_solve<double, KMAX>(Gd, K, zd);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
      if (j < K) s += okd ? zd[j] : 1.0;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) w[j] = (float)((okd ? zd[j] : 1.0) / s);
    atomicAdd(&counters[CNT_FP64], 1ull);
  }
  for (int j = 0; j < K; ++j) wgt[q * K + j] = w[j];
}

template <int D>
cudaError_t knn_dispatch_k(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq,
                           int K, int32_t* nbr, float* dist, unsigned long long* counters,
                           const int32_t* qidx, const unsigned long long* qcount, cudaStream_t st) {
  zoom_dict d = ix->dict;
  int blocks = (int)((nq + KNN_THREADS - 1) / KNN_THREADS);
  // under the cap the candidate rule ignores t (only capped queries whose
  // bins hold fewer than K IDs come here: their candidates are the union)
  const int tmin = ix->cap > 0 ? 1 : ix->t;
  if (K <= 8)
    k_knn_exact<D, 8><<<blocks, KNN_THREADS, 0, st>>>(qfeat, d->dpad, nq, qkeys, d->feat, d->n,
                                                     ix->dkeys, ix->L, tmin, K, nbr, dist,
                                                     counters, qidx, qcount);
  else
    k_knn_exact<D, 16><<<blocks, KNN_THREADS, 0, st>>>(qfeat, d->dpad, nq, qkeys, d->feat, d->n,
                                                      ix->dkeys, ix->L, tmin, K, nbr, dist,
                                                      counters, qidx, qcount);
  return cudaGetLastError();
}

template <int D>
cudaError_t capped_dispatch_k(zoom_index ix, const float* qfeat, const uint64_t* qkeys, int64_t nq, int K,
                              int32_t* nbr, float* dist, int32_t* cand, int32_t* fb,
                              unsigned long long* fb_count, cudaStream_t st) {
  zoom_dict d = ix->dict;
  const int blocks = (int)((nq + 127) / 128);
  if (K <= 8)
    k_knn_capped<D, 8><<<blocks, 128, 0, st>>>(qfeat, d->dpad, nq, qkeys, d->feat, d->n, ix->L, ix->ukeys,
                                               ix->offs, ix->ids, ix->nuniq, ix->cap, K, nbr, dist, cand,
                                               fb, fb_count);
  else
    k_knn_capped<D, 16><<<blocks, 128, 0, st>>>(qfeat, d->dpad, nq, qkeys, d->feat, d->n, ix->L, ix->ukeys,
                                                ix->offs, ix->ids, ix->nuniq, ix->cap, K, nbr, dist, cand,
                                                fb, fb_count);
  return cudaGetLastError();
}

template <int D>
cudaError_t lle_dispatch_k(zoom_dict d, const float* qfeat, int64_t nq, const int32_t* nbr,
                           const float* dist, int K, float reg_rel, double cond_thr, float* wgt,
                           unsigned long long* counters, cudaStream_t st) {
  int blocks = (int)((nq + 127) / 128);
  if (K <= 8)
    k_lle<D, 8><<<blocks, 128, 0, st>>>(qfeat, d->dpad, nq, d->feat, nbr, dist, K, reg_rel,
                                        cond_thr, wgt, counters);
  else
    k_lle<D, 16><<<blocks, 128, 0, st>>>(qfeat, d->dpad, nq, d->feat, nbr, dist, K, reg_rel,
                                         cond_thr, wgt, counters);
  return cudaGetLastError();
}

}  // namespace
