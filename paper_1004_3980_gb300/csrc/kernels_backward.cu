// Adjoint (backward) kernels of the reconstruction and of the degradation,
// and the MAP energy of Sec. 4 (Eq. 5, 8, 9): with the neighbour IDs and
// weights held fixed,
//   E(R) = || D B x - y ||^2 + lambda * sum_{4-neighbour patches p,q} ||P_p - P_q||^2_overlap,
//   x = overlap average of the patches P_n = mu_n + sum_m w_nm R[nbr_nm].
// All reductions are deterministic (fixed order, no atomics on values).
#include <math.h>

#include "device_common.cuh"
#include "zoom_internal.h"

namespace {

// P[n][p] = mu_n + sum_m w_nm R[nbr_nm][p]; one thread per (patch, pixel).
__global__ void k_patches(const int32_t* __restrict__ nbr, const float* __restrict__ wgt,
                          const float* __restrict__ mu, const float* __restrict__ hr_res, int ph2pad,
                          int K, int64_t nq, int ph2, float* __restrict__ P) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * ph2) return;
  const int64_t n = t / ph2;
  const int p = (int)(t % ph2);
  float v = mu[n];
  for (int m = 0; m < K; ++m) v = fmaf(wgt[n * K + m], hr_res[(int64_t)nbr[n * K + m] * ph2pad + p], v);
  P[t] = v;
}

// 1-D weights of the blur + s-box decimation (see the forward kernels).
struct Wts {
  int n;
  float w[8];
};

// y = D B x (- sub): FP32, separable, clamped.
__global__ void k_degrade(const float* __restrict__ x, int H, int W, int h, int w, int s, Wts wt,
                          const float* __restrict__ sub, float* __restrict__ y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= h || j >= w) return;
  float acc = 0.f;
  for (int a = 0; a < wt.n; ++a) {
    const int r = zoom_clampi(s * i + a - 1, 0, H - 1);
    float row = 0.f;
    for (int b = 0; b < wt.n; ++b) row = fmaf(wt.w[b], x[(int64_t)r * W + zoom_clampi(s * j + b - 1, 0, W - 1)], row);
    acc = fmaf(wt.w[a], row, acc);
  }
  y[(int64_t)i * w + j] = sub ? acc - sub[(int64_t)i * w + j] : acc;
}

// g = alpha * B^T D^T r in gather form: HR pixel (Y, X) collects, from every
// LR pixel (i, j) whose window reads it (through the clamp), the weights
// W_a(i -> Y) W_b(j -> X) times r(i, j).
__global__ void k_degrade_adjoint(const float* __restrict__ r, int h, int w, int H, int W, int s, Wts wt,
                                  float alpha, float* __restrict__ g) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= W || Y >= H) return;
  // LR rows whose window [s*i - 1, s*i + s] (clamped) contains Y
  const int i0 = max(0, (Y - s) / s - 1), i1 = min(h - 1, (Y + 1) / s + 1);
  const int j0 = max(0, (X - s) / s - 1), j1 = min(w - 1, (X + 1) / s + 1);
  float acc = 0.f;
  for (int i = i0; i <= i1; ++i) {
    float wy = 0.f;
    for (int a = 0; a < wt.n; ++a)
      if (zoom_clampi(s * i + a - 1, 0, H - 1) == Y) wy += wt.w[a];
    if (wy == 0.f) continue;
    float row = 0.f;
    for (int j = j0; j <= j1; ++j) {
      float wx = 0.f;
      for (int b = 0; b < wt.n; ++b)
        if (zoom_clampi(s * j + b - 1, 0, W - 1) == X) wx += wt.w[b];
      row = fmaf(wx, r[(int64_t)i * w + j], row);
    }
    acc = fmaf(wy, row, acc);
  }
  g[(int64_t)Y * W + X] = alpha * acc;
}

// dE/dP[n][p] = gx(Y, X) / n_cov(Y, X) + lambda * 2 * sum over the 4 LR-grid
// neighbour patches q overlapping pixel p of (P_n - P_q) at that pixel.
__global__ void k_patch_grad(const float* __restrict__ gx, const float* __restrict__ P, int h, int w, int s,
                             int Pp, float lambda, float* __restrict__ gP) {
  const int PH = s * Pp, ph2 = PH * PH;
  const int nh = h - Pp + 1, nw = w - Pp + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nh * nw * ph2) return;
  const int64_t n = t / ph2;
  const int p = (int)(t % ph2);
  const int i = (int)(n / nw), j = (int)(n % nw);
  const int a = p / PH, b = p % PH;
  const int Y = s * i + a, X = s * j + b;
  const int W = s * w;
  const int ci = min(Y / s, nh - 1) - (Y >= PH ? (Y - PH) / s + 1 : 0) + 1;
  const int cj = min(X / s, nw - 1) - (X >= PH ? (X - PH) / s + 1 : 0) + 1;
  float g = gx[(int64_t)Y * W + X] / (float)(ci * cj);
  if (lambda != 0.f) {   // P is read only for the prior term
    const float pv = P[t];
    float pr = 0.f;
    if (j + 1 < nw && b >= s) pr += pv - P[(n + 1) * ph2 + a * PH + (b - s)];
    if (j > 0 && b < PH - s) pr += pv - P[(n - 1) * ph2 + a * PH + (b + s)];
    if (i + 1 < nh && a >= s) pr += pv - P[(n + nw) * ph2 + (a - s) * PH + b];
    if (i > 0 && a < PH - s) pr += pv - P[(n - nw) * ph2 + (a + s) * PH + b];
    g = fmaf(2.f * lambda, pr, g);
  }
  gP[t] = g;
}

// grad_R[id][p] = sum over the uses u of entry id (sorted, ascending) of
// w[u] * gP[u / K][p]; one block per used entry, one thread per pixel.
__global__ void k_dict_grad(const int32_t* __restrict__ sorted_use, const int32_t* __restrict__ offs,
                            const uint64_t* __restrict__ ukeys, const int32_t* __restrict__ nuniq,
                            const float* __restrict__ wgt, const float* __restrict__ gP, int K, int ph2,
                            int ph2pad_out, float* __restrict__ grad) {
  const int seg = blockIdx.x;
  if (seg >= *nuniq) return;
  const int id = (int)ukeys[seg];
  for (int p = threadIdx.x; p < ph2; p += blockDim.x) {
    float acc = 0.f;
    for (int u = offs[seg]; u < offs[seg + 1]; ++u) {
      const int use = sorted_use[u];
      acc = fmaf(wgt[use], gP[(int64_t)(use / K) * ph2 + p], acc);
    }
    grad[(int64_t)id * ph2pad_out + p] = acc;
  }
}

// grad_mu[n] = sum_p OA^T(g)[n][p] (the patch mean enters every pixel).
__global__ void k_mu_grad(const float* __restrict__ gP, int64_t nq, int ph2, float* __restrict__ gmu) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nq) return;
  float acc = 0.f;
  for (int p = 0; p < ph2; ++p) acc += gP[n * ph2 + p];
  gmu[n] = acc;
}

// per-block partial sums (in FP64) of r^2 over n values
__global__ void k_sumsq_partials(const float* __restrict__ r, int64_t n, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)r[i] * (double)r[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// per-block partial sums of the overlap prior: each (patch, pixel) adds the
// squared difference to its right and down neighbours where they overlap
__global__ void k_prior_partials(const float* __restrict__ P, int h, int w, int s, int Pp,
                                 double* __restrict__ part) {
  __shared__ double sh[256];
  const int PH = s * Pp, ph2 = PH * PH;
  const int nh = h - Pp + 1, nw = w - Pp + 1;
  const int64_t total = (int64_t)nh * nw * ph2;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t / ph2;
    const int p = (int)(t % ph2);
    const int i = (int)(n / nw), j = (int)(n % nw);
    const int a = p / PH, b = p % PH;
    const float pv = P[t];
    if (j + 1 < nw && b >= s) {
      const double d = (double)pv - (double)P[(n + 1) * ph2 + a * PH + (b - s)];
      acc += d * d;
    }
    if (i + 1 < nh && a >= s) {
      const double d = (double)pv - (double)P[(n + nw) * ph2 + (a - s) * PH + b];
      acc += d * d;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// dist[n][m] = |q_n - c_{nbr[n][m]}|^2 (FP32 difference form)
template <int D>
__global__ void k_nbr_dist(const float* __restrict__ qfeat, int dpad, int64_t nq, const float* __restrict__ dfeat,
                           const int32_t* __restrict__ nbr, int K, float* __restrict__ dist) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nq * K) return;
  const int64_t n = t / K;
  const int64_t id = nbr[t];
  float dd = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float df = qfeat[n * dpad + i] - dfeat[id * dpad + i];
    dd = fmaf(df, df, dd);
  }
  dist[t] = dd;
}

Wts degrade_wts(int s, double sigma) {
  Wts wt;
  double e = exp(-1.0 / (2.0 * sigma * sigma));
  double t[3] = {e / (1.0 + 2.0 * e), 1.0 / (1.0 + 2.0 * e), e / (1.0 + 2.0 * e)};
  double acc[8] = {0};
  for (int b = 0; b < s; ++b)
    for (int u = 0; u < 3; ++u) acc[b + u] += t[u] / s;
  wt.n = s + 2;
  for (int a = 0; a < 8; ++a) wt.w[a] = (float)acc[a];
  return wt;
}

}  // namespace

cudaError_t launch_patches(const int32_t* nbr, const float* wgt, const float* mu, const float* hr_res,
                           int ph2pad, int K, int64_t nq, int ph2, float* P, cudaStream_t st) {
  const int64_t tot = nq * ph2;
  k_patches<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(nbr, wgt, mu, hr_res, ph2pad, K, nq, ph2, P);
  return cudaGetLastError();
}

cudaError_t launch_degrade(const float* x, int H, int W, int s, double sigma, const float* sub, float* y,
                           cudaStream_t st) {
  const int h = H / s, w = W / s;
  dim3 blk(32, 8), grd((w + 31) / 32, (h + 7) / 8);
  k_degrade<<<grd, blk, 0, st>>>(x, H, W, h, w, s, degrade_wts(s, sigma), sub, y);
  return cudaGetLastError();
}

cudaError_t launch_degrade_adjoint(const float* r, int h, int w, int H, int W, int s, double sigma,
                                   float alpha, float* g, cudaStream_t st) {
  dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
  k_degrade_adjoint<<<grd, blk, 0, st>>>(r, h, w, H, W, s, degrade_wts(s, sigma), alpha, g);
  return cudaGetLastError();
}

cudaError_t launch_patch_grad(const float* gx, const float* P, int h, int w, int s, int Pp, float lambda,
                              float* gP, cudaStream_t st) {
  const int64_t tot = (int64_t)(h - Pp + 1) * (w - Pp + 1) * (s * Pp) * (s * Pp);
  k_patch_grad<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(gx, P, h, w, s, Pp, lambda, gP);
  return cudaGetLastError();
}

cudaError_t launch_dict_grad(const int32_t* sorted_use, const int32_t* offs, const uint64_t* ukeys,
                             const int32_t* nuniq, int64_t max_segments, const float* wgt, const float* gP,
                             int K, int ph2, int ph2pad_out, float* grad, cudaStream_t st) {
  if (max_segments <= 0) return cudaSuccess;
  k_dict_grad<<<(unsigned)max_segments, 128, 0, st>>>(sorted_use, offs, ukeys, nuniq, wgt, gP, K, ph2,
                                                      ph2pad_out, grad);
  return cudaGetLastError();
}

cudaError_t launch_mu_grad(const float* gP, int64_t nq, int ph2, float* gmu, cudaStream_t st) {
  k_mu_grad<<<(unsigned)((nq + 127) / 128), 128, 0, st>>>(gP, nq, ph2, gmu);
  return cudaGetLastError();
}

cudaError_t launch_energy_partials(const float* r, int64_t n_r, const float* P, int h, int w, int s, int Pp,
                                   double* part, int nblocks, cudaStream_t st) {
  k_sumsq_partials<<<nblocks, 256, 0, st>>>(r, n_r, part);
  k_prior_partials<<<nblocks, 256, 0, st>>>(P, h, w, s, Pp, part + nblocks);
  return cudaGetLastError();
}

cudaError_t launch_nbr_dist(const float* qfeat, int dpad, int d, int64_t nq, const float* dfeat,
                            const int32_t* nbr, int K, float* dist, cudaStream_t st) {
  const int64_t tot = nq * K;
  const unsigned blocks = (unsigned)((tot + 127) / 128);
  if (d == 9) k_nbr_dist<9><<<blocks, 128, 0, st>>>(qfeat, dpad, nq, dfeat, nbr, K, dist);
  else if (d == 25) k_nbr_dist<25><<<blocks, 128, 0, st>>>(qfeat, dpad, nq, dfeat, nbr, K, dist);
  else if (d == 18) k_nbr_dist<18><<<blocks, 128, 0, st>>>(qfeat, dpad, nq, dfeat, nbr, K, dist);
  else if (d == 50) k_nbr_dist<50><<<blocks, 128, 0, st>>>(qfeat, dpad, nq, dfeat, nbr, K, dist);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
