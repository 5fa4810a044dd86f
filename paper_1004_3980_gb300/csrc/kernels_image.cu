// HR image steps: blend + overlap average (Eq. 14; averaging of overlaps)
// and the error back-projection with the approximate cross-bilateral filter
// (Sec. 4, Eq. 6-7; Sec. 4.3, Eq. 15-17).
#include <math.h>

#include "device_common.cuh"
#include "zoom_internal.h"

namespace {

// Gather form: each HR pixel sums, over the patches covering it, the
// patch's blended value mu_n + sum_m w_nm R[nbr_nm] at its offset, and
// divides by the number of covering patches.  No atomics.
__global__ void k_overlap_add(const int32_t* __restrict__ nbr, const float* __restrict__ wgt,
                              const float* __restrict__ mu, const float* __restrict__ hr_res,
                              int ph2pad, int K, int h, int w, int s, int P,
                              float* __restrict__ hr) {
  const int W = s * w, H = s * h;
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= W || Y >= H) return;
  const int PH = s * P, nh = h - P + 1, nw = w - P + 1;
  const int i_hi = min(Y / s, nh - 1), j_hi = min(X / s, nw - 1);
  const int i_lo = Y >= PH ? (Y - PH) / s + 1 : 0;
  const int j_lo = X >= PH ? (X - PH) / s + 1 : 0;
  float acc = 0.f;
  int cnt = 0;
  for (int i = i_lo; i <= i_hi; ++i) {
    for (int j = j_lo; j <= j_hi; ++j) {
      const int64_t n = (int64_t)i * nw + j;
      const int off = (Y - s * i) * PH + (X - s * j);
      float v = mu[n];
      for (int m = 0; m < K; ++m)
        v = fmaf(wgt[n * K + m], hr_res[(int64_t)nbr[n * K + m] * ph2pad + off], v);
      acc += v;
      ++cnt;
    }
  }
  hr[(int64_t)Y * W + X] = acc / (float)cnt;
}

// The same average in two passes, for callers with nq * PH^2 floats of
// scratch.  Pass 1 blends the patches of 32 consecutive queries of one patch
// row: the neighbours' residual rows are read whole, in order and 16 bytes
// per load, each thread blending 4 adjacent patch pixels (the one-pass form
// reads each 4-byte value from the pixels it covers, scattered over the
// row), and the blended values leave through shared memory,
// transposed to the layout [patch row i][patch pixel p][patch column j].
// Pass 2 averages them per HR pixel: for one covering patch the lanes of a
// warp then read s runs of consecutive j.  Each blended value is computed
// with the same operations in the same order as in the one-pass form, and
// pass 2 sums them in its order, so both forms give the same bits.
constexpr int kBlendQ = 32;       // queries of one patch row per block
constexpr int kBlendPC = 128;     // patch pixels per shared-memory round
constexpr int kBlendMaxK = 64;

__global__ void __launch_bounds__(256) k_blend_rows(const int32_t* __restrict__ nbr,
                                                    const float* __restrict__ wgt,
                                                    const float* __restrict__ mu,
                                                    const float* __restrict__ hr_res, int ph2pad, int K,
                                                    int nw, int ph2, float* __restrict__ out) {
  __shared__ int32_t s_nbr[kBlendQ * kBlendMaxK];
  __shared__ float s_w[kBlendQ * kBlendMaxK];
  __shared__ float s_mu[kBlendQ];
  __shared__ float s_t[kBlendPC * (kBlendQ + 1)];
  const int i = blockIdx.y;
  const int j0 = blockIdx.x * kBlendQ;
  const int nqc = min(kBlendQ, nw - j0);
  const int64_t n0 = (int64_t)i * nw + j0;
  for (int e = threadIdx.x; e < nqc * K; e += blockDim.x) {
    s_nbr[e] = nbr[n0 * K + e];
    s_w[e] = wgt[n0 * K + e];
  }
  if ((int)threadIdx.x < nqc) s_mu[threadIdx.x] = mu[n0 + threadIdx.x];
  __syncthreads();
  for (int p0 = 0; p0 < ph2; p0 += kBlendPC) {
    const int pc = min(kBlendPC, ph2 - p0);
    const int pq = (pc + 3) / 4;   // 4-pixel groups; the last may reach into the row's padding
    for (int e = threadIdx.x; e < nqc * pq; e += blockDim.x) {
      const int q = e / pq, pl = 4 * (e - q * pq);
      const int32_t* nb = s_nbr + q * K;
      const float* wq = s_w + q * K;
      const float* col = hr_res + p0 + pl;
      float4 v = make_float4(s_mu[q], s_mu[q], s_mu[q], s_mu[q]);
      for (int m0 = 0; m0 < K; m0 += 8) {
        float4 r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          r[u] = m0 + u < K ? __ldg(reinterpret_cast<const float4*>(col + (int64_t)nb[m0 + u] * ph2pad))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (m0 + u < K) {
            const float wm = wq[m0 + u];
            v.x = fmaf(wm, r[u].x, v.x);
            v.y = fmaf(wm, r[u].y, v.y);
            v.z = fmaf(wm, r[u].z, v.z);
            v.w = fmaf(wm, r[u].w, v.w);
          }
      }
      float* t = s_t + pl * (kBlendQ + 1) + q;
      t[0] = v.x;
      if (pl + 1 < pc) t[kBlendQ + 1] = v.y;
      if (pl + 2 < pc) t[2 * (kBlendQ + 1)] = v.z;
      if (pl + 3 < pc) t[3 * (kBlendQ + 1)] = v.w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < pc * kBlendQ; e += blockDim.x) {
      const int pl = e / kBlendQ, q = e % kBlendQ;
      if (q < nqc) out[((int64_t)i * ph2 + p0 + pl) * nw + j0 + q] = s_t[pl * (kBlendQ + 1) + q];
    }
    __syncthreads();
  }
}

__global__ void k_overlap_average(const float* __restrict__ pb, int h, int w, int s, int P,
                                  float* __restrict__ hr) {
  const int W = s * w, H = s * h;
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  const int Y = blockIdx.y * blockDim.y + threadIdx.y;
  if (X >= W || Y >= H) return;
  const int PH = s * P, nh = h - P + 1, nw = w - P + 1, ph2 = PH * PH;
  const int i_hi = min(Y / s, nh - 1), j_hi = min(X / s, nw - 1);
  const int i_lo = Y >= PH ? (Y - PH) / s + 1 : 0;
  const int j_lo = X >= PH ? (X - PH) / s + 1 : 0;
  float acc = 0.f;
  int cnt = 0;
  for (int i = i_lo; i <= i_hi; ++i) {
    const float* row = pb + ((int64_t)i * ph2 + (Y - s * i) * PH) * nw;
    for (int j = j_lo; j <= j_hi; ++j) {
      acc += __ldg(row + (int64_t)(X - s * j) * nw + j);
      ++cnt;
    }
  }
  hr[(int64_t)Y * W + X] = acc / (float)cnt;
}

// e = D(B x) - y on the LR grid (FP32).  The blur and the box mean combine
// into separable 1-D weights over the (s+2)-wide window.
struct Wts1D {
  int n;
  float w[8];
};

__global__ void k_bp_error(const float* __restrict__ x, int H, int W, const float* __restrict__ y,
                           int h, int w, int s, Wts1D wt, float* __restrict__ e) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= h || j >= w) return;
  float acc = 0.f;
  for (int a = 0; a < wt.n; ++a) {
    const int r = zoom_clampi(s * i + a - 1, 0, H - 1);
    float row = 0.f;
    for (int b = 0; b < wt.n; ++b) {
      const int c = zoom_clampi(s * j + b - 1, 0, W - 1);
      row = fmaf(wt.w[b], x[(int64_t)r * W + c], row);
    }
    acc = fmaf(wt.w[a], row, acc);
  }
  e[(int64_t)i * w + j] = acc - y[(int64_t)i * w + j];
}

// x' = x - r * G, G = normalised spatial Gaussian over the replicated LR
// error, r = exp(-(x - mean_Gamma x)^2 / (2 sigma_r^2)); clamped borders.
struct Gauss1D {
  int R;
  float c[16];
};

// One block computes a 64-row x 32-column tile of x' from shared memory: the
// tile of x with its R-pixel halo (clamped), then the separable sums -- each
// row's box sum over the 2R+1 columns, and for each LR error row the
// Gaussian-weighted sum over the 2R+1 replicated columns -- and per pixel the
// column sums over 2R+1 rows.  The summation order is that of the direct
// double loop (columns t within a row, then rows u), so the result is the
// same bit for bit; x is read from memory once (with the halo) instead of
// (2R+1)^2 times, and the LR row and column of every clamped tile row and
// column are computed once per block.
constexpr int kBpTileW = 32, kBpTileH = 64;
template <int R>
__global__ void __launch_bounds__(256) k_bp_update(const float* __restrict__ x, float* __restrict__ xo, int H,
                                                   int W, const float* __restrict__ e, int w, int s, Gauss1D g,
                                                   float inv_two_sr2) {
  constexpr int T = 2 * R + 1;
  constexpr int NW = kBpTileW + 2 * R, NH = kBpTileH + 2 * R;   // the tile with its halo
  __shared__ float xs[NH][NW + 1];      // x, clamped
  __shared__ float hs[NH][kBpTileW];    // row box sums
  __shared__ float hg[NH][kBpTileW];    // per LR row: Gaussian row sums of the replicated error
  __shared__ int lrow[NH], lcol[NW];    // LR row (relative to lr0) / column of each clamped tile row / column
  const int X0 = blockIdx.x * kBpTileW, Y0 = blockIdx.y * kBpTileH;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lr0 = zoom_clampi(Y0 - R, 0, H - 1) / s;
  const int nlr = zoom_clampi(Y0 + kBpTileH - 1 + R, 0, H - 1) / s - lr0 + 1;
  for (int i = tid; i < NH; i += 256) lrow[i] = zoom_clampi(Y0 - R + i, 0, H - 1) / s - lr0;
  for (int i = tid; i < NW; i += 256) lcol[i] = zoom_clampi(X0 - R + i, 0, W - 1) / s;
  for (int i = tid; i < NH * NW; i += 256) {
    const int r = i / NW, c = i % NW;
    xs[r][c] = x[(int64_t)zoom_clampi(Y0 - R + r, 0, H - 1) * W + zoom_clampi(X0 - R + c, 0, W - 1)];
  }
  __syncthreads();
  for (int i = tid; i < nlr * kBpTileW; i += 256) {
    const int r = i / kBpTileW, c = i % kBpTileW;
    const float* er = e + (int64_t)(lr0 + r) * w;
    float grow = 0.f;
#pragma unroll
    for (int t = 0; t < T; ++t) grow = fmaf(g.c[t], er[lcol[c + t]], grow);
    hg[r][c] = grow;
  }
  for (int i = tid; i < NH * kBpTileW; i += 256) {
    const int r = i / kBpTileW, c = i % kBpTileW;
    float brow = 0.f;
#pragma unroll
    for (int t = 0; t < T; ++t) brow += xs[r][c + t];
    hs[r][c] = brow;
  }
  __syncthreads();
  const int c = threadIdx.x;
  const int X = X0 + c;
  if (X >= W) return;
  for (int y = threadIdx.y; y < kBpTileH; y += blockDim.y) {
    const int Y = Y0 + y;
    if (Y >= H) break;
    float gs = 0.f, box = 0.f;
#pragma unroll
    for (int u = 0; u < T; ++u) {
      gs = fmaf(g.c[u], hg[lrow[y + u]][c], gs);
      box += hs[y + u][c];
    }
    const float m = box / (float)(T * T);
    const float xv = xs[y + R][c + R];
    const float dv = xv - m;
    const float r = expf(-dv * dv * inv_two_sr2);
    xo[(int64_t)Y * W + X] = xv - r * gs;
  }
}

}  // namespace

cudaError_t launch_overlap_add(const int32_t* nbr, const float* wgt, const float* mu,
                               const float* hr_res, int ph2pad, int K, int h, int w, int s, int P,
                               float* hr, cudaStream_t st) {
  dim3 blk(32, 8), grd((s * w + 31) / 32, (s * h + 7) / 8);
  k_overlap_add<<<grd, blk, 0, st>>>(nbr, wgt, mu, hr_res, ph2pad, K, h, w, s, P, hr);
  return cudaGetLastError();
}

cudaError_t launch_overlap_add_staged(const int32_t* nbr, const float* wgt, const float* mu,
                                      const float* hr_res, int ph2pad, int K, int h, int w, int s, int P,
                                      float* patches, float* hr, cudaStream_t st) {
  const int nh = h - P + 1, nw = w - P + 1, PH = s * P;
  // 16-byte loads of the residual rows: 16-byte aligned rows, padded to 4
  if (K > kBlendMaxK || nh > 65535 || !patches || ph2pad % 4 != 0 || ph2pad < PH * PH ||
      reinterpret_cast<uintptr_t>(hr_res) % 16 != 0)
    return launch_overlap_add(nbr, wgt, mu, hr_res, ph2pad, K, h, w, s, P, hr, st);
  dim3 g1((nw + kBlendQ - 1) / kBlendQ, nh);
  k_blend_rows<<<g1, 256, 0, st>>>(nbr, wgt, mu, hr_res, ph2pad, K, nw, PH * PH, patches);
  dim3 blk(32, 8), g2((s * w + 31) / 32, (s * h + 7) / 8);
  k_overlap_average<<<g2, blk, 0, st>>>(patches, h, w, s, P, hr);
  return cudaGetLastError();
}

cudaError_t launch_bp_iteration(const float* x, float* x_out, const float* lr, float* err, int h,
                                int w, int s, double blur_sigma, float sigma_sp, float sigma_r,
                                int radius, cudaStream_t st) {
  const int H = s * h, W = s * w;
  Wts1D wt;
  {
    double e = exp(-1.0 / (2.0 * blur_sigma * blur_sigma));
    double t[3] = {e / (1.0 + 2.0 * e), 1.0 / (1.0 + 2.0 * e), e / (1.0 + 2.0 * e)};
    double acc[8] = {0};
    for (int b = 0; b < s; ++b)
      for (int u = 0; u < 3; ++u) acc[b + u] += t[u] / s;
    wt.n = s + 2;
    for (int a = 0; a < 8; ++a) wt.w[a] = (float)acc[a];
  }
  Gauss1D g;
  {
    g.R = radius;
    double c[16], tot = 0.0;
    for (int d = -radius; d <= radius; ++d) {
      c[d + radius] = exp(-(double)(d * d) / (2.0 * (double)sigma_sp * (double)sigma_sp));
      tot += c[d + radius];
    }
    for (int d = 0; d < 16; ++d) g.c[d] = d < 2 * radius + 1 ? (float)(c[d] / tot) : 0.f;
  }
  dim3 blk(32, 8);
  dim3 g1((w + 31) / 32, (h + 7) / 8);
  k_bp_error<<<g1, blk, 0, st>>>(x, H, W, lr, h, w, s, wt, err);
  dim3 g2((W + kBpTileW - 1) / kBpTileW, (H + kBpTileH - 1) / kBpTileH);
  const float inv = (float)(1.0 / (2.0 * (double)sigma_r * (double)sigma_r));
  switch (radius) {
#define ZOOM_BPU(RR) \
  case RR: k_bp_update<RR><<<g2, blk, 0, st>>>(x, x_out, H, W, err, w, s, g, inv); break;
    ZOOM_BPU(1) ZOOM_BPU(2) ZOOM_BPU(3) ZOOM_BPU(4) ZOOM_BPU(5) ZOOM_BPU(6) ZOOM_BPU(7)
#undef ZOOM_BPU
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
