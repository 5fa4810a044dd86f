// Device helpers shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define ZOOM_GOLDEN64 0x9E3779B97F4A7C15ull

// Stafford's variant-13 64-bit finaliser (the SplitMix64 output mixer).
__device__ __forceinline__ uint64_t zoom_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One step of the bucket-key fold: x <- mix64(x ^ (uint32(h_j) + G * (j + 1))).
__device__ __forceinline__ uint64_t zoom_fold_step(uint64_t x, int h, int j) {
  return zoom_mix64(x ^ ((uint64_t)(uint32_t)h + ZOOM_GOLDEN64 * (uint64_t)(j + 1)));
}

// Feature of one patch: mean mu (sequential FP32 sum / D) and v = px - mu.
// The same routine serves dictionary entries and queries, so a query equal
// to an entry has bit-identical features and distance exactly 0.
template <int D>
__device__ __forceinline__ void zoom_patch_feature(const float (&px)[D], float (&v)[D], float& mu,
                                                   float& norm2) {
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) s += px[i];
  mu = __fdiv_rn(s, (float)D);
  float n2 = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    v[i] = px[i] - mu;
    n2 = fmaf(v[i], v[i], n2);
  }
  norm2 = n2;
}

__device__ __forceinline__ int zoom_clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Feature dimension of a P x P patch: the pixels minus their mean (mode 0) or
// the first- or second-order gradients at the patch's pixels (modes 1, 2).
__host__ __device__ constexpr int zoom_feature_dim(int P, int F) { return F ? 2 * P * P : P * P; }

// Gradient feature of the P x P patch at (i, j) of an h x w image (row
// stride ld), image coordinates clamped to the image.  ORDER 1: g_x(r, c) =
// x(r, c+1) - x(r, c-1), g_y(r, c) = x(r+1, c) - x(r-1, c) (the correlation
// with [-1, 0, 1] and its transpose).  ORDER 2: g_xx(r, c) = 2 x(r, c) -
// x(r, c-2) - x(r, c+2) and g_yy likewise ([-1, 0, 2, 0, -1]).  v = [g_x |
// g_y], each row-major over the patch; norm2 = sum of v^2 (sequential FMA).
// Dictionary entries and queries share it, so equal neighbourhoods give
// bit-identical features.
template <int P, int ORDER>
__device__ __forceinline__ void zoom_gradient_feature(const float* __restrict__ img, int h, int w,
                                                      size_t ld, int i, int j, float (&v)[2 * P * P],
                                                      float& norm2) {
#pragma unroll
  for (int a = 0; a < P; ++a) {
    const int r = i + a;
    const int rm = r - ORDER > 0 ? r - ORDER : 0, rp = r + ORDER < h ? r + ORDER : h - 1;
#pragma unroll
    for (int b = 0; b < P; ++b) {
      const int c = j + b;
      const int cm = c - ORDER > 0 ? c - ORDER : 0, cp = c + ORDER < w ? c + ORDER : w - 1;
      const float xm = img[(size_t)r * ld + cm], xp = img[(size_t)r * ld + cp];
      const float ym = img[(size_t)rm * ld + c], yp = img[(size_t)rp * ld + c];
      if constexpr (ORDER == 1) {
        v[a * P + b] = xp - xm;
        v[P * P + a * P + b] = yp - ym;
      } else {
        const float x0 = img[(size_t)r * ld + c];
        v[a * P + b] = fmaf(2.f, x0, -xm) - xp;
        v[P * P + a * P + b] = fmaf(2.f, x0, -ym) - yp;
      }
    }
  }
  float n2 = 0.f;
#pragma unroll
  for (int q = 0; q < 2 * P * P; ++q) n2 = fmaf(v[q], v[q], n2);
  norm2 = n2;
}
