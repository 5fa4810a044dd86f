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
