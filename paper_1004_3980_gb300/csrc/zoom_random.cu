// Seeded random draws of the library: the projections and offsets of the
// hash (Sec. 4.1, Eq. 10; Cauchy vectors by the rule of Eq. 11) and the
// dictionary positions (Sec. 2.1, Sec. 5.1), for callers that give a seed
// instead of the arrays.  All from the counter-based generator
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): output k of a stream is a pure function of
// (seed, counter), so the draws do not depend on the order, thread or
// machine that computes them.  Host code (a one-off step of a build).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "zoom_internal.h"

namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;   // round multipliers
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;   // key increments
constexpr double kPi = 3.141592653589793;

// Ten rounds of (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
// hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key (low, high word of the seed)
// gains (W0, W1) before every round but the first.
void philox4x32_10(const uint32_t in[4], uint64_t seed, uint32_t out[4]) {
  uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kW0;
      k1 += kW1;
    }
    const uint64_t p0 = (uint64_t)kM0 * c0, p1 = (uint64_t)kM1 * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// Counter (n, t, c2, c3) of stream n, draw t.
void draw(uint64_t n, uint32_t t, uint32_t c2, uint32_t c3, uint64_t seed, uint32_t out[4]) {
  const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32) + t, c2, c3};
  philox4x32_10(ctr, seed, out);
}

// A 32-bit word to a uniform value in (0, 1).
double unit(uint32_t x) { return ((double)x + 0.5) * 0x1p-32; }

// Box-Muller, cosine branch, in FP64.
double normal(const uint32_t w[4]) { return sqrt(-2.0 * log(unit(w[0]))) * cos(2.0 * kPi * unit(w[1])); }

}  // namespace

void zoom_draw_projections(int L, int k, int D, float w, int dist, uint64_t seed, float* alpha, float* beta) {
  const int64_t n = (int64_t)L * k * D;
  uint32_t o[4];
  for (int64_t i = 0; i < n; ++i) {
    draw((uint64_t)i, 0, 0, 0, seed, o);
    double a = normal(o);
    if (dist == 1) {   // Eq. 11: a / b with b ~ N(0, 1) redrawn until |b| >= eps
      double b = 0.0;
      for (uint32_t t = 0;; ++t) {
        draw((uint64_t)i, t, 1, 0, seed, o);
        b = normal(o);
        if (fabs(b) >= kCauchyEps) break;
      }
      a = a / b;
    }
    alpha[i] = (float)a;
  }
  const float below_w = nextafterf(w, 0.f);
  for (int j = 0; j < L * k; ++j) {
    draw((uint64_t)j, 0, 0, 1, seed, o);
    const float b = (float)(unit(o[0]) * (double)w);
    beta[j] = b < w ? b : below_w;
  }
}

int64_t zoom_count_origins(int n_images, const int32_t* lr_h, const int32_t* lr_w, int P) {
  int64_t total = 0;
  for (int m = 0; m < n_images; ++m) {
    if (lr_h[m] < P || lr_w[m] < P) return -1;
    total += (int64_t)(lr_h[m] - P + 1) * (lr_w[m] - P + 1);
  }
  return total;
}

bool zoom_sample_positions_host(uint64_t seed, int n_images, const int32_t* lr_h, const int32_t* lr_w, int P,
                                int64_t n_pairs, int32_t* positions) {
  const int64_t total = zoom_count_origins(n_images, lr_h, lr_w, P);
  if (total < 1 || n_pairs < 1 || n_pairs > total) return false;
  // origin o draws the 64-bit key of counter (o, 0, 0, 2); the n_pairs
  // smallest (key, o) form a uniform subset without replacement
  std::vector<std::pair<uint64_t, int64_t>> key((size_t)total);
  uint32_t o[4];
  for (int64_t i = 0; i < total; ++i) {
    draw((uint64_t)i, 0, 0, 2, seed, o);
    key[(size_t)i] = {((uint64_t)o[0] << 32) | o[1], i};
  }
  if (n_pairs < total) std::nth_element(key.begin(), key.begin() + (n_pairs - 1), key.end());
  std::vector<int64_t> chosen((size_t)n_pairs);
  for (int64_t i = 0; i < n_pairs; ++i) chosen[(size_t)i] = key[(size_t)i].second;
  std::sort(chosen.begin(), chosen.end());   // origin order: the rank is the ID
  int m = 0;
  int64_t start = 0, count = (int64_t)(lr_h[0] - P + 1) * (lr_w[0] - P + 1);
  for (int64_t i = 0; i < n_pairs; ++i) {
    while (chosen[(size_t)i] >= start + count) {
      start += count;
      ++m;
      count = (int64_t)(lr_h[m] - P + 1) * (lr_w[m] - P + 1);
    }
    const int64_t r = chosen[(size_t)i] - start, nw = lr_w[m] - P + 1;
    positions[3 * i] = m;
    positions[3 * i + 1] = (int32_t)(r / nw);
    positions[3 * i + 2] = (int32_t)(r % nw);
  }
  return true;
}

extern "C" {

zoom_status zoom_lsh_draws(const zoom_lsh_params* lsh, int32_t dim, float* alpha, float* beta) {
  if (!lsh || !alpha || !beta) {
    zoom_set_error("NULL argument");
    return ZOOM_ERR_INVALID_ARG;
  }
  if (lsh->L < 1 || lsh->L > 32 || lsh->k < 1 || lsh->k > 32 || dim < 1 || dim > 64 || !(lsh->w > 0.f) ||
      lsh->proj_dist < 0 || lsh->proj_dist > 1) {
    zoom_set_error("L, k in 1..32, dim in 1..64, w > 0, proj_dist 0 or 1");
    return ZOOM_ERR_INVALID_ARG;
  }
  zoom_draw_projections(lsh->L, lsh->k, dim, lsh->w, lsh->proj_dist, lsh->seed, alpha, beta);
  return ZOOM_OK;
}

zoom_status zoom_sample_positions(uint64_t seed, int32_t n_images, const int32_t* lr_heights,
                                  const int32_t* lr_widths, int32_t lr_patch, int64_t n_pairs,
                                  int32_t* positions) {
  if (!lr_heights || !lr_widths || !positions || n_images < 1 || lr_patch < 1) {
    zoom_set_error("NULL argument or no image");
    return ZOOM_ERR_INVALID_ARG;
  }
  const int64_t total = zoom_count_origins(n_images, lr_heights, lr_widths, lr_patch);
  if (total < 1 || n_pairs < 1 || n_pairs > total) {
    zoom_set_error("n_pairs must be in 1.." + std::to_string(total < 0 ? 0 : total) +
                   " (the patch origins of the images)");
    return ZOOM_ERR_INVALID_ARG;
  }
  zoom_sample_positions_host(seed, n_images, lr_heights, lr_widths, lr_patch, n_pairs, positions);
  return ZOOM_OK;
}

}  // extern "C"
