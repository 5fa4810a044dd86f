// Training-crop sampling (Sec. 5.1, "Training Data Generation"): a CDF over
// each HR training image's pixels from its first-order gradient magnitude,
// the centre pixel of each crop drawn from it, and the crops themselves.
//
// The mass of a pixel is sqrt(g_x^2 + g_y^2) in FP64 (g: the clamped central
// differences of the feature representation, Sec. 4.1), each operation
// rounded once, so it equals the FP64 definition bit for bit.  The CDF is a
// deterministic FP64 sum: tiles of 1024 row-major pixels, each summed by one
// warp (lane l adds pixels l, l + 32, ... in order, then a fixed xor tree),
// tile sums accumulated in order per image.  A draw u selects the first
// pixel whose cumulative mass exceeds u * total: one warp finds the tile by
// binary search over the tile prefix sums, then scans the tile 32 pixels at
// a time.  This order differs from a sequential sum only by FP64 rounding.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "zoom_internal.h"

namespace {

constexpr int kTile = 1024;
constexpr unsigned kAll = 0xffffffffu;

struct ImgDesc {
  const float* p;
  int32_t h, w;
  int64_t tile0;   // first tile of this image in the tile arrays
};

__device__ __forceinline__ double pixel_mass(const float* __restrict__ img, int h, int w, int64_t idx) {
  const int r = (int)(idx / w), c = (int)(idx % w);
  const int cm = c > 0 ? c - 1 : 0, cp = c + 1 < w ? c + 1 : w - 1;
  const int rm = r > 0 ? r - 1 : 0, rp = r + 1 < h ? r + 1 : h - 1;
  const double gx = __dsub_rn((double)img[(size_t)r * w + cp], (double)img[(size_t)r * w + cm]);
  const double gy = __dsub_rn((double)img[(size_t)rp * w + c], (double)img[(size_t)rm * w + c]);
  return sqrt(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)));
}

// The image a global tile belongs to (binary search over the first tiles).
__device__ __forceinline__ int image_of_tile(const ImgDesc* __restrict__ im, int n_images, int64_t t) {
  int lo = 0, hi = n_images - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (im[mid].tile0 <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One warp per tile: the tile's FP64 mass.
__global__ void k_tile_mass(const ImgDesc* __restrict__ im, int n_images, int64_t n_tiles,
                            double* __restrict__ tile_sum) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n_tiles) return;   // warp-uniform
  const ImgDesc d = im[image_of_tile(im, n_images, t)];
  const int64_t n = (int64_t)d.h * d.w;
  const int64_t base = (t - d.tile0) * kTile;
  double s = 0.0;
  for (int k = 0; k < kTile / 32; ++k) {
    const int64_t idx = base + k * 32 + lane;
    if (idx < n) s = __dadd_rn(s, pixel_mass(d.p, d.h, d.w, idx));
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) s = __dadd_rn(s, __shfl_xor_sync(kAll, s, off));
  if (lane == 0) tile_sum[t] = s;
}

// One thread per image: inclusive prefix of its tile sums, in order.
__global__ void k_tile_prefix(const ImgDesc* __restrict__ im, int n_images, double* __restrict__ tile_sum) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_images) return;
  const ImgDesc d = im[m];
  const int64_t nt = ((int64_t)d.h * d.w + kTile - 1) / kTile;
  double acc = 0.0;
  for (int64_t t = 0; t < nt; ++t) {
    acc = __dadd_rn(acc, tile_sum[d.tile0 + t]);
    tile_sum[d.tile0 + t] = acc;
  }
}

// One warp per draw: the drawn pixel and the crop window around it.
// win: int32 [n_draws][4] = centre row, centre column, top, left.
__global__ void k_draw(const ImgDesc* __restrict__ im, const double* __restrict__ pref,
                       const double* __restrict__ u, int64_t n_draws, int draws_per_image, int ch, int cw,
                       int32_t* __restrict__ win) {
  const int64_t dr = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (dr >= n_draws) return;   // warp-uniform
  const ImgDesc d = im[dr / draws_per_image];
  const int64_t n = (int64_t)d.h * d.w;
  const int64_t nt = (n + kTile - 1) / kTile;
  const double* tp = pref + d.tile0;
  const double total = tp[nt - 1];
  const double ud = u[dr];
  int64_t idx;
  if (!(total > 0.0)) {
    idx = (int64_t)floor(ud * (double)n);
    if (idx > n - 1) idx = n - 1;
  } else {
    const double target = __dmul_rn(ud, total);
    // the first tile whose inclusive prefix exceeds the target (the last if none)
    int64_t lo = 0, hi = nt - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (tp[mid] > target) hi = mid; else lo = mid + 1;
    }
    double base = lo > 0 ? tp[lo - 1] : 0.0;
    // no cumulative mass exceeds the target (u * total rounded up to the
    // total): the last pixel, as a search past the end would clamp to
    idx = tp[lo] > target ? -1 : n - 1;
    int64_t last_pos = -1;   // the tile's last pixel with mass, if rounding skips past its end
    for (int k = 0; k < kTile / 32 && idx < 0; ++k) {
      const int64_t p = lo * kTile + k * 32 + lane;
      const double m = p < n ? pixel_mass(d.p, d.h, d.w, p) : 0.0;
      double cum = m;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const double o = __shfl_up_sync(kAll, cum, off);
        if (lane >= off) cum = __dadd_rn(cum, o);
      }
      cum = __dadd_rn(cum, base);
      const unsigned hit = __ballot_sync(kAll, p < n && m > 0.0 && cum > target);
      const unsigned pos = __ballot_sync(kAll, p < n && m > 0.0);
      if (pos) last_pos = lo * kTile + k * 32 + (31 - __clz((int)pos));
      if (hit) idx = lo * kTile + k * 32 + (__ffs((int)hit) - 1);
      base = __shfl_sync(kAll, cum, 31);
    }
    if (idx < 0) idx = last_pos >= 0 ? last_pos : lo * kTile;
  }
  if (lane == 0) {
    const int r = (int)(idx / d.w), c = (int)(idx % d.w);
    int top = r - ch / 2, left = c - cw / 2;
    top = top < 0 ? 0 : (top > d.h - ch ? d.h - ch : top);
    left = left < 0 ? 0 : (left > d.w - cw ? d.w - cw : left);
    win[dr * 4 + 0] = r;
    win[dr * 4 + 1] = c;
    win[dr * 4 + 2] = top;
    win[dr * 4 + 3] = left;
  }
}

// crops[dr][y][x] = image(top + y, left + x); one thread per output pixel.
__global__ void k_crop_gather(const ImgDesc* __restrict__ im, const int32_t* __restrict__ win, int64_t n_draws,
                              int draws_per_image, int ch, int cw, float* __restrict__ crops) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)ch * cw;
  if (t >= n_draws * per) return;
  const int64_t dr = t / per;
  const int y = (int)((t % per) / cw), x = (int)(t % cw);
  const ImgDesc d = im[dr / draws_per_image];
  crops[t] = d.p[(size_t)(win[dr * 4 + 2] + y) * d.w + win[dr * 4 + 3] + x];
}

zoom_status fail(zoom_status s, const std::string& m) {
  zoom_set_error(m);
  return s;
}

}  // namespace

extern "C" zoom_status zoom_sample_crops(zoom_ctx ctx, const float* const* images, const int32_t* heights,
                                         const int32_t* widths, int32_t n_images, const double* u,
                                         int32_t draws_per_image, int32_t crop_h, int32_t crop_w,
                                         int32_t* windows, float* crops, void* stream) {
  if (!ctx || !images || !heights || !widths || !u || !windows) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  if (n_images < 1 || draws_per_image < 1 || (int64_t)n_images * draws_per_image > (1LL << 26))
    return fail(ZOOM_ERR_INVALID_ARG, "n_images and draws_per_image must be positive (at most 2^26 draws)");
  if (crop_h < 1 || crop_w < 1) return fail(ZOOM_ERR_INVALID_ARG, "crop sides must be positive");
  std::vector<ImgDesc> hd(n_images);
  int64_t n_tiles = 0;
  for (int m = 0; m < n_images; ++m) {
    if (!images[m]) return fail(ZOOM_ERR_INVALID_ARG, "NULL image pointer");
    if (heights[m] < crop_h || widths[m] < crop_w)
      return fail(ZOOM_ERR_INVALID_ARG, "image " + std::to_string(m) + " is smaller than the crop");
    hd[m] = {images[m], heights[m], widths[m], n_tiles};
    n_tiles += ((int64_t)heights[m] * widths[m] + kTile - 1) / kTile;
  }
  const int64_t n_draws = (int64_t)n_images * draws_per_image;
  for (int64_t j = 0; j < n_draws; ++j)
    if (!(u[j] >= 0.0 && u[j] < 1.0)) return fail(ZOOM_ERR_INVALID_ARG, "draws must lie in [0, 1)");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ZOOM_ERR_CUDA, "cudaSetDevice");
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_im = al(n_images * sizeof(ImgDesc)), b_ts = al(n_tiles * 8), b_u = al(n_draws * 8),
               b_win = al(n_draws * 16);
  const size_t bytes = b_im + b_ts + b_u + b_win;
  char* mem = (char*)zoom_alloc(ctx, bytes, st);
  if (!mem) return fail(ZOOM_ERR_OOM, "crop-sampling scratch");
  ImgDesc* d_im = (ImgDesc*)mem;
  double* d_ts = (double*)(mem + b_im);
  double* d_u = (double*)(mem + b_im + b_ts);
  int32_t* d_win = (int32_t*)(mem + b_im + b_ts + b_u);
  cudaError_t e = cudaMemcpyAsync(d_im, hd.data(), n_images * sizeof(ImgDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_u, u, n_draws * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_tile_mass<<<(unsigned)((n_tiles * 32 + 255) / 256), 256, 0, st>>>(d_im, n_images, n_tiles, d_ts);
    k_tile_prefix<<<(n_images + 127) / 128, 128, 0, st>>>(d_im, n_images, d_ts);
    k_draw<<<(unsigned)((n_draws * 32 + 255) / 256), 256, 0, st>>>(d_im, d_ts, d_u, n_draws, draws_per_image,
                                                                   crop_h, crop_w, d_win);
    if (crops) {
      const int64_t tot = n_draws * crop_h * crop_w;
      k_crop_gather<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(d_im, d_win, n_draws, draws_per_image, crop_h,
                                                                   crop_w, crops);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(windows, d_win, n_draws * 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  zoom_free(ctx, mem, bytes, st);
  if (e != cudaSuccess) return fail(ZOOM_ERR_CUDA, std::string("crop sampling: ") + cudaGetErrorString(e));
  return ZOOM_OK;
}
