// Dictionary and LSH index construction (Sec. 2.1, Sec. 3.2, Sec. 4.1).
#include <math.h>

#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "zoom_internal.h"

namespace {

constexpr int kMaxScale = 4;

// Combined blur+box weights of one output pixel, W_a * W_b over the
// (s+2) x (s+2) window, as unevaluated float pairs hi + lo.
struct PairWeights {
  int n;  // s + 2
  float hi[(kMaxScale + 2) * (kMaxScale + 2)];
  float lo[(kMaxScale + 2) * (kMaxScale + 2)];
};

// 1-D weights of "3-tap Gaussian then s-box mean": output i reads input
// s*i + a - 1, a in [0, s+2), with weight (1/s) * sum_{b + u = a} taps[u].
void degrade_weights_1d(int s, double sigma, double* wts) {
  double e = exp(-1.0 / (2.0 * sigma * sigma));
  double t[3] = {e / (1.0 + 2.0 * e), 1.0 / (1.0 + 2.0 * e), e / (1.0 + 2.0 * e)};
  for (int a = 0; a < s + 2; ++a) wts[a] = 0.0;
  for (int b = 0; b < s; ++b)
    for (int u = 0; u < 3; ++u) wts[b + u] += t[u] / s;
}

// LR[i][j] = sum_{a,b} W_a W_b HR[clamp(s i + a - 1)][clamp(s j + b - 1)],
// accumulated as a float pair (two-sum / fma two-product) so that the final
// float is the correctly rounded value of the exact sum in all but
// vanishingly rare cases.  The dictionary stores this rounded LR image.
__global__ void k_degrade_exact(const float* __restrict__ hr, int H, int W, int s, PairWeights pw,
                                float* __restrict__ lr, int h, int w) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= h || j >= w) return;
  float shi = 0.f, slo = 0.f;
  for (int a = 0; a < pw.n; ++a) {
    int r = zoom_clampi(s * i + a - 1, 0, H - 1);
    for (int b = 0; b < pw.n; ++b) {
      int c = zoom_clampi(s * j + b - 1, 0, W - 1);
      float x = hr[(size_t)r * W + c];
      float whi = pw.hi[a * pw.n + b], wlo = pw.lo[a * pw.n + b];
      float p = x * whi;
      float pe = fmaf(x, whi, -p);
      pe = fmaf(x, wlo, pe);
      float t = shi + p;
      float bp = t - shi;
      float err = (shi - (t - bp)) + (p - bp);
      shi = t;
      slo += err + pe;
    }
  }
  lr[(size_t)i * w + j] = shi + slo;
}

template <int P, int F>
__global__ void k_dict_gather(const float* const* __restrict__ lr_images,
                              const int32_t* __restrict__ lr_h, const int32_t* __restrict__ lr_w,
                              const float* const* __restrict__ hr_images,
                              const int32_t* __restrict__ hr_w, const int32_t* __restrict__ pos,
                              int64_t n, int s, int dpad, int ph2pad, float* __restrict__ lr_pix,
                              float* __restrict__ feat, float* __restrict__ mu,
                              float* __restrict__ norm2, float* __restrict__ hr_res) {
  constexpr int P2 = P * P;
  constexpr int D = zoom_feature_dim(P, F);
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  int m = pos[e * 3 + 0], i = pos[e * 3 + 1], j = pos[e * 3 + 2];
  const float* lr = lr_images[m];
  int lw = lr_w[m];
  float px[P2], v[P2], mean, n2;
#pragma unroll
  for (int a = 0; a < P; ++a)
#pragma unroll
    for (int b = 0; b < P; ++b) px[a * P + b] = lr[(size_t)(i + a) * lw + j + b];
  zoom_patch_feature<P2>(px, v, mean, n2);
#pragma unroll
  for (int q = 0; q < P2; ++q) lr_pix[e * P2 + q] = px[q];
  if constexpr (F == 0) {
    for (int q = 0; q < dpad; ++q) feat[e * dpad + q] = q < D ? v[q] : 0.f;
  } else {
    float g[D];
    zoom_gradient_feature<P, F>(lr, lr_h[m], lw, (size_t)lw, i, j, g, n2);
    for (int q = 0; q < dpad; ++q) feat[e * dpad + q] = q < D ? g[q] : 0.f;
  }
  mu[e] = mean;
  norm2[e] = n2;
  const float* hr = hr_images[m];
  int hw = hr_w[m];
  int PH = s * P;
  for (int a = 0; a < PH; ++a)
    for (int b = 0; b < PH; ++b)
      hr_res[e * ph2pad + a * PH + b] = hr[(size_t)(s * i + a) * hw + s * j + b] - mean;
  for (int q = PH * PH; q < ph2pad; ++q) hr_res[e * ph2pad + q] = 0.f;
}

// Eq. 10 for every projection and the key fold of every table; one thread
// per feature row.  alpha/beta are staged in shared memory.
template <int D>
__global__ void k_hash(const float* __restrict__ feat, int dpad, int64_t n,
                       const float* __restrict__ alpha, const float* __restrict__ beta, int L, int k,
                       float w, uint64_t* __restrict__ keys) {
  // projections staged with rows padded to DP floats (16-byte loads; the
  // multiply-adds keep the order of the feature's values)
  constexpr int DP = (D + 3) / 4 * 4;
  extern __shared__ float4 s_ab4[];
  float* s_ab = reinterpret_cast<float*>(s_ab4);
  int nproj = L * k;
  for (int t = threadIdx.x; t < nproj * DP; t += blockDim.x) {
    const int pj = t / DP, q = t % DP;
    s_ab[t] = q < D ? alpha[pj * D + q] : 0.f;
  }
  for (int t = threadIdx.x; t < nproj; t += blockDim.x) s_ab[nproj * DP + t] = beta[t];
  __syncthreads();
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float v[DP];
#pragma unroll
  for (int q = 0; q < DP; ++q) v[q] = q < D ? feat[r * dpad + q] : 0.f;
  const float* s_beta = s_ab + nproj * DP;
  for (int l = 0; l < L; ++l) {
    uint64_t x = (uint64_t)l;
    for (int j = 0; j < k; ++j) {
      const float4* a4 = s_ab4 + (l * k + j) * (DP / 4);
      float acc = 0.f;
#pragma unroll
      for (int q4 = 0; q4 < DP / 4; ++q4) {
        const float4 av = a4[q4];
        acc = fmaf(av.x, v[4 * q4], acc);
        if (4 * q4 + 1 < D) acc = fmaf(av.y, v[4 * q4 + 1], acc);
        if (4 * q4 + 2 < D) acc = fmaf(av.z, v[4 * q4 + 2], acc);
        if (4 * q4 + 3 < D) acc = fmaf(av.w, v[4 * q4 + 3], acc);
      }
      float t = acc + s_beta[l * k + j];
      int h = (int)floorf(__fdiv_rn(t, w));
      x = zoom_fold_step(x, h, j);
    }
    keys[r * L + l] = x;
  }
}

// ---------------------------------------------------------------------------
// LSD radix sort of (uint64 key, int32 id) pairs, 8 bits per pass, stable.
// ---------------------------------------------------------------------------

constexpr int RS_THREADS = 256;
constexpr int RS_TILE = 4096;
constexpr int SCAN_SEG = 4096;

__global__ void k_extract_column(const uint64_t* __restrict__ src, int L, int l, int64_t n,
                                 uint64_t* __restrict__ keys, int32_t* __restrict__ ids) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = src[i * L + l];
  ids[i] = (int32_t)i;
}

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                             int32_t* __restrict__ hist, int ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  // lanes of equal digit add their count once (digits of compacted ranks
  // take few values, which would pile the atomics onto a few counters)
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  for (int t = threadIdx.x; t < RS_TILE; t += RS_THREADS) {
    int64_t g = base + t;
    const int digit = g < n ? (int)((keys[g] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    if (digit < 256 && (peers & lt) == 0) atomicAdd(&h[digit], __popc(peers));
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items of a tile are ranked in index order.  The tile is
// processed in chunks of 256 (one item per thread); within a chunk,
// __match_any_sync groups lanes of equal digit, and per-digit prefix counts
// over the warps give each item its place after all earlier items.
__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                                int shift, const int32_t* __restrict__ offs, int ntiles) {
  __shared__ int run[256];
  __shared__ int wh[RS_THREADS / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < RS_TILE / RS_THREADS; ++c) {
    int64_t g = (int64_t)blockIdx.x * RS_TILE + c * RS_THREADS + tid;
    bool valid = g < n;
    uint64_t key = valid ? kin[g] : 0ull;
    int32_t val = valid ? vin[g] : 0;
    int digit = valid ? (int)((key >> shift) & 255) : 256;
    for (int q = tid; q < (RS_THREADS / 32) * 256; q += RS_THREADS) (&wh[0][0])[q] = 0;
    __syncthreads();
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & lt);
    if (valid && rank == 0) wh[warp][digit] = __popc(peers);
    __syncthreads();
    {
      int s = run[tid];
#pragma unroll
      for (int q = 0; q < RS_THREADS / 32; ++q) {
        int t = wh[q][tid];
        wh[q][tid] = s;
        s += t;
      }
      run[tid] = s;
    }
    __syncthreads();
    if (valid) {
      int p = wh[warp][digit] + rank;
      kout[p] = key;
      vout[p] = val;
    }
    __syncthreads();
  }
}

// Exclusive scan of int32 in three phases: per-segment sums, a one-block
// scan of the sums, per-segment scans with the segment offset.
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  int excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0);
  total = s_warp[nw - 1];
  __syncthreads();
  return excl;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ part) {
  __shared__ int s_warp[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_SEG;
  int acc = 0;
  for (int t = threadIdx.x; t < SCAN_SEG; t += blockDim.x) {
    int64_t g = base + t;
    if (g < n) acc += in[g];
  }
  int total;
  block_exclusive_scan(acc, s_warp, total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void k_scan_partials(int32_t* __restrict__ part, int np) {
  __shared__ int s_warp[32];
  // each thread scans a contiguous run of parts sequentially
  const int per = (np + blockDim.x - 1) / blockDim.x;
  int b0 = threadIdx.x * per;
  int acc = 0;
  for (int q = 0; q < per; ++q)
    if (b0 + q < np) acc += part[b0 + q];
  int total;
  int ex = block_exclusive_scan(acc, s_warp, total);
  for (int q = 0; q < per; ++q)
    if (b0 + q < np) {
      int t = part[b0 + q];
      part[b0 + q] = ex;
      ex += t;
    }
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ part,
                             int32_t* __restrict__ out) {
  __shared__ int s_warp[32];
  constexpr int PER = SCAN_SEG / 256;  // launched with 256 threads
  int64_t base = (int64_t)blockIdx.x * SCAN_SEG + threadIdx.x * PER;
  int v[PER];
  int acc = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int64_t g = base + q;
    v[q] = g < n ? in[g] : 0;
    acc += v[q];
  }
  int total;
  int ex = block_exclusive_scan(acc, s_warp, total) + part[blockIdx.x];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int64_t g = base + q;
    if (g < n) out[g] = ex;
    ex += v[q];
  }
}

cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* part, cudaStream_t st) {
  int nseg = (int)((n + SCAN_SEG - 1) / SCAN_SEG);
  k_scan_reduce<<<nseg, 256, 0, st>>>(in, n, part);
  k_scan_partials<<<1, 1024, 0, st>>>(part, nseg);
  k_scan_apply<<<nseg, 256, 0, st>>>(in, n, part, out);
  return cudaGetLastError();
}

__global__ void k_csr_heads(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ head) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_csr_write(const uint64_t* __restrict__ keys, const int32_t* __restrict__ head,
                            const int32_t* __restrict__ pos, int64_t n, uint64_t* __restrict__ ukeys,
                            int32_t* __restrict__ offs, int32_t* __restrict__ nuniq) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (head[i]) {
    ukeys[pos[i]] = keys[i];
    offs[pos[i]] = (int32_t)i;
  }
  if (i == n - 1) {
    int32_t u = pos[i] + head[i];
    offs[u] = (int32_t)n;
    *nuniq = u;
  }
}

// ---------------------------------------------------------------------------
// Key compaction for the bins (a3): a table of N entries holds few distinct
// keys (68 to 661 per table with 1M pairs), so the 64-bit keys are replaced by
// their rank among the table's distinct keys, and the stable sort by key
// becomes a stable sort by a 12-bit rank: 2 radix passes of 8 bits instead
// of 8.  Distinct keys go into a small open-addressing set per table (linear
// probing, a slot claimed by a 64-bit compare-and-swap; the one key equal to
// the empty marker is recorded by a flag); one block per table sorts them in
// shared memory and gives every slot its rank.  A table with more distinct
// keys than kKeySetCap keeps the 64-bit radix sort.
// ---------------------------------------------------------------------------
constexpr int kKeySetCap = 4096;            // distinct keys per table for the compacted sort
constexpr int kKeySetSlots = 2 * kKeySetCap;
constexpr uint64_t kEmptyKey = ~0ull;

__device__ __forceinline__ uint32_t keyset_hash(uint64_t k) {
  k ^= k >> 31;
  k *= 0x7FB5D329728EA185ull;
  return (uint32_t)(k >> 51) & (kKeySetSlots - 1);
}

// One thread per entry: its L keys (one 128-byte row) into the L sets.
__global__ void k_keyset_insert(const uint64_t* __restrict__ dkeys, int64_t n, int L, uint64_t* slots,
                                uint32_t* __restrict__ count, uint32_t* __restrict__ eflag,
                                uint32_t* __restrict__ full) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int l = 0; l < L; ++l) {
    const uint64_t key = dkeys[i * L + l];
    if (key == kEmptyKey) {
      if (atomicOr(eflag + l, 1u) == 0u) atomicAdd(count + l, 1u);
      continue;
    }
    uint64_t* set = slots + (int64_t)l * kKeySetSlots;
    uint32_t h = keyset_hash(key);
    int p = 0;
    for (; p < kKeySetSlots; ++p, h = (h + 1) & (kKeySetSlots - 1)) {
      const uint64_t cur = *(volatile uint64_t*)(set + h);
      if (cur == key) break;
      if (cur == kEmptyKey) {
        const unsigned long long old = atomicCAS((unsigned long long*)(set + h), (unsigned long long)kEmptyKey,
                                                 (unsigned long long)key);
        if (old == kEmptyKey) {
          atomicAdd(count + l, 1u);
          break;
        }
        if (old == key) break;
      }
    }
    if (p == kKeySetSlots) atomicOr(full + l, 1u);   // no free slot left: the table keeps the 64-bit sort
  }
}

// One block (1024 threads) per table with at most kKeySetCap distinct keys:
// the set's keys sorted ascending (bitonic, in shared memory) into ukeys,
// and the rank of each slot's key (and of the empty-marker key) recorded.
__global__ void __launch_bounds__(1024) k_keyset_rank(const uint64_t* __restrict__ slots,
                                                      const uint32_t* __restrict__ eflag,
                                                      const uint32_t* __restrict__ compact, int64_t n,
                                                      uint64_t* __restrict__ ukeys, int32_t* __restrict__ nuniq,
                                                      uint16_t* __restrict__ slot_rank,
                                                      uint16_t* __restrict__ erank) {
  __shared__ uint64_t sk[kKeySetCap];
  __shared__ uint16_t ss[kKeySetCap];   // slot of each key (kKeySetSlots: the empty-marker key)
  __shared__ int m;
  const int l = blockIdx.x;
  if (!compact[l]) return;   // block-uniform
  if (threadIdx.x == 0) m = 0;
  __syncthreads();
  const uint64_t* set = slots + (int64_t)l * kKeySetSlots;
  for (int h = threadIdx.x; h < kKeySetSlots; h += blockDim.x) {
    const uint64_t k = set[h];
    if (k != kEmptyKey) {
      const int j = atomicAdd(&m, 1);
      sk[j] = k;
      ss[j] = h;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && eflag[l]) {   // the empty-marker key is the largest of all
    sk[m] = kEmptyKey;
    ss[m] = kKeySetSlots;
    ++m;
  }
  __syncthreads();
  const int u = m;
  int pw = 1;
  while (pw < u) pw <<= 1;
  for (int j = u + threadIdx.x; j < pw; j += blockDim.x) {   // padding sorts after every real key
    sk[j] = kEmptyKey;
    ss[j] = 0xFFFF;
  }
  __syncthreads();
  for (int k = 2; k <= pw; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < pw; i += blockDim.x) {
        const int o = i ^ j;
        if (o > i) {
          const bool up = (i & k) == 0;
          const bool gt = sk[i] > sk[o] || (sk[i] == sk[o] && ss[i] > ss[o]);
          if (gt == up) {
            const uint64_t tk = sk[i];
            sk[i] = sk[o];
            sk[o] = tk;
            const uint16_t ts = ss[i];
            ss[i] = ss[o];
            ss[o] = ts;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < u; r += blockDim.x) {
    ukeys[(int64_t)l * n + r] = sk[r];
    if (ss[r] < kKeySetSlots) slot_rank[(int64_t)l * kKeySetSlots + ss[r]] = (uint16_t)r;
    else erank[l] = (uint16_t)r;
  }
  if (threadIdx.x == 0) nuniq[l] = u;
}

// One thread per entry: the rank of each of its keys in its table's set
// (compacted tables only).
__global__ void k_keyset_lookup(const uint64_t* __restrict__ dkeys, int64_t n, int L,
                                const uint64_t* __restrict__ slots, const uint16_t* __restrict__ slot_rank,
                                const uint16_t* __restrict__ erank, const uint32_t* __restrict__ compact,
                                uint16_t* __restrict__ rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int l = 0; l < L; ++l) {
    if (!compact[l]) continue;
    const uint64_t key = dkeys[i * L + l];
    uint16_t r = 0;
    if (key == kEmptyKey) {
      r = erank[l];
    } else {
      const uint64_t* set = slots + (int64_t)l * kKeySetSlots;
      uint32_t h = keyset_hash(key);
      for (int p = 0; p < kKeySetSlots; ++p, h = (h + 1) & (kKeySetSlots - 1)) {
        if (set[h] == key) {
          r = slot_rank[(int64_t)l * kKeySetSlots + h];
          break;
        }
      }
    }
    rank[(int64_t)l * n + i] = r;
  }
}

__global__ void k_rank_pairs(const uint16_t* __restrict__ rank, int64_t n, uint64_t* __restrict__ keys,
                             int32_t* __restrict__ ids) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = rank[i];
  ids[i] = (int32_t)i;
}

// The same stable radix sort by rank for every table at once (blockIdx.y:
// the table).  The histogram is laid out [table][digit][tile], so one
// exclusive scan over all of it gives each item its position in the
// concatenated [table][n] output: a table's items land after every earlier
// table's n items.  ids_in == nullptr: the items' ids are their indices.
__global__ void k_rank_hist_b(const uint16_t* __restrict__ r, int64_t n, int shift, int32_t* __restrict__ hist,
                              int ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint16_t* rt = r + (int64_t)blockIdx.y * n;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  for (int t = threadIdx.x; t < RS_TILE; t += RS_THREADS) {
    const int64_t g = base + t;
    const int digit = g < n ? (int)((rt[g] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    if (digit < 256 && (peers & lt) == 0) atomicAdd(&h[digit], __popc(peers));
  }
  __syncthreads();
  hist[((int64_t)blockIdx.y * 256 + threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rank_scatter_b(const uint16_t* __restrict__ rin, const int32_t* __restrict__ ids_in,
                                 uint16_t* __restrict__ rout, int32_t* __restrict__ ids_out, int64_t n, int shift,
                                 const int32_t* __restrict__ offs, int ntiles) {
  __shared__ int run[256];
  __shared__ int wh[RS_THREADS / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t tb = (int64_t)blockIdx.y * n;   // this table's slice of the inputs
  run[tid] = offs[((int64_t)blockIdx.y * 256 + tid) * ntiles + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < RS_TILE / RS_THREADS; ++c) {
    const int64_t g = (int64_t)blockIdx.x * RS_TILE + c * RS_THREADS + tid;
    const bool valid = g < n;
    const uint16_t key = valid ? rin[tb + g] : 0;
    const int32_t val = valid ? (ids_in ? ids_in[tb + g] : (int32_t)g) : 0;
    const int digit = valid ? (int)((key >> shift) & 255) : 256;
    for (int q = tid; q < (RS_THREADS / 32) * 256; q += RS_THREADS) (&wh[0][0])[q] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wh[warp][digit] = __popc(peers);
    __syncthreads();
    {
      int sacc = run[tid];
#pragma unroll
      for (int q = 0; q < RS_THREADS / 32; ++q) {
        const int t = wh[q][tid];
        wh[q][tid] = sacc;
        sacc += t;
      }
      run[tid] = sacc;
    }
    __syncthreads();
    if (valid) {
      const int64_t pos = (int64_t)wh[warp][digit] + rank;
      rout[pos] = key;
      ids_out[pos] = val;
    }
    __syncthreads();
  }
}

// Bin offsets of every table from its rank-sorted ranks (blockIdx.y: table).
__global__ void k_csr_rank_offsets_b(const uint16_t* __restrict__ r, int64_t n, int32_t* __restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint16_t* rt = r + (int64_t)blockIdx.y * n;
  int32_t* ot = offs + (int64_t)blockIdx.y * (n + 1);
  if (i == 0 || rt[i] != rt[i - 1]) ot[rt[i]] = (int32_t)i;
  if (i == n - 1) ot[rt[i] + 1] = (int32_t)n;
}

// Offsets of the runs of a rank-sorted table (its keys already written by
// k_keyset_rank): a run starts where the rank changes, and the rank is the
// run's index.
__global__ void k_csr_rank_offsets(const uint64_t* __restrict__ r, int64_t n, int32_t* __restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i == 0 || r[i] != r[i - 1]) offs[r[i]] = (int32_t)i;
  if (i == n - 1) offs[r[i] + 1] = (int32_t)n;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_degrade_exact(const float* hr, int H, int W, int s, double sigma, float* lr,
                                 cudaStream_t st) {
  double w1[kMaxScale + 2];
  degrade_weights_1d(s, sigma, w1);
  PairWeights pw;
  pw.n = s + 2;
  for (int a = 0; a < s + 2; ++a)
    for (int b = 0; b < s + 2; ++b) {
      double p = w1[a] * w1[b];
      float hi = (float)p;
      pw.hi[a * pw.n + b] = hi;
      pw.lo[a * pw.n + b] = (float)(p - (double)hi);
    }
  int h = H / s, w = W / s;
  dim3 blk(32, 8), grd((w + 31) / 32, (h + 7) / 8);
  k_degrade_exact<<<grd, blk, 0, st>>>(hr, H, W, s, pw, lr, h, w);
  return cudaGetLastError();
}

cudaError_t launch_dict_gather(const float* const* d_lr_images, const int32_t* d_lr_h,
                               const int32_t* d_lr_w, const float* const* d_hr_images,
                               const int32_t* d_hr_w, const int32_t* d_pos, int64_t n, int P, int s,
                               zoom_dict d, cudaStream_t st) {
  int blocks = (int)((n + 127) / 128);
#define ZOOM_GATHER(PP, FF)                                                                     \
  k_dict_gather<PP, FF><<<blocks, 128, 0, st>>>(d_lr_images, d_lr_h, d_lr_w, d_hr_images, d_hr_w, \
                                                d_pos, n, s, d->dpad, d->ph2pad, d->lr_pix,      \
                                                d->feat, d->mu, d->norm2, d->hr_res)
  if (P == 3 && d->feature == 0) ZOOM_GATHER(3, 0);
  else if (P == 5 && d->feature == 0) ZOOM_GATHER(5, 0);
  else if (P == 3 && d->feature == 1) ZOOM_GATHER(3, 1);
  else if (P == 5 && d->feature == 1) ZOOM_GATHER(5, 1);
  else if (P == 3 && d->feature == 2) ZOOM_GATHER(3, 2);
  else if (P == 5 && d->feature == 2) ZOOM_GATHER(5, 2);
  else return cudaErrorInvalidValue;
#undef ZOOM_GATHER
  return cudaGetLastError();
}

cudaError_t launch_hash(const float* feat, int dpad, int d, int64_t n, const float* alpha,
                        const float* beta, int L, int k, float w, uint64_t* keys, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  size_t smem = (size_t)L * k * ((d + 3) / 4 * 4 + 1) * sizeof(float);
  int blocks = (int)((n + 127) / 128);
#define ZOOM_HASH(DD)                                                                       \
  do {                                                                                      \
    if (smem > 48 * 1024)                                                                   \
      cudaFuncSetAttribute(k_hash<DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    k_hash<DD><<<blocks, 128, smem, st>>>(feat, dpad, n, alpha, beta, L, k, w, keys);        \
  } while (0)
  switch (d) {
    case 9: ZOOM_HASH(9); break;
    case 25: ZOOM_HASH(25); break;
    case 18: ZOOM_HASH(18); break;
    case 50: ZOOM_HASH(50); break;
    default: return cudaErrorInvalidValue;
  }
#undef ZOOM_HASH
  return cudaGetLastError();
}

namespace {
__global__ void k_make_pairs(const int32_t* __restrict__ keys32, int64_t n, uint64_t* __restrict__ keys,
                             int32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = (uint64_t)(uint32_t)keys32[i];
  vals[i] = (int32_t)i;
}
}  // namespace

// Stable sort of the positions 0..n-1 by a non-negative int32 key, then the
// CSR of equal-key runs: sorted_pos[n] (positions grouped by key, ascending
// within a run), ukeys[u] (run keys, ascending), offs[u+1], *nuniq = u.
cudaError_t sort_keys_csr(const int32_t* keys32, int64_t n, int32_t* sorted_pos, uint64_t* ukeys,
                          int32_t* offs, int32_t* nuniq, void* scratch, size_t scratch_bytes,
                          cudaStream_t st) {
  if (scratch_bytes < csr_scratch_bytes(n)) return cudaErrorInvalidValue;
  const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
  char* p = (char*)scratch;
  uint64_t* ka = (uint64_t*)p; p += n * 8;
  uint64_t* kb = (uint64_t*)p; p += n * 8;
  int32_t* va = (int32_t*)p; p += n * 4;
  int32_t* vb = (int32_t*)p; p += n * 4;
  int32_t* hist = (int32_t*)p; p += (int64_t)256 * ntiles * 4;
  int32_t* head = (int32_t*)p; p += n * 4;
  int32_t* pos = (int32_t*)p; p += n * 4;
  int32_t* part = (int32_t*)p;
  const int eb = (int)((n + 255) / 256);
  k_make_pairs<<<eb, 256, 0, st>>>(keys32, n, ka, va);
  uint64_t* kin = ka; uint64_t* kout = kb;
  int32_t* vin = va; int32_t* vout = vb;
  for (int shift = 0; shift < 32; shift += 8) {   // keys fit in 32 bits
    k_radix_hist<<<ntiles, RS_THREADS, 0, st>>>(kin, n, shift, hist, ntiles);
    cudaError_t e = exclusive_scan(hist, hist, (int64_t)256 * ntiles, part, st);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<ntiles, RS_THREADS, 0, st>>>(kin, vin, kout, vout, n, shift, hist, ntiles);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  k_csr_heads<<<eb, 256, 0, st>>>(kin, n, head);
  cudaError_t e = exclusive_scan(head, pos, n, part, st);
  if (e != cudaSuccess) return e;
  k_csr_write<<<eb, 256, 0, st>>>(kin, head, pos, n, ukeys, offs, nuniq);
  cudaMemcpyAsync(sorted_pos, vin, n * 4, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

size_t csr_scratch_bytes(int64_t n) {
  int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  int64_t hist = 256 * ntiles;
  int64_t nseg = (std::max<int64_t>(hist, n) + SCAN_SEG - 1) / SCAN_SEG;
  // keys x2, ids x2, hist, head, pos, parts
  return (size_t)(2 * n * 8 + 2 * n * 4 + hist * 4 + 2 * n * 4 + nseg * 4 + 1024);
}

size_t csr_build_scratch_bytes(int64_t n, int L) {
  // the radix sort's buffers, then the key sets, the slot ranks, the per-table
  // flags, the 16-bit ranks of every entry in every table (twice) and their
  // ids, and the all-table histogram with its scan partials
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  const int64_t hist = (int64_t)L * 256 * ntiles;
  return csr_scratch_bytes(n) + 256 + (size_t)L * kKeySetSlots * 8 + (size_t)L * kKeySetSlots * 2 +
         (size_t)5 * L * 4 + 256 + (size_t)L * n * 2 + 256 + (size_t)L * n * 2 + 256 + (size_t)L * n * 4 + 256 +
         (size_t)hist * 4 + 256 + (size_t)((hist + SCAN_SEG - 1) / SCAN_SEG) * 4 + 1024;
}

cudaError_t build_csr_tables(zoom_index ix, void* scratch, size_t scratch_bytes, cudaStream_t st) {
  const int64_t n = ix->dict->n;
  const int L = ix->L;
  if (scratch_bytes < csr_build_scratch_bytes(n, L)) return cudaErrorInvalidValue;
  const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
  char* p = (char*)scratch;
  uint64_t* ka = (uint64_t*)p; p += n * 8;
  uint64_t* kb = (uint64_t*)p; p += n * 8;
  int32_t* va = (int32_t*)p; p += n * 4;
  int32_t* vb = (int32_t*)p; p += n * 4;
  int32_t* hist = (int32_t*)p; p += (int64_t)256 * ntiles * 4;
  int32_t* head = (int32_t*)p; p += n * 4;
  int32_t* pos = (int32_t*)p; p += n * 4;
  int32_t* part = (int32_t*)p;
  // compaction arrays after the radix sort's (csr_scratch_bytes(n) of them)
  char* q = (char*)scratch + ((csr_scratch_bytes(n) + 255) & ~(size_t)255);
  uint64_t* slots = (uint64_t*)q; q += (size_t)L * kKeySetSlots * 8;
  uint16_t* slot_rank = (uint16_t*)q; q += (size_t)L * kKeySetSlots * 2;
  uint32_t* flags = (uint32_t*)q; q += (size_t)5 * L * 4;   // count, eflag, full, compact, erank (16-bit)
  uint32_t* count = flags;
  uint32_t* eflag = flags + L;
  uint32_t* full = flags + 2 * L;
  uint32_t* compact = flags + 3 * L;
  uint16_t* erank = (uint16_t*)(flags + 4 * L);
  q = (char*)(((uintptr_t)q + 255) & ~(uintptr_t)255);
  uint16_t* rank = (uint16_t*)q; q += (size_t)L * n * 2;
  q = (char*)(((uintptr_t)q + 255) & ~(uintptr_t)255);
  uint16_t* rank_b = (uint16_t*)q; q += (size_t)L * n * 2;
  q = (char*)(((uintptr_t)q + 255) & ~(uintptr_t)255);
  int32_t* ids_b = (int32_t*)q; q += (size_t)L * n * 4;
  q = (char*)(((uintptr_t)q + 255) & ~(uintptr_t)255);
  int32_t* hist_b = (int32_t*)q; q += (size_t)L * 256 * ntiles * 4;
  q = (char*)(((uintptr_t)q + 255) & ~(uintptr_t)255);
  int32_t* part_b = (int32_t*)q;
  const int eb = (int)((n + 255) / 256);

  // distinct keys per table; the host reads the counts (the build ends with
  // a stream synchronisation anyway)
  cudaError_t e = cudaMemsetAsync(slots, 0xFF, (size_t)L * kKeySetSlots * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, (size_t)5 * L * 4, st);
  if (e != cudaSuccess) return e;
  k_keyset_insert<<<eb, 256, 0, st>>>(ix->dkeys, n, L, slots, count, eflag, full);
  std::vector<uint32_t> h_flags((size_t)3 * L);
  e = cudaMemcpyAsync(h_flags.data(), flags, (size_t)3 * L * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  std::vector<uint32_t> h_compact(L);
  bool any = false;
  for (int l = 0; l < L; ++l) {
    h_compact[l] = h_flags[2 * L + l] == 0 && h_flags[l] <= (uint32_t)kKeySetCap ? 1u : 0u;
    any = any || h_compact[l];
  }
  if (any) {
    e = cudaMemcpyAsync(compact, h_compact.data(), (size_t)L * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_keyset_rank<<<L, 1024, 0, st>>>(slots, eflag, compact, n, ix->ukeys, ix->nuniq, slot_rank, erank);
    k_keyset_lookup<<<eb, 256, 0, st>>>(ix->dkeys, n, L, slots, slot_rank, erank, compact, rank);
    // the copy of h_compact must finish before the vector goes
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
  }
  bool all = true;
  uint32_t umax = 0;
  for (int l = 0; l < L; ++l) {
    all = all && h_compact[l];
    umax = std::max(umax, h_flags[l]);
  }
  if (all && (int64_t)L * n < (int64_t{1} << 31)) {   // positions in 32-bit scans
    // every table at once: 1 pass of 8 bits when no table has more than 256
    // distinct keys, else 2; the last pass writes the ids into the index
    const int passes = umax <= 256u ? 1 : 2;
    const dim3 grid(ntiles, L);
    const uint16_t* rin = rank;
    uint16_t* rout = rank_b;
    const int32_t* iin = nullptr;
    for (int ps = 0; ps < passes; ++ps) {
      int32_t* iout = ps == passes - 1 ? ix->ids : ids_b;
      k_rank_hist_b<<<grid, RS_THREADS, 0, st>>>(rin, n, 8 * ps, hist_b, ntiles);
      e = exclusive_scan(hist_b, hist_b, (int64_t)L * 256 * ntiles, part_b, st);
      if (e != cudaSuccess) return e;
      k_rank_scatter_b<<<grid, RS_THREADS, 0, st>>>(rin, iin, rout, iout, n, 8 * ps, hist_b, ntiles);
      iin = iout;
      rin = rout;
      rout = rout == rank_b ? rank : rank_b;
    }
    k_csr_rank_offsets_b<<<dim3(eb, L), 256, 0, st>>>(rin, n, ix->offs);
    return cudaGetLastError();
  }
  for (int l = 0; l < L; ++l) {
    uint64_t* kin = ka; uint64_t* kout = kb;
    int32_t* vin = va; int32_t* vout = vb;
    if (h_compact[l]) {
      // stable sort of the entries by their rank (below 4096): 2 passes of
      // 8 bits, 1 when the table has at most 256 distinct keys
      k_rank_pairs<<<eb, 256, 0, st>>>(rank + (int64_t)l * n, n, ka, va);
      const int bits = h_flags[l] <= 256u ? 8 : 16;
      for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<ntiles, RS_THREADS, 0, st>>>(kin, n, shift, hist, ntiles);
        e = exclusive_scan(hist, hist, (int64_t)256 * ntiles, part, st);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<ntiles, RS_THREADS, 0, st>>>(kin, vin, kout, vout, n, shift, hist, ntiles);
        std::swap(kin, kout);
        std::swap(vin, vout);
      }
      k_csr_rank_offsets<<<eb, 256, 0, st>>>(kin, n, ix->offs + (int64_t)l * (n + 1));
    } else {
      k_extract_column<<<eb, 256, 0, st>>>(ix->dkeys, L, l, n, ka, va);
      for (int shift = 0; shift < 64; shift += 8) {
        k_radix_hist<<<ntiles, RS_THREADS, 0, st>>>(kin, n, shift, hist, ntiles);
        e = exclusive_scan(hist, hist, (int64_t)256 * ntiles, part, st);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<ntiles, RS_THREADS, 0, st>>>(kin, vin, kout, vout, n, shift, hist, ntiles);
        std::swap(kin, kout);
        std::swap(vin, vout);
      }
      k_csr_heads<<<eb, 256, 0, st>>>(kin, n, head);
      e = exclusive_scan(head, pos, n, part, st);
      if (e != cudaSuccess) return e;
      k_csr_write<<<eb, 256, 0, st>>>(kin, head, pos, n, ix->ukeys + (int64_t)l * n,
                                      ix->offs + (int64_t)l * (n + 1), ix->nuniq + l);
    }
    e = cudaMemcpyAsync(ix->ids + (int64_t)l * n, vin, n * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

