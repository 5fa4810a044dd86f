// Neighbour search on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The candidate set of a query is, at the bin widths of the workloads, most
// of the dictionary, so the search is a dense (queries x dictionary)
// contraction.  A tensor-core pass computes, for every (query, entry) pair,
//   acc = ||c||^2 - 2 q.c        (d~ = ||q||^2 + acc approximates |q - c|^2)
// and keeps per query, for every dictionary split, the MC 32-entry chunks
// (consecutive entries) with the smallest minimum d~; the minimum of a chunk
// comes with its TMEM load (tcgen05.ld.red), so the epilogue costs one
// comparison per chunk.  Any entry of the top MC lies in one of those chunks.
// A rerank kernel then computes the exact FP32 difference-form distance of
// the entries of the listed chunks in ascending chunk order, tests LSH
// membership and selects the K nearest members.
//
// Three operand forms, one kernel:
// * single-term FP16 (K = 32, or 64 for 50 features): A = [q | 1 1 1],
//   B = [-2c | n1 n2 n3] with ||c||^2 as three FP16 terms; q and c rounded to
//   11 significant bits.  With an error bound delta on |d~ - d|, a query whose
//   K-th exact distance D_K satisfies T - delta > D_K (T: smallest list
//   threshold over the splits) provably has every nearer member inside the
//   listed chunks; the queries it cannot settle are searched again by the
//   split form (on the device's count of them), and what that leaves by the
//   exact SIMT scan.  This is the exact search; its result equals the scan's.
// * FP16 hi/lo split (K = 80, or 160): q = q_hi + q_lo, c = c_hi + c_lo,
//   A row = [q_hi | q_lo | q_hi | 1 | 1 | 0 0 0],
//   B row = [-2c_hi | -2c_hi | -2c_lo | n_hi | n_lo | 0 0 0], so acc misses
//   only -2 q_lo.c_lo (about 2^-22 relative): the same proof with a 30x
//   smaller bound (the second stage, or alone).
// * BF16 (K = 32, or 64): A = [q | 1 1 1 | 0..], B = [-2c | n1 n2 n3 | 0..];
//   the rerank examines the listed chunks until a BF16 error bound rules the
//   rest out, without the proof (the precision form).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <float.h>
#include <type_traits>

#include "device_common.cuh"
#include "zoom_internal.h"

namespace {

// Warp 0 producer, warps 2..9 epilogue, and MMA-issuing warps: one thread
// issues a 128x128x16 MMA in about 75 cycles (the tensor core executes it in
// 64), plus about 250 cycles of waits, fence and commit per tile, so one
// issuing thread per (accumulator buffer, query tile) -- warps 1, 10, 11, 12
// -- keeps the tensor pipe fed at K = 80.  Thirteen warps sit 4/3/3/3 on the
// SM sub-partitions (16K registers each), which caps a thread at 128
// registers: the 32-entry lists do not fit, so they keep two issuing warps (1
// and 10, one per query tile; 11 warps, 168 registers).  So do the narrowest
// operands (K = 32): a tile's MMAs take less time than reading its
// accumulator, and each round of TMEM loads and their wait costs about 200
// cycles whatever its width, so their epilogue reads a tile's 128 columns in
// one round (128 registers) and keeps its chunk list in shared memory (at
// K = 64 the two issuing threads would cost more than the round saves).
__host__ __device__ constexpr bool tc_one_round(int KC, int MC) { return KC <= 4 && MC <= 16; }
__host__ __device__ constexpr int tc_mma_warps(int KC, int MC) {
  return (MC <= 16 && !tc_one_round(KC, MC)) ? 4 : 2;
}
__host__ __device__ constexpr int tc_threads(int KC, int MC) { return (9 + tc_mma_warps(KC, MC)) * 32; }
__host__ __device__ constexpr int tc_max_regs(int KC, int MC) { return tc_mma_warps(KC, MC) == 4 ? 128 : 168; }
constexpr int kBarBytes = 512;
constexpr int TC_ROWS = 128;      // rows per operand tile (M and N of one MMA)
// Per epilogue lane, chunks below the threshold are first appended to a
// shared-memory buffer of tc_buf(KC) slots (a few instructions each) and merged
// into the sorted register list when some lane of the warp runs out of room:
// the merge loop then runs for all lanes together, so the sorted insertions
// execute with the warp converged.  A tile adds at most 4 entries per lane,
// so 8 slots suffice; 16 flush half as often.  The widest operands (K = 160)
// take 8, which frees room for a third ring stage.
__host__ __device__ constexpr int tc_buf(int KC) { return KC >= 20 ? 8 : 16; }
constexpr int kSmemMax = 232448;  // shared memory a CTA may opt into (227 KB)
// shared memory of the epilogue: append buffers, and the lists when they
// live there (value + index per entry and lane)
__host__ __device__ constexpr int tc_epi_bytes(int KC, int MC) {
  return tc_buf(KC) * 256 * 8 + (tc_one_round(KC, MC) ? MC * 256 * 8 : 0);
}
// Dictionary-tile ring depth: as many bulk copies in flight as the shared
// memory left by the two query tiles, the barriers and the epilogue holds, up
// to 16 (KC = 4: 16, 8: 10, 10: 7, 20: 3).
__host__ __device__ constexpr int tc_stages(int KC, int MC) {
  return (kSmemMax - 1024 - kBarBytes - tc_epi_bytes(KC, MC) - 2 * KC * TC_ROWS * 16) / (KC * TC_ROWS * 16) < 16
             ? (kSmemMax - 1024 - kBarBytes - tc_epi_bytes(KC, MC) - 2 * KC * TC_ROWS * 16) / (KC * TC_ROWS * 16)
             : 16;
}
static_assert(tc_stages(4, 16) == 16 && tc_stages(8, 16) == 10 && tc_stages(8, 32) == 10 &&
                  tc_stages(10, 16) == 7 && tc_stages(20, 16) == 3,
              "ring depths");
constexpr uint32_t kWaitNs = 2000000000u;   // 2 s bound on any single wait

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// As mbar_try_wait, but the thread may sleep in hardware until the phase
// completes or about `hint_ns` pass, instead of re-issuing polls.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Waits for the phase of `parity` to complete.  Gives up after limit_ns
// (kWaitNs unless the context set another limit; or 2^30 polls), or as soon
// as another role gave up: then it raises the shared abort flag, records
// ZOOM_ERR_TIMEOUT in the status word and returns false.
__device__ __noinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                       unsigned int* status, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait_sleep(bar, parity, 1000000u)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) break;
  }
  *abort_flag = 1;
  atomicExch(status, 1u);
  return false;
}
// Non-blocking poll of the phase of `parity`.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The common case inline: a short spin of non-blocking polls, then the
// bounded slow path.  A thread suspended in try_wait resumes noticeably later
// than a polling one sees the phase complete; on the filter's hand-offs
// (accumulator full / free, a few hundred cycles apart) the spin takes about
// 15 % off the step.
constexpr int kSpinPolls = 32;
__device__ __forceinline__ bool mbar_wait_fast(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                               unsigned int* status, uint64_t limit_ns) {
  for (int i = 0; i < kSpinPolls; ++i)
    if (mbar_test_wait(bar, parity)) return true;
  return mbar_wait(bar, parity, abort_flag, status, limit_ns);
}
// Before a CTA exits, also after an abort: waits for an asynchronous
// operation it started (a bulk copy, or the MMAs a commit tracks) to signal
// its barrier, whatever the abort flag says, for at most kWaitNs.
__device__ __noinline__ bool mbar_drain(uint64_t* bar, uint32_t parity, unsigned int* status) {
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 0; it < (1u << 30); ++it) {
    if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;
    if (globaltimer() - t0 > kWaitNs) break;
  }
  atomicExch(status, 1u);
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, M = N = 128, kind::f16 (fp16 or bf16 in,
// fp32 accumulate).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Issues the load of 32 consecutive TMEM columns of this warp's 32 lanes
// (one lane per thread) into `v`, and `m` receives the minimum of the 32
// values, reduced in the TMEM load path (tcgen05.ld.red, sm_103a): the
// threshold test of a chunk costs one comparison instead of a min tree on the
// 16-lane ALU pipe.  The registers are valid after tmem_ld_wait.
__device__ __forceinline__ void tmem_ld32_min_issue(uint32_t taddr, float (&v)[32], float& m) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x32.min.f32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=f"(m)
      : "r"(taddr)
      : "memory");
}
// Waits for the TMEM loads in flight; `v` and `m` (the destinations of the
// last one) are in-out operands, so the compiler reads those registers only
// after the wait and may do other work between the load and the wait.
__device__ __forceinline__ void tmem_ld_wait(float (&v)[32], float& m) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                 "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
                 "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
                 "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+f"(m)
               :
               : "memory");
}

// After a tcgen05.wait::ld that covered the load into `v` and `m`: tells the
// compiler those registers are valid from here on (no instruction).
__device__ __forceinline__ void tmem_regs_ready(float (&v)[32], float& m) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                 "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
                 "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
                 "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+f"(m)
               :
               : "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes stored as 128 contiguous bytes; `lbo` = byte distance
// between core matrices adjacent along K, `sbo` = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100-family tcgen05
  return d;                // base offset 0, absolute LBO mode, no swizzle
}

// Instruction descriptor of kind::f16: D fp32, A and B of the same type
// (fp16: 0, bf16: 1), both K-major, M = N = 128.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t ab_type) {
  return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((uint32_t)(TC_ROWS >> 3) << 17) |
         ((uint32_t)(TC_ROWS >> 4) << 24);
}

struct TcArgs {
  const uint16_t* qop;   // [q_tiles (even)][KC][128][8] fp16/bf16 bits
  const float* qn;       // [nq] ||q||^2 (FP32)
  const uint16_t* dop;   // [d_tiles][KC][128][8]
  int64_t nq;
  int64_t nd;
  int nq_pairs;          // ceil(nq / 256)
  int nd_tiles;          // ceil(nd / 128)
  int nsplit;
  int tiles_per_split;
  float* out_d;          // [nsplit][nq][MC] chunk minimum d~, ascending (FLT_MAX: none)
  int32_t* out_id;       // [nsplit][nq][MC] chunk index (entries 32c..32c+31; -1: none)
  unsigned int* status;
  // tail_split (> 0): the first full_rounds * gridDim.x query pairs are
  // whole items (one per CTA and round, every CTA streaming the dictionary
  // from tile 0 in step, so L2 serves the tiles); the remaining pairs are
  // cut into tail_split equal dictionary parts, nsplit = tail_split lists,
  // so the last round is shorter.  0: items are (split, pair) round robin.
  int tail_split;
  int full_rounds;
  // nq_dev != nullptr: only the first min(*nq_dev, nq) queries are searched
  // (a count written by an earlier kernel); nq stays the lists' row stride
  const unsigned long long* nq_dev;
  // bound on every wait (ns), and the testing aid: inject == 1 makes each
  // CTA's epilogue withhold the release of its accumulators from the third
  // tile of its first item on, so the issuing threads' waits run out
  uint64_t wait_ns;
  int inject;
  // packed chunk lists (the BF16 form of the wide-step filter): bits of a
  // list key that hold the chunk number
  int id_bits;
};

// Queries searched: nq, or the device count when one is given (read where
// needed, so that nothing extra stays live in the roles' loops).
__device__ __forceinline__ int64_t searched_queries(const TcArgs& a) {
  if (!a.nq_dev) return a.nq;
  const int64_t c = (int64_t)*a.nq_dev;
  return c < a.nq ? c : a.nq;
}

// The work items of one CTA, in order; every role walks the same sequence.
struct WorkIter {
  int k = 0;   // item number of this CTA
  // qp: query pair, seg: list index, [t0, t1): dictionary tiles
  __device__ bool next(const TcArgs& a, int& qp, int& seg, int& t0, int& t1) {
    const int G = gridDim.x, c = blockIdx.x;
    const int nq_pairs = a.nq_dev ? (int)((searched_queries(a) + 2 * TC_ROWS - 1) / (2 * TC_ROWS)) : a.nq_pairs;
    if (a.tail_split > 0) {
      if (k < a.full_rounds) {
        qp = c + k * G;
        seg = 0;
        t0 = 0;
        t1 = a.nd_tiles;
      } else {
        const int tail = nq_pairs - a.full_rounds * G;
        const int j = c + (k - a.full_rounds) * G;   // tail item: part j / tail of pair j % tail
        if (j >= tail * a.tail_split) return false;
        qp = a.full_rounds * G + j % tail;
        seg = j / tail;
        t0 = seg * a.tiles_per_split;
        t1 = min(a.nd_tiles, t0 + a.tiles_per_split);
      }
    } else {
      const int item = c + k * G;
      if (item >= a.nsplit * nq_pairs) return false;
      seg = item / nq_pairs;
      qp = item % nq_pairs;
      t0 = seg * a.tiles_per_split;
      t1 = min(a.nd_tiles, t0 + a.tiles_per_split);
    }
    ++k;
    return true;
  }
};

// Inserts (v, id) into the ascending list, dropping its last entry; nothing
// changes when v >= ld[MC-1].  Selects only, no branches: the lanes of a
// warp insert at different positions without diverging (a branchy insertion
// serialised those paths and cost ~1000 cycles per merged entry).
template <int MC>
__device__ __forceinline__ void list_push(float (&ld)[MC], int (&li)[MC], float v, int id) {
#pragma unroll
  for (int j = MC - 1; j > 0; --j) {
    const bool shift = v < ld[j - 1];
    const bool here = v < ld[j];
    ld[j] = shift ? ld[j - 1] : (here ? v : ld[j]);
    li[j] = shift ? li[j - 1] : (here ? id : li[j]);
  }
  const bool first = v < ld[0];
  ld[0] = first ? v : ld[0];
  li[0] = first ? id : li[0];
}

constexpr unsigned kFull = 0xffffffffu;

template <int MC>
__device__ __forceinline__ void flush_appends(float (&ld)[MC], int (&li)[MC], float& thr,
                                              const float* bv, const int* bi, int& cnt) {
  const int n = cnt;
  const int nmax = __reduce_max_sync(kFull, n);
  for (int s = 0; s < nmax; ++s) {
    const bool has = s < n;
    const float x = has ? bv[s * 256] : FLT_MAX;
    const int xi = has ? bi[s * 256] : -1;
    list_push<MC>(ld, li, x, xi);
  }
  thr = ld[MC - 1];
  cnt = 0;
}

// A 32-column chunk whose minimum `m` is below the list threshold is a
// candidate: its index is appended (rare after the first tiles).
__device__ __forceinline__ void chunk_test(float m, int chunk, float thr, float* bv, int* bi, int& cnt) {
  if (m < thr) {
    bv[cnt * 256] = m;
    bi[cnt * 256] = chunk;
    ++cnt;
  }
}

template <int KC, int MC, uint32_t AB_TYPE>
__global__ void __maxnreg__(tc_max_regs(KC, MC)) k_knn_tc(TcArgs a) {
  constexpr int kMma = tc_mma_warps(KC, MC);
  constexpr bool kOneRound = tc_one_round(KC, MC);
  constexpr uint32_t kTileBytes = KC * TC_ROWS * 16;  // one 128-row operand tile
  constexpr int kKSteps = KC / 2;                     // MMA K = 16 = two 8-element chunks
  constexpr uint32_t kIdesc = instr_desc(AB_TYPE);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                                  // 2 query tiles
  constexpr int kStages = tc_stages(KC, MC);
  unsigned char* sB = smem + 2 * kTileBytes;                 // kStages dictionary tiles
  uint64_t* bars = (uint64_t*)(sB + kStages * kTileBytes);
  uint64_t* a_full = bars + 0;
  uint64_t* a_empty = bars + 1;
  uint64_t* b_full = bars + 2;                 // [kStages]
  uint64_t* b_empty = b_full + kStages;        // [kStages]
  // accumulator hand-off per (buffer, query tile): a query tile's 128
  // columns go back to the MMA as soon as its 4 epilogue warps have read them
  uint64_t* acc_full = b_empty + kStages;      // [2][2]
  uint64_t* acc_empty = acc_full + 4;          // [2][2]
  uint64_t* drain = acc_empty + 4;             // [4] one per MMA-issuing thread, at exit
  uint32_t* tmem_slot = (uint32_t*)(drain + 4);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  constexpr int kBuf = tc_buf(KC);
  float* buf_v = (float*)((unsigned char*)bars + kBarBytes);   // [kBuf][256]
  int* buf_i = (int*)(buf_v + kBuf * 256);               // [kBuf][256]
  float* lst_v = (float*)(buf_i + kBuf * 256);           // [MC][256] lists (one round only)
  int* lst_i = (int*)(lst_v + MC * 256);                 // [MC][256]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    mbar_init(a_empty, kMma);   // one commit per MMA thread
    for (int s = 0; s < kStages; ++s) {
      mbar_init(b_full + s, 1);
      mbar_init(b_empty + s, 2);
    }
    for (int b = 0; b < 4; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 128);
      mbar_init(drain + b, 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- producer: bulk copies of operand tiles ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, a_phase = 0;
      bool first = true;
      int a_copies = 0;
      int64_t b_copies = 0;
      WorkIter it;
      int qp, seg, t0, t1;
      while (!*abort_flag && it.next(a, qp, seg, t0, t1)) {
        if (!first) {
          if (!mbar_wait(a_empty, a_phase, abort_flag, a.status, a.wait_ns)) break;
          a_phase ^= 1u;
        }
        first = false;
        mbar_arrive_expect_tx(a_full, 2 * kTileBytes);
        bulk_g2s(sA, (const unsigned char*)a.qop + (size_t)qp * 2 * kTileBytes, 2 * kTileBytes, a_full);
        ++a_copies;
        for (int t = t0; t < t1; ++t) {
          if (!mbar_wait_fast(b_empty + stage, phase ^ 1u, abort_flag, a.status, a.wait_ns)) break;
          mbar_arrive_expect_tx(b_full + stage, kTileBytes);
          bulk_g2s(sB + stage * kTileBytes, (const unsigned char*)a.dop + (size_t)t * kTileBytes,
                   kTileBytes, b_full + stage);
          ++b_copies;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // no bulk copy may still be writing into shared memory at exit: wait
      // for the last query-tile copy and the last copy into every ring stage
      if (a_copies > 0) mbar_drain(a_full, (uint32_t)(a_copies - 1) & 1u, a.status);
      for (int64_t i = b_copies - kStages > 0 ? b_copies - kStages : 0; i < b_copies; ++i)
        mbar_drain(b_full + i % kStages, (uint32_t)(i / kStages) & 1u, a.status);
    }
  } else if (warp == 1 || warp >= 10) {
    // ------- MMA issue: one thread per query tile (and buffer, kMma = 4) -------
    if (lane == 0) {
      const int m = warp == 1 ? 0 : warp - 9;   // warps 1, 10, 11, 12
      const int qt = m & 1;
      const int mine_buf = kMma == 4 ? (m >> 1) : -1;   // -1: both buffers
      int stage = 0, buf = 0, items = 0;
      uint32_t phase = 0, a_phase = 0;
      uint32_t accp[2] = {0u, 0u};
      // Descriptors of the first K step of this query tile and of ring
      // stage 0; a K step adds 2 core-matrix columns (4 KiB), a stage one tile
      // (start address field in 16-byte units; every address stays below
      // 256 KiB, so the 14-bit field never carries).
      const uint64_t ad0 = smem_desc(smem_u32(sA + qt * kTileBytes), TC_ROWS * 16, 128);
      const uint64_t bd0 = smem_desc(smem_u32(sB), TC_ROWS * 16, 128);
      constexpr uint64_t kKStepAdv = (2 * TC_ROWS * 16) >> 4;
      constexpr uint64_t kTileAdv = kTileBytes >> 4;
      WorkIter it;
      int qp, seg, t0, t1;
      while (!*abort_flag && it.next(a, qp, seg, t0, t1)) {
        if (!mbar_wait_fast(a_full, a_phase, abort_flag, a.status, a.wait_ns)) break;
        a_phase ^= 1u;
        tc_fence_after();
        bool ok = true;
        for (int t = t0; t < t1; ++t) {
          if (mine_buf < 0 || buf == mine_buf) {
            if (!mbar_wait_fast(b_full + stage, phase, abort_flag, a.status, a.wait_ns) ||
                !mbar_wait_fast(acc_empty + buf * 2 + qt, accp[buf] ^ 1u, abort_flag, a.status, a.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t bd_s = bd0 + (uint64_t)stage * kTileAdv;
            const uint32_t d_addr = tmem + (uint32_t)(buf * 256 + qt * 128);
#pragma unroll
            for (int ks = 0; ks < kKSteps; ++ks)
              mma_f16(d_addr, ad0 + ks * kKStepAdv, bd_s + ks * kKStepAdv, kIdesc, ks > 0 ? 1u : 0u);
            mma_commit(acc_full + buf * 2 + qt);   // also frees the ring stage (epilogue)
          }
          accp[buf] ^= 1u;
          buf ^= 1;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        mma_commit(a_empty);
        ++items;
        if (!ok) break;
      }
      // the last item's release of the query tiles is never consumed by the
      // producer: wait for it so no tensor-core arrival is pending at exit;
      // then (also after an abort) one more commit, whose arrival means every
      // MMA this thread issued has completed before TMEM is freed
      if (items > 0) mbar_drain(a_empty, (uint32_t)(items - 1) & 1u, a.status);
      mma_commit(drain + m);
      mbar_drain(drain + m, 0u, a.status);
    }
  } else {
    // ------------- epilogue: per query, the MC best 32-entry chunks -------------
    const int ew = warp - 2;            // 0..7
    const int qt = ew >> 2;             // query tile within the pair
    const int quad = warp & 3;          // TMEM lane quadrant this warp may access
    const int row = quad * 32 + lane;   // row in the 128-row tile
    // this lane's append buffer: slot s at [s * 256] (one bank per lane)
    float* bv = buf_v + ew * 32 + lane;
    int* bi = buf_i + ew * 32 + lane;
    int buf = 0;
    uint32_t accp[2] = {0u, 0u};
    // The accumulator of a (tile, query tile) being complete means its MMAs
    // have read their ring stage: one lane per query tile releases the stage
    // (two arrivals free it), which keeps that commit off the MMA threads.
    int stage = 0;
    const bool releaser = (ew & 3) == 0 && lane == 0;
    WorkIter it;
    int qp, split, t0, t1;
    int item_no = 0;
    while (it.next(a, qp, split, t0, t1)) {
      if (__any_sync(kFull, *abort_flag != 0)) break;   // warp-uniform exit
      const bool withhold = a.inject == 1 && item_no++ == 0;   // testing aid (see TcArgs)
      const int64_t q = ((int64_t)qp * 2 + qt) * TC_ROWS + row;
      const bool valid = q < searched_queries(a);
      const float qn = valid ? a.qn[q] : 0.f;
      // The sorted chunk list: registers (ld, li), or -- one-round epilogue --
      // this lane's column of the shared lists, brought into registers only
      // to merge appended chunks and at the end of the item.
      float ld[MC];
      int li[MC];
      float* sl_v = lst_v + ew * 32 + lane;
      int* sl_i = lst_i + ew * 32 + lane;
#pragma unroll
      for (int j = 0; j < MC; ++j) {
        ld[j] = FLT_MAX;
        li[j] = -1;
        if constexpr (kOneRound) {
          sl_v[j * 256] = FLT_MAX;
          sl_i[j * 256] = -1;
        }
      }
      float thr = FLT_MAX;   // in acc units: d~ - ||q||^2
      int cnt = 0;           // entries in this lane's append buffer
      auto flush = [&]() {
        if constexpr (kOneRound) {
#pragma unroll
          for (int j = 0; j < MC; ++j) {
            ld[j] = sl_v[j * 256];
            li[j] = sl_i[j * 256];
          }
        }
        flush_appends<MC>(ld, li, thr, bv, bi, cnt);
        if constexpr (kOneRound) {
#pragma unroll
          for (int j = 0; j < MC; ++j) {
            sl_v[j * 256] = ld[j];
            sl_i[j * 256] = li[j];
          }
        }
      };
      bool ok = true;
      for (int t = t0; t < t1; ++t) {
        // every lane polls, then the warp agrees (and reconverges) before the
        // warp-collective TMEM loads
        const bool w = __all_sync(kFull, mbar_wait_fast(acc_full + buf * 2 + qt, accp[buf], abort_flag, a.status, a.wait_ns));
        if (!w) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (releaser) mbar_arrive(b_empty + stage);
        if (++stage == kStages) stage = 0;
        const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 256 + qt * 128);
        // only the chunk minima are used (the loaded values are dead)
        if constexpr (kOneRound) {
          // the tile's four chunks in one round of loads and one wait
          float va[32], vb[32], vc[32], vd[32], ma, mb, mc, md;
          tmem_ld32_min_issue(tb, va, ma);
          tmem_ld32_min_issue(tb + 32, vb, mb);
          tmem_ld32_min_issue(tb + 64, vc, mc);
          tmem_ld32_min_issue(tb + 96, vd, md);
          tmem_ld_wait(va, ma);
          tmem_regs_ready(vb, mb);
          tmem_regs_ready(vc, mc);
          tmem_regs_ready(vd, md);
          tc_fence_before();
          if (!withhold || t < t0 + 2)
            mbar_arrive(acc_empty + buf * 2 + qt);   // every TMEM read of this tile is done
          chunk_test(ma, t * 4, thr, bv, bi, cnt);
          chunk_test(mb, t * 4 + 1, thr, bv, bi, cnt);
          chunk_test(mc, t * 4 + 2, thr, bv, bi, cnt);
          chunk_test(md, t * 4 + 3, thr, bv, bi, cnt);
        } else {
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            float va[32], vb[32], ma, mb;
            tmem_ld32_min_issue(tb + h * 64, va, ma);
            tmem_ld32_min_issue(tb + h * 64 + 32, vb, mb);
            tmem_ld_wait(va, ma);
            tmem_regs_ready(vb, mb);
            if (h == 1) {   // every TMEM read of this tile is done: hand the buffer back
              tc_fence_before();
              if (!withhold || t < t0 + 2) mbar_arrive(acc_empty + buf * 2 + qt);
            }
            chunk_test(ma, t * 4 + 2 * h, thr, bv, bi, cnt);
            chunk_test(mb, t * 4 + 2 * h + 1, thr, bv, bi, cnt);
          }
        }
        accp[buf] ^= 1u;
        buf ^= 1;
        // room for the next tile's up to 4 appends in every lane; merging
        // here, with the accumulator already handed back, keeps the merge off
        // the MMA's path
        if (__any_sync(kFull, cnt > kBuf - 4)) flush();
      }
      if (!ok) break;
      flush();
      if (valid) {
        float* od = a.out_d + ((int64_t)split * a.nq + q) * MC;
        int32_t* oi = a.out_id + ((int64_t)split * a.nq + q) * MC;
#pragma unroll
        for (int j = 0; j < MC; ++j) {
          const bool real = li[j] >= 0 && (int64_t)li[j] * 32 < a.nd;
          od[j] = real ? qn + ld[j] : FLT_MAX;
          oi[j] = real ? li[j] : -1;
        }
        if (a.tail_split > 0 && t0 == 0 && t1 == a.nd_tiles) {
          // a whole pair: its other lists are empty
          for (int s2 = 1; s2 < a.tail_split; ++s2) {
            float* od1 = a.out_d + ((int64_t)s2 * a.nq + q) * MC;
            int32_t* oi1 = a.out_id + ((int64_t)s2 * a.nq + q) * MC;
#pragma unroll
            for (int j = 0; j < MC; ++j) {
              od1[j] = FLT_MAX;
              oi1[j] = -1;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// The wide-step filter for the narrow operands (single FP16 term or BF16,
// K = 32 or 64): each query tile's MMA is M = 128 x N = 256 (two 128-row
// dictionary tiles in one 256-row step), one 256-column accumulator per
// query tile (the two fill the TMEM), so an issuing thread spends half the
// instructions and commits of the 128 x 128 form per unit of work and, while
// the epilogue reads one query tile's accumulator, the tensor pipe computes
// the other's.
//   warp 0      producer: the item's two query tiles, then 256-row steps of
//               the dictionary (one bulk copy each) into a ring
//   warps 1, 10 issue the MMAs of query tile 0 and 1
//   warps 2..9  epilogue: warps 2..5 read query tile 0's accumulator (one
//               warp per TMEM lane quadrant), warps 6..9 tile 1's; each reads
//               its 32 rows x 256 columns per step in two rounds of four
//               32-column loads, testing the first round's chunk minima while
//               the second round's loads are in flight
// Chunk c of step t is entries 256 t + 32 c .. +31 (columns 32 c .. 32 c + 31).
// ---------------------------------------------------------------------------
constexpr int TW_ROWS = 256;              // dictionary rows per step (MMA N)
// append slots per epilogue lane ((value, index) pairs), and the lists:
// (value, index) pairs, or 32-bit keys
__host__ __device__ constexpr int tw_buf(bool) { return 16; }
__host__ __device__ constexpr int tw_epi_bytes(int MC, bool packed) {
  return tw_buf(packed) * 256 * 8 + MC * 256 * (packed ? 4 : 8);
}
__host__ __device__ constexpr int tw_stages(int KC, int MC, bool packed) {
  return (kSmemMax - 1024 - kBarBytes - tw_epi_bytes(MC, packed) - 2 * KC * TC_ROWS * 16) / (KC * TW_ROWS * 16) < 12
             ? (kSmemMax - 1024 - kBarBytes - tw_epi_bytes(MC, packed) - 2 * KC * TC_ROWS * 16) / (KC * TW_ROWS * 16)
             : 12;
}
static_assert(tw_stages(4, 16, false) == 9 && tw_stages(4, 32, false) == 7 && tw_stages(8, 16, false) == 4 &&
                  tw_stages(8, 32, false) == 3 && tw_stages(4, 16, true) == 10 && tw_stages(4, 32, true) == 9 &&
                  tw_stages(8, 16, true) == 4 && tw_stages(8, 32, true) == 4,
              "wide ring depths");

// The per-query list of the MC best chunks, kept by one epilogue lane: a
// sorted list in shared memory (this lane's column, entry j at [j * 256]),
// candidates appended to a shared-memory buffer and merged when some lane
// of the warp runs out of room (the merge runs with the warp converged).
// ChunkListF: FP32 minima d~ - ||q||^2 with chunk numbers, in two arrays.
template <int MC, int BUFW>
struct ChunkListF {
  float* bv;
  int* bi;
  float* sv;
  int* si;
  float thr = FLT_MAX;
  int cnt = 0;
  __device__ void init() {
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      sv[j * 256] = FLT_MAX;
      si[j * 256] = -1;
    }
    thr = FLT_MAX;
    cnt = 0;
  }
  __device__ __forceinline__ void test(float m, int chunk) { chunk_test(m, chunk, thr, bv, bi, cnt); }
  __device__ __forceinline__ bool full() const { return cnt > BUFW - 8; }
  __device__ void flush() {
    float ld[MC];
    int li[MC];
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      ld[j] = sv[j * 256];
      li[j] = si[j * 256];
    }
    flush_appends<MC>(ld, li, thr, bv, bi, cnt);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      sv[j * 256] = ld[j];
      si[j * 256] = li[j];
    }
  }
  // the list as chunk minima of d~ (FLT_MAX / -1: none)
  __device__ void write(float qn, int64_t nd, float* od, int32_t* oi) const {
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const float v = sv[j * 256];
      const int c = si[j * 256];
      const bool real = c >= 0 && (int64_t)c * 32 < nd;
      od[j] = real ? qn + v : FLT_MAX;
      oi[j] = real ? c : -1;
    }
  }
};

// Order-preserving map of FP32 values to 32-bit keys (a < b iff key(a) <
// key(b)) and back.
__device__ __forceinline__ uint32_t f32_order_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float f32_from_order_key(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// ChunkListK: the sorted list holds one 32-bit key per entry, the order
// key of the chunk minimum d~ = ||q||^2 + (d~ - ||q||^2) with its low
// id_bits replaced by the chunk number.  The replaced bits round d~ down (to
// 32 - id_bits significant key bits: 6 mantissa bits for up to 2^17
// chunks), so the listed value stays a lower bound of the chunk's entries,
// which is all the rerank's stop rule needs; chunks closer than that are
// ranked by number.  Merging into sorted keys takes two integer min/max per
// position (l[j] = max(l[j-1], min(x, l[j]))) against six compare-selects
// for a (value, index) pair.  Candidates are appended as (m, chunk) pairs
// after one FP32 comparison, as in ChunkListF, and keyed in the merge, so
// the per-step test costs the same in both lists.
template <int MC, int BUFW>
struct ChunkListK {
  float* bv;
  int* bi;
  uint32_t* sk;
  uint32_t hi;    // mask of the value bits
  float qn;
  uint32_t thr = 0xFFFFFFFFu;
  // a chunk minimum m (d~ - ||q||^2) at or above thr_m cannot make a key
  // below thr
  float thr_m = FLT_MAX;
  int cnt = 0;
  __device__ void init() {
#pragma unroll
    for (int j = 0; j < MC; ++j) sk[j * 256] = 0xFFFFFFFFu;
    thr = 0xFFFFFFFFu;
    thr_m = FLT_MAX;
    cnt = 0;
  }
  __device__ __forceinline__ void test(float m, int chunk) { chunk_test(m, chunk, thr_m, bv, bi, cnt); }
  __device__ __forceinline__ bool full() const { return cnt > BUFW - 8; }
  __device__ void flush() {
    uint32_t l[MC];
#pragma unroll
    for (int j = 0; j < MC; ++j) l[j] = sk[j * 256];
    const int n = cnt;
    const int nmax = __reduce_max_sync(kFull, n);
    for (int s = 0; s < nmax; ++s) {
      const uint32_t x =
          s < n ? (f32_order_key(qn + bv[s * 256]) & hi) | (uint32_t)bi[s * 256] : 0xFFFFFFFFu;
#pragma unroll
      for (int j = MC - 1; j > 0; --j) l[j] = max(l[j - 1], min(x, l[j]));
      l[0] = min(x, l[0]);
    }
    thr = l[MC - 1];
    cnt = 0;
    // Keys below thr have value bits at most those of thr, so their d~ lies
    // below U, the first value of the next key bucket; fl(qn + m) < U needs
    // m < U - qn, which fl(U - qn) plus a few ulps of the operands bounds
    // from above.
    const uint32_t next = (thr & hi) + (~hi + 1u);
    const float U = f32_from_order_key(next);
    if (thr == 0xFFFFFFFFu || next < (thr & hi) || !(U < FLT_MAX)) {
      thr_m = FLT_MAX;   // no bound below infinity (or the list is not full): test nothing away
    } else {
      thr_m = (U - qn) + (fabsf(U) + fabsf(qn)) * 2.4e-7f;
    }
#pragma unroll
    for (int j = 0; j < MC; ++j) sk[j * 256] = l[j];
  }
  __device__ void write(float, int64_t nd, float* od, int32_t* oi) const {
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      const uint32_t k = sk[j * 256];
      const uint32_t c = k & ~hi;
      const bool real = k != 0xFFFFFFFFu && (int64_t)c * 32 < nd;
      od[j] = real ? f32_from_order_key(k & hi) : FLT_MAX;
      oi[j] = real ? (int32_t)c : -1;
    }
  }
};

// kind::f16, D fp32, A and B of one type, K-major, M = 128, N = 256.
__host__ __device__ constexpr uint32_t instr_desc_wide(uint32_t ab_type) {
  return (1u << 4) | (ab_type << 7) | (ab_type << 10) | ((uint32_t)(TW_ROWS >> 3) << 17) |
         ((uint32_t)(TC_ROWS >> 4) << 24);
}

template <int KC, int MC, uint32_t AB_TYPE, bool PACKED>
__global__ void __launch_bounds__(352, 1) k_knn_tw(TcArgs a) {
  constexpr uint32_t kATile = KC * TC_ROWS * 16;     // one 128-row query tile
  constexpr uint32_t kStep = KC * TW_ROWS * 16;      // one 256-row dictionary step
  constexpr int kKSteps = KC / 2;
  constexpr uint32_t kIdesc = instr_desc_wide(AB_TYPE);
  constexpr int kStages = tw_stages(KC, MC, PACKED);
  constexpr int kBufW = tw_buf(PACKED);              // append slots per epilogue lane
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                          // 2 query tiles
  unsigned char* sB = smem + 2 * kATile;             // kStages dictionary steps
  uint64_t* bars = (uint64_t*)(sB + kStages * kStep);
  uint64_t* a_full = bars + 0;
  uint64_t* a_empty = bars + 1;
  uint64_t* b_full = bars + 2;                 // [kStages]
  uint64_t* b_empty = b_full + kStages;        // [kStages]
  uint64_t* acc_full = b_empty + kStages;      // [2] per query tile
  uint64_t* acc_empty = acc_full + 2;          // [2]
  uint64_t* drain = acc_empty + 2;             // [2] one per issuing thread, at exit
  uint32_t* tmem_slot = (uint32_t*)(drain + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  // epilogue: append buffers [kBufW][256] and lists [MC][256], one column
  // per query row (values and indices, or keys)
  unsigned char* epi = (unsigned char*)bars + kBarBytes;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    mbar_init(a_empty, 2);   // one commit per issuing thread
    for (int s = 0; s < kStages; ++s) {
      mbar_init(b_full + s, 1);
      mbar_init(b_empty + s, 2);   // one release per query tile
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(acc_full + q, 1);
      mbar_init(acc_empty + q, 4);   // the query tile's four epilogue warps
      mbar_init(drain + q, 1);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, a_phase = 0;
      bool first = true;
      int a_copies = 0;
      int64_t b_copies = 0;
      WorkIter it;
      int qp, seg, t0, t1;
      while (!*abort_flag && it.next(a, qp, seg, t0, t1)) {
        if (!first) {
          if (!mbar_wait(a_empty, a_phase, abort_flag, a.status, a.wait_ns)) break;
          a_phase ^= 1u;
        }
        first = false;
        mbar_arrive_expect_tx(a_full, 2 * kATile);
        bulk_g2s(sA, (const unsigned char*)a.qop + (size_t)qp * 2 * kATile, 2 * kATile, a_full);
        ++a_copies;
        for (int t = t0; t < t1; ++t) {
          if (!mbar_wait_fast(b_empty + stage, phase ^ 1u, abort_flag, a.status, a.wait_ns)) break;
          mbar_arrive_expect_tx(b_full + stage, kStep);
          bulk_g2s(sB + stage * kStep, (const unsigned char*)a.dop + (size_t)t * kStep, kStep, b_full + stage);
          ++b_copies;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (a_copies > 0) mbar_drain(a_full, (uint32_t)(a_copies - 1) & 1u, a.status);
      for (int64_t i = b_copies - kStages > 0 ? b_copies - kStages : 0; i < b_copies; ++i)
        mbar_drain(b_full + i % kStages, (uint32_t)(i / kStages) & 1u, a.status);
    }
  } else if (warp == 1 || warp == 10) {
    // ---------------- MMA issue: one thread per query tile ----------------
    if (lane == 0) {
      const int qt = warp == 1 ? 0 : 1;
      int stage = 0, items = 0;
      uint32_t phase = 0, a_phase = 0, accp = 0;
      // query tile: K-major, core matrices 8 rows x 16 B, K chunks 128 rows
      // apart; dictionary step: the same with 256 rows (LBO 4 KiB)
      const uint64_t ad0 = smem_desc(smem_u32(sA + qt * kATile), TC_ROWS * 16, 128);
      const uint64_t bd0 = smem_desc(smem_u32(sB), TW_ROWS * 16, 128);
      constexpr uint64_t kAStep = (2 * TC_ROWS * 16) >> 4;
      constexpr uint64_t kBStep = (2 * TW_ROWS * 16) >> 4;
      constexpr uint64_t kStageAdv = kStep >> 4;
      const uint32_t d_addr = tmem + (uint32_t)(qt * TW_ROWS);
      WorkIter it;
      int qp, seg, t0, t1;
      while (!*abort_flag && it.next(a, qp, seg, t0, t1)) {
        if (!mbar_wait_fast(a_full, a_phase, abort_flag, a.status, a.wait_ns)) break;
        a_phase ^= 1u;
        tc_fence_after();
        // The step's dictionary stage is awaited right after the previous
        // step's commit, while the epilogue still reads the accumulator, so
        // only the accumulator hand-off stands between two steps' MMAs.
        bool ok = t0 >= t1 || mbar_wait_fast(b_full + stage, phase, abort_flag, a.status, a.wait_ns);
        for (int t = t0; ok && t < t1; ++t) {
          if (!mbar_wait_fast(acc_empty + qt, accp ^ 1u, abort_flag, a.status, a.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t bd_s = bd0 + (uint64_t)stage * kStageAdv;
#pragma unroll
          for (int ks = 0; ks < kKSteps; ++ks)
            mma_f16(d_addr, ad0 + ks * kAStep, bd_s + ks * kBStep, kIdesc, ks > 0 ? 1u : 0u);
          mma_commit(acc_full + qt);   // also frees the ring stage (the epilogue releases it)
          accp ^= 1u;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
          if (t + 1 < t1 && !mbar_wait_fast(b_full + stage, phase, abort_flag, a.status, a.wait_ns)) {
            ok = false;
            break;
          }
        }
        mma_commit(a_empty);
        ++items;
        if (!ok) break;
      }
      if (items > 0) mbar_drain(a_empty, (uint32_t)(items - 1) & 1u, a.status);
      mma_commit(drain + qt);
      mbar_drain(drain + qt, 0u, a.status);
    }
  } else {
    // ------------- epilogue: per query, the MC best 32-entry chunks -------------
    const int ew = warp - 2;            // 0..7
    const int qt = ew >> 2;             // query tile
    const int quad = warp & 3;          // TMEM lane quadrant this warp may access
    const int row = quad * 32 + lane;
    const int col = ew * 32 + lane;     // this lane's column of the buffers and lists
    using List = typename std::conditional<PACKED, ChunkListK<MC, kBufW>, ChunkListF<MC, kBufW>>::type;
    List L;
    float* bv = (float*)epi;
    int* bi = (int*)(bv + kBufW * 256);
    L.bv = bv + col;
    L.bi = bi + col;
    if constexpr (PACKED) {
      L.sk = (uint32_t*)(bi + kBufW * 256) + col;
      L.hi = ~((1u << a.id_bits) - 1u);
    } else {
      float* sv = (float*)(bi + kBufW * 256);
      L.sv = sv + col;
      L.si = (int*)(sv + MC * 256) + col;
    }
    const bool releaser = quad == 0 && lane == 0;   // frees each step's ring stage (one per query tile)
    int stage = 0, item_no = 0;
    uint32_t accp = 0;
    WorkIter it;
    int qp, split, t0, t1;
    while (it.next(a, qp, split, t0, t1)) {
      if (__any_sync(kFull, *abort_flag != 0)) break;   // warp-uniform exit
      const bool withhold = a.inject == 1 && item_no++ == 0;   // testing aid (see TcArgs)
      const int64_t q = ((int64_t)qp * 2 + qt) * TC_ROWS + row;
      const bool valid = q < a.nq;
      const float qn = valid ? a.qn[q] : 0.f;
      if constexpr (PACKED) L.qn = qn;
      L.init();
      bool ok = true;
      for (int t = t0; t < t1; ++t) {
        const bool w = __all_sync(kFull, mbar_wait_fast(acc_full + qt, accp, abort_flag, a.status, a.wait_ns));
        if (!w) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (releaser) mbar_arrive(b_empty + stage);   // the MMAs that read the stage are done
        const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(qt * TW_ROWS);
        float va[32], vb[32], vc[32], vd[32], m0, m1, m2, m3, m4, m5, m6, m7;
        tmem_ld32_min_issue(tb, va, m0);
        tmem_ld32_min_issue(tb + 32, vb, m1);
        tmem_ld32_min_issue(tb + 64, vc, m2);
        tmem_ld32_min_issue(tb + 96, vd, m3);
        tmem_ld_wait(va, m0);
        tmem_regs_ready(vb, m1);
        tmem_regs_ready(vc, m2);
        tmem_regs_ready(vd, m3);
        // the second half's loads run while the first half's chunks are tested
        tmem_ld32_min_issue(tb + 128, va, m4);
        tmem_ld32_min_issue(tb + 160, vb, m5);
        tmem_ld32_min_issue(tb + 192, vc, m6);
        tmem_ld32_min_issue(tb + 224, vd, m7);
        const int c0 = t * 8;
        L.test(m0, c0);
        L.test(m1, c0 + 1);
        L.test(m2, c0 + 2);
        L.test(m3, c0 + 3);
        tmem_ld_wait(va, m4);
        tmem_regs_ready(vb, m5);
        tmem_regs_ready(vc, m6);
        tmem_regs_ready(vd, m7);
        tc_fence_before();
        __syncwarp();
        if (lane == 0 && (!withhold || t < t0 + 2)) mbar_arrive(acc_empty + qt);   // every read of it is done
        L.test(m4, c0 + 4);
        L.test(m5, c0 + 5);
        L.test(m6, c0 + 6);
        L.test(m7, c0 + 7);
        accp ^= 1u;
        if (++stage == kStages) stage = 0;
        // room for the next step's up to 8 appends in every lane
        if (__any_sync(kFull, L.full())) L.flush();
      }
      if (!ok) break;
      L.flush();
      if (valid) {
        L.write(qn, a.nd, a.out_d + ((int64_t)split * a.nq + q) * MC, a.out_id + ((int64_t)split * a.nq + q) * MC);
        if (a.tail_split > 0 && t0 == 0 && t1 == a.nd_tiles) {
          for (int s2 = 1; s2 < a.tail_split; ++s2) {
            float* od1 = a.out_d + ((int64_t)s2 * a.nq + q) * MC;
            int32_t* oi1 = a.out_id + ((int64_t)s2 * a.nq + q) * MC;
#pragma unroll
            for (int j = 0; j < MC; ++j) {
              od1[j] = FLT_MAX;
              oi1[j] = -1;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------

// Offset (in 16-bit elements) of element k of row r in the tiled layout
// [tile][kc][128][8].
__device__ __forceinline__ int64_t op_off(int64_t r, int k, int KC) {
  return (r / TC_ROWS) * ((int64_t)KC * TC_ROWS * 8) + (int64_t)(k >> 3) * (TC_ROWS * 8) +
         (r % TC_ROWS) * 8 + (k & 7);
}
// The same layout with tiles of `rows` rows ([tile][kc][rows][8]): the
// dictionary operands of the wide-step filter use 256-row tiles.
__device__ __forceinline__ int64_t op_off_rows(int64_t r, int k, int KC, int rows) {
  return (r / rows) * ((int64_t)KC * rows * 8) + (int64_t)(k >> 3) * (rows * 8) + (r % rows) * 8 + (k & 7);
}

__device__ __forceinline__ uint16_t h_bits(__half h) { return __half_as_ushort(h); }
__device__ __forceinline__ uint16_t b_bits(__nv_bfloat16 h) { return __bfloat16_as_ushort(h); }

// role 0: query rows, role 1: dictionary rows.  Rows in [n, n_rows) are
// padding: queries get zeros, dictionary entries a huge norm so that they
// never rank.  Exact form: the three D-element groups start at 0, S and 2S
// and the norm pair sits at 3S (S = 25 for K = 80, 50 for K = 160).
template <int D, int KC>
__global__ void k_operand_f16x3(const float* __restrict__ feat, int dpad, int64_t n, int64_t n_rows,
                                int role, uint16_t* __restrict__ op, float* __restrict__ norm_out,
                                const unsigned long long* __restrict__ n_dev) {
  constexpr int S = KC * 5 / 2;
  static_assert(D <= S && 3 * S + 2 <= KC * 8, "operand layout");
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  if (n_dev && (int64_t)*n_dev < n) n = (int64_t)*n_dev;   // rows past a device count are padding
  uint16_t row[KC * 8];
#pragma unroll
  for (int k = 0; k < KC * 8; ++k) row[k] = 0;
  if (r < n) {
    float n2 = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float v = feat[r * dpad + i];
      n2 = fmaf(v, v, n2);
      const __half hi = __float2half_rn(v);
      const __half lo = __float2half_rn(v - __half2float(hi));
      if (role == 0) {
        row[i] = h_bits(hi);
        row[S + i] = h_bits(lo);
        row[2 * S + i] = h_bits(hi);
      } else {
        const __half mh = __float2half_rn(-2.f * __half2float(hi));
        row[i] = h_bits(mh);
        row[S + i] = h_bits(mh);
        row[2 * S + i] = h_bits(__float2half_rn(-2.f * __half2float(lo)));
      }
    }
    if (role == 0) {
      row[3 * S] = h_bits(__float2half_rn(1.f));
      row[3 * S + 1] = h_bits(__float2half_rn(1.f));
    } else {
      const __half nh = __float2half_rn(n2);
      row[3 * S] = h_bits(nh);
      row[3 * S + 1] = h_bits(__float2half_rn(n2 - __half2float(nh)));
    }
    if (norm_out) norm_out[r] = n2;
  } else if (role == 1) {
    row[3 * S] = h_bits(__float2half_rn(60000.f));
  }
#pragma unroll
  for (int kc = 0; kc < KC; ++kc) {
    uint4 pk;
    pk.x = (uint32_t)row[kc * 8 + 0] | ((uint32_t)row[kc * 8 + 1] << 16);
    pk.y = (uint32_t)row[kc * 8 + 2] | ((uint32_t)row[kc * 8 + 3] << 16);
    pk.z = (uint32_t)row[kc * 8 + 4] | ((uint32_t)row[kc * 8 + 5] << 16);
    pk.w = (uint32_t)row[kc * 8 + 6] | ((uint32_t)row[kc * 8 + 7] << 16);
    *reinterpret_cast<uint4*>(op + op_off(r, kc * 8, KC)) = pk;
  }
}

template <int D, int KC>
__global__ void k_operand_bf16(const float* __restrict__ feat, int dpad, int64_t n, int64_t n_rows,
                                int role, uint16_t* __restrict__ op, float* __restrict__ norm_out,
                                const unsigned long long* __restrict__ n_dev) {
  static_assert(D + 3 <= KC * 8, "operand layout");
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  if (n_dev && (int64_t)*n_dev < n) n = (int64_t)*n_dev;   // rows past a device count are padding
  uint16_t row[KC * 8];
#pragma unroll
  for (int k = 0; k < KC * 8; ++k) row[k] = 0;
  if (r < n) {
    float n2 = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float v = feat[r * dpad + i];
      n2 = fmaf(v, v, n2);
      row[i] = b_bits(__float2bfloat16_rn(role == 0 ? v : -2.f * v));
    }
    if (role == 0) {
      row[D] = row[D + 1] = row[D + 2] = b_bits(__float2bfloat16_rn(1.f));
    } else {
      const __nv_bfloat16 n1 = __float2bfloat16_rn(n2);
      const float r1 = n2 - __bfloat162float(n1);
      const __nv_bfloat16 nb = __float2bfloat16_rn(r1);
      const __nv_bfloat16 nc = __float2bfloat16_rn(r1 - __bfloat162float(nb));
      row[D] = b_bits(n1);
      row[D + 1] = b_bits(nb);
      row[D + 2] = b_bits(nc);
    }
    if (norm_out) norm_out[r] = n2;
  } else if (role == 1) {
    row[D] = b_bits(__float2bfloat16_rn(60000.f));
  }
#pragma unroll
  for (int kc = 0; kc < KC; ++kc) {
    uint4 pk;
    pk.x = (uint32_t)row[kc * 8 + 0] | ((uint32_t)row[kc * 8 + 1] << 16);
    pk.y = (uint32_t)row[kc * 8 + 2] | ((uint32_t)row[kc * 8 + 3] << 16);
    pk.z = (uint32_t)row[kc * 8 + 4] | ((uint32_t)row[kc * 8 + 5] << 16);
    pk.w = (uint32_t)row[kc * 8 + 6] | ((uint32_t)row[kc * 8 + 7] << 16);
    *reinterpret_cast<uint4*>(op + op_off_rows(r, kc * 8, KC, role == 1 ? 256 : TC_ROWS)) = pk;
  }
}

// Exact form with one FP16 term (K = 32, or 64 for D = 50): A [q | 1 1 1],
// B [-2c | n1 n2 n3] with ||c||^2 as three FP16 terms; acc misses the
// rounding of q and c to FP16 (2^-11 relative each), which the rerank's
// bound covers (2^-9 ||q|| r).
template <int D, int KC>
__global__ void k_operand_f16s(const float* __restrict__ feat, int dpad, int64_t n, int64_t n_rows,
                                int role, uint16_t* __restrict__ op, float* __restrict__ norm_out,
                                const unsigned long long* __restrict__ n_dev) {
  static_assert(D + 3 <= KC * 8, "operand layout");
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  if (n_dev && (int64_t)*n_dev < n) n = (int64_t)*n_dev;   // rows past a device count are padding
  uint16_t row[KC * 8];
#pragma unroll
  for (int k = 0; k < KC * 8; ++k) row[k] = 0;
  if (r < n) {
    float n2 = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float v = feat[r * dpad + i];
      n2 = fmaf(v, v, n2);
      row[i] = h_bits(__float2half_rn(role == 0 ? v : -2.f * v));
    }
    if (role == 0) {
      row[D] = row[D + 1] = row[D + 2] = h_bits(__float2half_rn(1.f));
    } else {
      const __half n1 = __float2half_rn(n2);
      const float r1 = n2 - __half2float(n1);
      const __half nb = __float2half_rn(r1);
      const __half nc = __float2half_rn(r1 - __half2float(nb));
      row[D] = h_bits(n1);
      row[D + 1] = h_bits(nb);
      row[D + 2] = h_bits(nc);
    }
    if (norm_out) norm_out[r] = n2;
  } else if (role == 1) {
    row[D] = h_bits(__float2half_rn(60000.f));
  }
#pragma unroll
  for (int kc = 0; kc < KC; ++kc) {
    uint4 pk;
    pk.x = (uint32_t)row[kc * 8 + 0] | ((uint32_t)row[kc * 8 + 1] << 16);
    pk.y = (uint32_t)row[kc * 8 + 2] | ((uint32_t)row[kc * 8 + 3] << 16);
    pk.z = (uint32_t)row[kc * 8 + 4] | ((uint32_t)row[kc * 8 + 5] << 16);
    pk.w = (uint32_t)row[kc * 8 + 6] | ((uint32_t)row[kc * 8 + 7] << 16);
    *reinterpret_cast<uint4*>(op + op_off_rows(r, kc * 8, KC, role == 1 ? 256 : TC_ROWS)) = pk;
  }
}

// ---------------------------------------------------------------------------
// rerank: one warp per query.  Chunks are taken in ascending order of their
// filter minimum over the split lists; the 32 entries of a chunk are examined
// by the 32 lanes (exact FP32 distance in difference form, LSH membership for
// the entries that could still enter the K best).  It stops once no entry of
// a further chunk can beat the K-th member: every entry of a chunk has
// d >= chunk minimum - delta, delta bounding |d~ - d| for any entry that
// could.  Exact form: the unlisted chunks have d~ >= T (smallest list
// threshold over the splits), so T - delta > D_K proves the result; a query
// it cannot settle is flagged for the SIMT re-run.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool lex_less(float a, int ai, float b, int bi) {
  return a < b || (a == b && ai < bi);
}

// Bitonic sort of one (value, ID) pair per lane, ascending across the lanes.
__device__ __forceinline__ void warp_sort32(float& v, int& id, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const float ov = __shfl_xor_sync(kFull, v, j);
      const int oi = __shfl_xor_sync(kFull, id, j);
      const bool keep_small = ((lane & j) == 0) == ((lane & k) == 0);
      if (keep_small == lex_less(ov, oi, v, id)) {
        v = ov;
        id = oi;
      }
    }
  }
}

// Merges 32 ascending candidates (one per lane) into the ascending K best
// held by lanes 0..K-1: min(A[j], B[31 - j]) is a bitonic sequence holding
// the 32 smallest of both, which a bitonic merge sorts.
__device__ __forceinline__ void warp_merge_best(float& bd, int& bi, float v, int id, int K, int lane) {
  float a = lane < K ? bd : FLT_MAX;
  int ai = lane < K ? bi : INT_MAX;
  const float rb = __shfl_sync(kFull, v, 31 - lane);
  const int rbi = __shfl_sync(kFull, id, 31 - lane);
  if (lex_less(rb, rbi, a, ai)) {
    a = rb;
    ai = rbi;
  }
#pragma unroll
  for (int j = 16; j > 0; j >>= 1) {
    const float ov = __shfl_xor_sync(kFull, a, j);
    const int oi = __shfl_xor_sync(kFull, ai, j);
    if (((lane & j) == 0) == lex_less(ov, oi, a, ai)) {
      a = ov;
      ai = oi;
    }
  }
  bd = a;
  bi = ai;
}

// t-of-L membership: at least tmin of the entry's L bucket keys equal the
// query's.  Eight tables at a time (loads issued together); stops at tmin
// hits.
__device__ __forceinline__ bool lsh_member(const uint64_t* __restrict__ dk, const uint64_t* qk, int L,
                                           int tmin) {
  int hits = 0;
  for (int l0 = 0; l0 < L && hits < tmin; l0 += 8) {
    uint64_t kk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) kk[j] = l0 + j < L ? __ldg(dk + l0 + j) : 0ull;
#pragma unroll
    for (int j = 0; j < 8; ++j) hits += (l0 + j < L && kk[j] == qk[l0 + j]) ? 1 : 0;
  }
  return hits >= tmin;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// queries (warps) per block: the staged rows of wide features (D = 50, two
// buffers of 32 rows of 52 floats per warp) would exceed 48 KB of static
// shared memory at four warps.  Seven blocks of four warps fill the shared
// memory at D <= 32 (73 registers a thread: no spills).
__host__ __device__ constexpr int rerank_warps(int D) { return D > 32 ? 2 : 4; }

template <int D, int MC>
__global__ __launch_bounds__(rerank_warps(D) * 32, D > 32 ? 8 : 7) void k_rerank(
    const float* __restrict__ qfeat, int dpad, const float* __restrict__ qn_arr,
    const uint64_t* __restrict__ qkeys, int64_t nq, const float* __restrict__ dfeat,
    const uint64_t* __restrict__ dkeys, int64_t nd, int L, int tmin, const float* __restrict__ lm,
    const int32_t* __restrict__ lc, int nsplit, int K, int exact, float c_qr, float c_sq, float c_abs,
    int32_t* __restrict__ nbr, float* __restrict__ dist, int32_t* __restrict__ fb_list,
    unsigned long long* __restrict__ fb_count, const int32_t* __restrict__ qmap,
    const unsigned long long* __restrict__ nq_dev) {
  constexpr int kDP = (D + 3) / 4 * 4;   // feature row stride (floats)
  constexpr int kRow4 = kDP / 4;         // 16-byte pieces per row
  // two buffers per warp: the next chunk's rows arrive (cp.async) while the
  // current chunk is examined
  constexpr int kRerankWarps = rerank_warps(D);
  // relative error of the FP32 difference-form distance of D terms
  constexpr float kRelD = D > 25 ? 8e-6f : 4e-6f;
  __shared__ float4 s_rows[kRerankWarps][2][32 * kRow4];
  __shared__ uint64_t s_qk[kRerankWarps][32];   // the query's bucket keys (L <= 32)
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= nq || (nq_dev && q >= (int64_t)*nq_dev)) return;   // warp-uniform
  // query q of this launch is query oq of the call (qmap: a compacted subset)
  const int64_t oq = qmap ? qmap[q] : q;
  if (lane < L) s_qk[wib][lane] = qkeys[q * L + lane];
  // the query's feature in shared memory (read as 16-byte pieces beside the
  // rows; registers stay free for the lists and the K best)
  __shared__ float4 s_q4[kRerankWarps][kRow4];
  if (lane < kRow4) s_q4[wib][lane] = reinterpret_cast<const float4*>(qfeat + q * dpad)[lane];
  const float qn = qn_arr[q];
  const float qnorm = sqrtf(qn);
  // The chunk lists of every split sit in registers: lane j holds entry j of
  // the list of split s in lv[s] / lcv[s] (FLT_MAX past nsplit or MC), and
  // hd[s] (the same in every lane) is the split's next unexamined entry, so
  // choosing the next chunk takes shuffles and no memory access.
  constexpr int kMaxSplit = 8;
  float lv[kMaxSplit];
  int lcv[kMaxSplit], hd[kMaxSplit];
#pragma unroll
  // An entry naming no chunk of the dictionary counts as "none" (FLT_MAX):
  // the filter writes only real chunks or (FLT_MAX, -1), but a filter that
  // gave up (a wait ran out) leaves its lists unwritten, and their contents
  // must not become addresses.
  for (int s = 0; s < kMaxSplit; ++s) {
    const bool has = s < nsplit && lane < MC;
    const int64_t o = ((int64_t)s * nq + q) * MC + lane;
    const int c = has ? lc[o] : -1;
    const bool real = c >= 0 && (int64_t)c * 32 < nd;
    lv[s] = real ? lm[o] : FLT_MAX;
    lcv[s] = real ? c : -1;
    hd[s] = 0;
  }
  // T: the smallest list threshold (MC-th listed minimum) over the splits
  float T = FLT_MAX;
#pragma unroll
  for (int s = 0; s < kMaxSplit; ++s)
    if (s < nsplit) T = fminf(T, __shfl_sync(kFull, lv[s], MC - 1));
  // the listed chunk with the smallest minimum among the list heads (ties:
  // lower split) and its split; -1 when the lists are exhausted
  auto peek = [&](float& best, int& bs) -> int {
    best = FLT_MAX;
    bs = -1;
    int ch = -1;
#pragma unroll
    for (int s = 0; s < kMaxSplit; ++s) {
      if (s < nsplit) {
        const float v = __shfl_sync(kFull, lv[s], hd[s] & 31);
        const int c = __shfl_sync(kFull, lcv[s], hd[s] & 31);
        if (hd[s] < MC && v < best) {
          best = v;
          bs = s;
          ch = c;
        }
      }
    }
    return ch;
  };
  auto advance = [&](int bs) {
#pragma unroll
    for (int s = 0; s < kMaxSplit; ++s)
      if (s == bs) ++hd[s];
  };
  // the chunk's rows are contiguous: 16-byte asynchronous copies
  auto stage = [&](int c, int b) {
    if (c >= 0) {
      const int64_t e0 = (int64_t)c * 32;
      const int nrows = (int)(nd - e0 < 32 ? nd - e0 : 32);
      const float4* g = reinterpret_cast<const float4*>(dfeat + e0 * kDP);
      float4* dst = s_rows[wib][b];
      for (int f = lane; f < nrows * kRow4; f += 32) cp_async16(dst + f, g + f);
    }
    cp_async_commit();
  };
  // the K best members so far, ascending by (distance, ID): lane j < K holds rank j
  float bd = FLT_MAX;
  int bi = INT_MAX;
  float dK = FLT_MAX, delta = 0.f;
  int iK = INT_MAX, members = 0;
  float best;
  int bs;
  int chunk = peek(best, bs);
  int buf = 0;
  if (chunk >= 0) {
    advance(bs);
    stage(chunk, 0);
  }
  while (chunk >= 0) {
    // the next chunk in order starts arriving in the other buffer, which held
    // the previous chunk: the __syncwarp puts every lane past its reads
    float nbest;
    int nbs;
    const int nchunk = peek(nbest, nbs);
    __syncwarp();
    stage(nchunk, buf ^ 1);
    cp_async_wait<1>();   // this lane's copies of the current chunk are done
    __syncwarp();         // ... and every lane's
    const int64_t e0 = (int64_t)chunk * 32;
    const int64_t e = e0 + lane;
    const int nrows = (int)(nd - e0 < 32 ? nd - e0 : 32);
    float dd = FLT_MAX;
    if (lane < nrows) {
      const float4* srow = s_rows[wib][buf];
      dd = 0.f;
      // each 16-byte piece is consumed as it is read (the order of i)
#pragma unroll
      for (int k = 0; k < kRow4; ++k) {
        const float4 v4 = srow[lane * kRow4 + k];
        const float x4[4] = {v4.x, v4.y, v4.z, v4.w};
        const float4 q4 = s_q4[wib][k];
        const float qx4[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (4 * k + t < D) {
            const float df = qx4[t] - x4[t];
            dd = fmaf(df, df, dd);
          }
        }
      }
    }
    // entries that could still enter the K best: LSH membership
    int eid = dd != FLT_MAX ? (int)e : INT_MAX;
    bool mem = false;
    if (members < K) {
      // fewer than K members so far (the first chunk): every entry could
      // enter, so the chunk is sorted by (distance, ID) across the lanes and
      // membership taken in that order, a few lanes past the members still
      // needed at a time; once K members are known no later entry can enter
      warp_sort32(dd, eid, lane);
      const int need = K - members;
      int found = 0;
      for (int j0 = 0; j0 < 32 && found < need;) {
        const int j1 = min(32, j0 + need - found + 4);
        if (lane >= j0 && lane < j1 && dd != FLT_MAX)
          mem = lsh_member(dkeys + (int64_t)eid * L, s_qk[wib], L, tmin);
        found = __popc(__ballot_sync(kFull, mem));
        j0 = j1;
      }
    } else if (dd != FLT_MAX && (dd < dK || (dd == dK && eid < iK))) {
      mem = lsh_member(dkeys + (int64_t)eid * L, s_qk[wib], L, tmin);
    }
    unsigned mm = __ballot_sync(kFull, mem);
    members += __popc(mm);
    if (__popc(mm) > 4) {
      // many (the first chunks): sort the chunk's members across the lanes
      // and merge them with the K best
      float v = mem ? dd : FLT_MAX;
      int id = mem ? eid : INT_MAX;
      warp_sort32(v, id, lane);
      warp_merge_best(bd, bi, v, id, K, lane);
      mm = 0;
    }
    // few: insert them one by one in ascending (distance, ID) order
    while (mm) {
      const bool mine = (mm >> lane) & 1u;
      float v = mine ? dd : FLT_MAX;
      int id = mine ? eid : INT_MAX;
      int src = lane;
#pragma unroll
      for (int off = 16; off; off >>= 1) {
        const float ov = __shfl_xor_sync(kFull, v, off);
        const int oi = __shfl_xor_sync(kFull, id, off);
        const int osr = __shfl_xor_sync(kFull, src, off);
        if (ov < v || (ov == v && oi < id)) {
          v = ov;
          id = oi;
          src = osr;
        }
      }
      mm &= ~(1u << src);
      const bool before = lane < K && (bd < v || (bd == v && bi < id));
      const int pos = __popc(__ballot_sync(kFull, before));
      if (pos >= K) break;   // the rest are larger still
      const float ud = __shfl_up_sync(kFull, bd, 1);
      const int ui = __shfl_up_sync(kFull, bi, 1);
      if (lane == pos) {
        bd = v;
        bi = id;
      } else if (lane > pos && lane < K) {
        bd = ud;
        bi = ui;
      }
    }
    if (members >= K) {
      dK = __shfl_sync(kFull, bd, K - 1);
      iK = __shfl_sync(kFull, bi, K - 1);
      // an entry that could beat dK has ||c|| <= ||q|| + sqrt(dK)
      const float rc = qnorm + sqrtf(dK) * 1.001f + 1e-6f;
      delta = c_qr * qnorm * rc + c_sq * (rc * rc + qn) + kRelD * dK + c_abs * (qnorm + rc) + 1e-12f;
    }
    // stop once no entry of a further chunk can beat the K-th member
    if (nchunk < 0 || (members >= K && nbest - delta > dK)) break;
    advance(nbs);
    chunk = nchunk;
    buf ^= 1;
  }
  cp_async_wait<0>();   // no copy may still target this warp's buffers
  const bool flagged = members < K || (exact && !(T - delta > dK));
  if (flagged) {
    if (lane == 0) {
      const unsigned long long slot = atomicAdd(fb_count, 1ull);
      fb_list[slot] = (int32_t)oq;
    }
    return;
  }
  if (lane < K) {
    nbr[oq * K + lane] = bi;
    dist[oq * K + lane] = bd;
  }
}

// Compacts the queries listed in idx[0 .. min(*count, cap)) -- their
// features and bucket keys -- for a second search; listed queries at or past
// cap go to the list `over` (count *over_count).  One thread per listed query.
__global__ void k_gather_queries(const int32_t* __restrict__ idx, const unsigned long long* __restrict__ count,
                                 int64_t cap, const float* __restrict__ feat, int dpad,
                                 const uint64_t* __restrict__ keys, int L, float* __restrict__ cfeat,
                                 uint64_t* __restrict__ ckeys, int32_t* __restrict__ over,
                                 unsigned long long* __restrict__ over_count) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (int64_t)*count) return;
  const int64_t q = idx[j];
  if (j >= cap) {
    const unsigned long long slot = atomicAdd(over_count, 1ull);
    over[slot] = (int32_t)q;
    return;
  }
  for (int i = 0; i < dpad; i += 4)
    *reinterpret_cast<float4*>(cfeat + j * dpad + i) = *reinterpret_cast<const float4*>(feat + q * dpad + i);
  for (int l = 0; l < L; ++l) ckeys[j * L + l] = keys[q * L + l];
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

int64_t tc_rows_padded(int64_t n, bool even_tiles) {
  int64_t t = (n + TC_ROWS - 1) / TC_ROWS;
  if (even_tiles && (t & 1)) ++t;
  if (t == 0) t = even_tiles ? 2 : 1;
  return t * TC_ROWS;
}

int tc_kc(int d, int precision) {
  if (precision == 0) return d <= 25 ? 10 : 20;
  return d + 3 <= 32 ? 4 : 8;   // BF16 and single-term FP16
}

cudaError_t launch_operand(const float* feat, int dpad, int d, int64_t n, int64_t n_rows, int role,
                           int precision, uint16_t* op, float* norm_out, cudaStream_t st,
                           const unsigned long long* n_dev) {
  const int blocks = (int)((n_rows + 127) / 128);
#define ZOOM_OP(DD)                                                                                  \
  do {                                                                                               \
    if (precision == 0)                                                                              \
      k_operand_f16x3<DD, (DD <= 25 ? 10 : 20)><<<blocks, 128, 0, st>>>(feat, dpad, n, n_rows, role, op, \
                                                                         norm_out, n_dev);           \
    else if (precision == 1)                                                                         \
      k_operand_bf16<DD, (DD + 3 <= 32 ? 4 : 8)><<<blocks, 128, 0, st>>>(feat, dpad, n, n_rows, role, op, \
                                                                          norm_out, n_dev);          \
    else                                                                                             \
      k_operand_f16s<DD, (DD + 3 <= 32 ? 4 : 8)><<<blocks, 128, 0, st>>>(feat, dpad, n, n_rows, role, op, \
                                                                          norm_out, n_dev);          \
  } while (0)
  switch (d) {
    case 9: ZOOM_OP(9); break;
    case 25: ZOOM_OP(25); break;
    case 18: ZOOM_OP(18); break;
    case 50: ZOOM_OP(50); break;
    default: return cudaErrorInvalidValue;
  }
#undef ZOOM_OP
  return cudaGetLastError();
}

size_t tc_smem_bytes(int KC, int MC) {
  // alignment pad + operand tiles + barriers + the epilogue's buffers (and lists)
  return 1024 + (size_t)(2 + tc_stages(KC, MC)) * KC * TC_ROWS * 16 + kBarBytes + (size_t)tc_epi_bytes(KC, MC);
}

int tc_list_size(int precision, int K, int rerank_mult) {
  if (precision != 1) return K <= 12 ? 16 : 32;
  return rerank_mult * K <= 16 ? 16 : 32;
}

size_t tw_smem_bytes(int KC, int MC, bool packed) {
  return 1024 + (size_t)2 * KC * TC_ROWS * 16 + (size_t)tw_stages(KC, MC, packed) * KC * TW_ROWS * 16 +
         kBarBytes + (size_t)tw_epi_bytes(MC, packed);
}

bool tc_wide_form(int precision, int kc) { return precision != 0 && (kc == 4 || kc == 8); }

template <int KC, int MC, uint32_t T, bool P>
static cudaError_t run_tw_kernel(const TcArgs& args, int grid, cudaStream_t st) {
  auto kern = k_knn_tw<KC, MC, T, P>;
  const size_t smem = tw_smem_bytes(KC, MC, P);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (fa.maxThreadsPerBlock < 352) return cudaErrorLaunchOutOfResources;
  kern<<<grid, 352, smem, st>>>(args);
  return cudaGetLastError();
}

template <int KC, int MC, uint32_t T>
static cudaError_t run_tc_kernel(const TcArgs& args, int grid, size_t smem, cudaStream_t st) {
  auto kern = k_knn_tc<KC, MC, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the block's warps must fit the register file as compiled (an SM
  // sub-partition holds 16K registers and takes every fourth warp)
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (fa.maxThreadsPerBlock < tc_threads(KC, MC)) return cudaErrorLaunchOutOfResources;
  kern<<<grid, tc_threads(KC, MC), smem, st>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_knn_tc(const uint16_t* qop, const float* qn, int64_t nq, const uint16_t* dop,
                          int64_t nd, int precision, int kc, int MC, int nsplit, int tail_split, int grid,
                          float* out_d, int32_t* out_id, unsigned int* status, cudaStream_t st,
                          const unsigned long long* nq_dev, uint64_t wait_ns, int inject) {
  if (tc_wide_form(precision, kc)) {
    // the wide-step kernel: items of 256 queries x a part of the 256-row steps
    if (nq_dev || (MC != 16 && MC != 32)) return cudaErrorInvalidValue;
    TcArgs a;
    a.wait_ns = wait_ns > 0 ? wait_ns : kWaitNs;
    a.inject = inject;
    a.qop = qop;
    a.qn = qn;
    a.dop = dop;
    a.nq = nq;
    a.nq_dev = nullptr;
    a.nd = nd;
    a.nq_pairs = (int)((nq + 2 * TC_ROWS - 1) / (2 * TC_ROWS));
    a.nd_tiles = (int)((nd + TW_ROWS - 1) / TW_ROWS);   // 256-row steps
    a.nsplit = nsplit;
    a.tiles_per_split = (a.nd_tiles + nsplit - 1) / nsplit;
    a.out_d = out_d;
    a.out_id = out_id;
    a.status = status;
    a.tail_split = tail_split;
    if (tail_split > 0 && nsplit != tail_split) return cudaErrorInvalidValue;
    const int items = tail_split > 0 ? a.nq_pairs : a.nsplit * a.nq_pairs;
    grid = grid < items ? grid : items;
    a.full_rounds = tail_split > 0 ? a.nq_pairs / grid : 0;
    // The BF16 form's 32-chunk lists are packed while the chunk numbers leave
    // the keys at least 15 value bits (up to 2^17 chunks, 4,194,304 entries):
    // there the merges dominate the list time (measured: 8 % off the filter
    // with 1M entries, 2 % with 4M); 16-chunk lists merge rarely and run
    // slightly faster unpacked.
    a.id_bits = 3;
    while ((int64_t{1} << a.id_bits) < (int64_t)a.nd_tiles * 8) ++a.id_bits;
    const bool packed = precision == 1 && MC == 32 && a.id_bits <= 17;
#define ZOOM_TW(KC, T) \
  return MC == 16 ? run_tw_kernel<KC, 16, T, false>(a, grid, st) : run_tw_kernel<KC, 32, T, false>(a, grid, st)
    if (precision == 1 && kc == 4 && packed) return run_tw_kernel<4, 32, 1, true>(a, grid, st);
    if (precision == 1 && kc == 8 && packed) return run_tw_kernel<8, 32, 1, true>(a, grid, st);
    if (precision == 2 && kc == 4) ZOOM_TW(4, 0);
    if (precision == 2 && kc == 8) ZOOM_TW(8, 0);
    if (precision == 1 && kc == 4) ZOOM_TW(4, 1);
    if (precision == 1 && kc == 8) ZOOM_TW(8, 1);
#undef ZOOM_TW
    return cudaErrorInvalidValue;
  }
  TcArgs a;
  a.wait_ns = wait_ns > 0 ? wait_ns : kWaitNs;
  a.inject = inject;
  a.qop = qop;
  a.qn = qn;
  a.dop = dop;
  a.nq = nq;
  a.nq_dev = nq_dev;
  if (nq_dev && tail_split > 0) return cudaErrorInvalidValue;   // the tail split needs the count on the host
  a.nd = nd;
  a.nq_pairs = (int)((nq + 2 * TC_ROWS - 1) / (2 * TC_ROWS));
  a.nd_tiles = (int)((nd + TC_ROWS - 1) / TC_ROWS);
  a.nsplit = nsplit;
  a.tiles_per_split = (a.nd_tiles + nsplit - 1) / nsplit;
  a.out_d = out_d;
  a.out_id = out_id;
  a.status = status;
  a.tail_split = tail_split;
  if (tail_split > 0 && nsplit != tail_split) return cudaErrorInvalidValue;
  if (MC != 16 && MC != 32) return cudaErrorInvalidValue;
  const size_t smem = tc_smem_bytes(kc, MC);
  const int items = tail_split > 0 ? a.nq_pairs : a.nsplit * a.nq_pairs;
  grid = grid < items ? grid : items;
  a.full_rounds = tail_split > 0 ? a.nq_pairs / grid : 0;
#define ZOOM_TC(KC, T)                                                                            \
  return MC == 16 ? run_tc_kernel<KC, 16, T>(a, grid, smem, st) : run_tc_kernel<KC, 32, T>(a, grid, smem, st)
  if (precision == 0 && kc == 10) ZOOM_TC(10, 0);
  if (precision == 0 && kc == 20) ZOOM_TC(20, 0);
  if (precision == 2 && kc == 4) ZOOM_TC(4, 0);
  if (precision == 2 && kc == 8) ZOOM_TC(8, 0);
  if (precision == 1 && kc == 4) ZOOM_TC(4, 1);
  if (precision == 1 && kc == 8) ZOOM_TC(8, 1);
#undef ZOOM_TC
  return cudaErrorInvalidValue;
}

template <int D, int MC>
static cudaError_t rerank_k(int K, const float* qfeat, int dpad, const float* qn, const uint64_t* qkeys,
                            int64_t nq, const float* dfeat, const uint64_t* dkeys, int64_t nd, int L,
                            int tmin, const float* ld, const int32_t* li, int nsplit, int exact, float c_qr,
                            float c_sq, float c_abs, int32_t* nbr, float* dist, int32_t* fb,
                            unsigned long long* fb_count, const int32_t* qmap,
                            const unsigned long long* nq_dev, cudaStream_t st) {
  constexpr int kRerankWarps = rerank_warps(D);
  const int64_t blocks = (nq + kRerankWarps - 1) / kRerankWarps;   // one warp per query
  k_rerank<D, MC><<<(unsigned)blocks, kRerankWarps * 32, 0, st>>>(qfeat, dpad, qn, qkeys, nq, dfeat, dkeys, nd, L, tmin, ld,
                                                    li, nsplit, K, exact, c_qr, c_sq, c_abs, nbr, dist, fb,
                                                    fb_count, qmap, nq_dev);
  return cudaGetLastError();
}

cudaError_t launch_rerank(int d, int MC, int K, const float* qfeat, int dpad, const float* qn,
                          const uint64_t* qkeys, int64_t nq, const float* dfeat, const uint64_t* dkeys,
                          int64_t nd, int L, int tmin, const float* ld, const int32_t* li, int nsplit,
                          int form, int32_t* nbr, float* dist, int32_t* fb, unsigned long long* fb_count,
                          cudaStream_t st, const int32_t* qmap, const unsigned long long* nq_dev) {
  if (nsplit > 8 || K < 1 || K > 16 || dpad != (d + 3) / 4 * 4 || form < 0 || form > 2)
    return cudaErrorInvalidValue;
  if (nq == 0) return cudaSuccess;
  // |d~ - d| <= c_qr ||q|| r + c_sq (r^2 + ||q||^2) + c_abs (||q|| + r)
  // + 4e-6 d for an entry with ||c|| <= r.  form 1 (FP16 hi/lo split): the
  // dropped q_lo.c_lo term and the rounding of the split, within
  // 6 * 2^-16 ||q|| r, FP32 accumulation of 80 terms and the FP32 rerank
  // (2^-16 (r^2 + ||q||^2), 4e-6 d).  form 2 (one FP16 term): q and c each
  // rounded to 11 significant bits, 2 (2^-10 + 2^-22) ||q|| r for the
  // product term (Cauchy-Schwarz), 1.05 * 2^-9 with the accumulation of 32
  // terms.  Both: FP16 subnormals round with an absolute error up to 2^-25
  // per element, 2 * 2^-25 * sum(|q_i| + |c_i|) <= 2^-23 sqrt(D) (||q|| + r)
  // with slack.  form 0 (BF16): each operand rounded to 8 significant bits
  // (2 * 2^-8 ||q|| r for the product term), 32 FP32 accumulations; used only
  // to stop examining (no proof).  Twice the operand width (gradient
  // features of 5 x 5 patches, K = 160 or 64) doubles the accumulation
  // terms: the coefficients are doubled (the kernel doubles the relative
  // term of its FP32 rerank for D > 25 too).
  const int prec = form == 1 ? 0 : (form == 0 ? 1 : 2);
  const float wide = tc_kc(d, prec) > (prec == 0 ? 10 : 4) ? 2.f : 1.f;
  const float c_qr = wide * (form == 1 ? 6.f / 65536.f : form == 2 ? 1.05f / 512.f : 1.05f / 128.f);
  const float c_sq = wide * (form == 0 ? 1.f / 262144.f : 1.f / 65536.f);
  const float c_abs = 1.1920929e-07f * sqrtf((float)d);   // 2^-23 sqrt(D)
  const int exact = form != 0;
#define ZOOM_RR(DD, MM)                                                                          \
  return rerank_k<DD, MM>(K, qfeat, dpad, qn, qkeys, nq, dfeat, dkeys, nd, L, tmin, ld, li, nsplit, \
                          exact, c_qr, c_sq, c_abs, nbr, dist, fb, fb_count, qmap, nq_dev, st)
  if (d == 25 && MC == 16) ZOOM_RR(25, 16);
  if (d == 25 && MC == 32) ZOOM_RR(25, 32);
  if (d == 9 && MC == 16) ZOOM_RR(9, 16);
  if (d == 9 && MC == 32) ZOOM_RR(9, 32);
  if (d == 18 && MC == 16) ZOOM_RR(18, 16);
  if (d == 18 && MC == 32) ZOOM_RR(18, 32);
  if (d == 50 && MC == 16) ZOOM_RR(50, 16);
  if (d == 50 && MC == 32) ZOOM_RR(50, 32);
#undef ZOOM_RR
  return cudaErrorInvalidValue;
}

cudaError_t launch_gather_queries(const int32_t* idx, const unsigned long long* count, int64_t max_count,
                                  int64_t cap, const float* feat, int dpad, const uint64_t* keys, int L,
                                  float* cfeat, uint64_t* ckeys, int32_t* over, unsigned long long* over_count,
                                  cudaStream_t st) {
  if (max_count == 0) return cudaSuccess;
  if (dpad % 4) return cudaErrorInvalidValue;
  k_gather_queries<<<(unsigned)((max_count + 127) / 128), 128, 0, st>>>(idx, count, cap, feat, dpad, keys, L,
                                                                         cfeat, ckeys, over, over_count);
  return cudaGetLastError();
}
