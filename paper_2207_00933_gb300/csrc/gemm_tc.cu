// One contraction step (Section 6.1: C = A B^T over the shared cut-edge
// index) on the tcgen05 tensor cores in split-BF16.
//
// Every operand is held as three BF16 planes x = hi + mid + lo (each plane
// the round-to-nearest of what the previous ones left).  The product keeps
// the six terms of order <= 2 -- hi*hi, hi*mid, mid*hi, hi*lo, mid*mid,
// lo*hi -- all accumulated in one FP32 accumulator in tensor memory, which
// gives about FP32 accuracy for the signed I/X/Y/Z sums.
//
// Persistent CTAs (one per SM) walk the 128 x 128 output tiles; 6 warps:
//   warp 0 (one thread): TMA producer -- for each 64-wide block of the
//     shared index it loads the three A planes and three B planes
//     (128 x 64 BF16 each, 128-byte swizzle) into one of two pipeline stages;
//   warp 1 (one thread): allocates 2 x 128 TMEM columns and issues
//     tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128, N = 128, K = 16):
//     6 plane pairs x 4 K-slices per stage, then commits the stage back to
//     the producer;
//   warps 2-5: epilogue -- wait for a tile's last commit, read the
//     accumulator rows with tcgen05.ld (warp w reads TMEM lanes 32*(w%4) ..
//     +31), scale by alpha, write through rowmap/colmap (vector stores where
//     the 16 columns are contiguous; FP32, FP64 or BF16 planes), add the
//     written values into the per-CTA probability sum, and hand the TMEM
//     buffer back.  Two accumulator buffers let the epilogue of one tile run
//     under the MMAs of the next.
// Every mbarrier wait is bounded; on timeout the CTA records an error code,
// drains its own copies (bounded) and frees its TMEM before returning.
#include <cuda.h>

#include "common.cuh"

namespace sqc {

namespace {

constexpr int kBM = 128;
constexpr int kKAlign = 64;        // the shared index is padded to a multiple of this
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, each half of the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kSpinLimit = 1u << 24;

// Tile configurations: BN output columns per tile, BK shared-index columns
// per stage (BK BF16 = one swizzle row: 64 -> 128-byte swizzle, 32 ->
// 64-byte swizzle), STAGES pipeline stages.
//   128 x 128, BK 64, 2 stages of 96 KB (narrow steps)
//   128 x 256, BK 32, 3 stages of 72 KB: 25% less operand traffic per flop
template <int BN_, int BK_, int STAGES_>
struct TcCfg {
  static constexpr int BN = BN_, BK = BK_, STAGES = STAGES_;
  static constexpr int kTileA = kBM * BK * 2;
  static constexpr int kTileB = BN * BK * 2;
  static constexpr int kStageBytes = 3 * kTileA + 3 * kTileB;
  static constexpr int kTmemCols = BN;          // one FP32 accumulator buffer
  static constexpr int kSmemBytes = STAGES * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int kSwizzleBytes = BK * 2;
  // instruction descriptor: D = FP32, A = B = BF16, both K-major, M x N
  static constexpr uint32_t kIdesc =
      (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(kBM >> 4) << 24);
  // the same with N = BN / 2 (half-width tail units of the pair kernel)
  static constexpr uint32_t kIdescHalf =
      (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 4) << 17) | (uint32_t(kBM >> 4) << 24);
};
using CfgNarrow = TcCfg<128, 64, 2>;
using CfgWide = TcCfg<256, 32, 3>;
//   the same in 2-CTA pairs sharing B (a 16-deep, 6-stage, 32-byte-swizzle
//   variant measured 19% slower)
using CfgPair = CfgWide;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// The same load delivered to every CTA of the cluster in `mask`, at the same
// shared-memory offset, completing on the barrier at the same offset in each.
__device__ __forceinline__ void tma_load_3d_mc(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, "
      "{%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major tile of 8-row swizzle atoms
// (rows of SW bytes: 128-byte or 64-byte swizzle), atoms 8 x SW bytes apart.
template <int SW>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  static_assert(SW == 128 || SW == 64 || SW == 32, "swizzle");
  uint64_t d = 0;
  d |= uint64_t((addr & 0x3FFFFu) >> 4);   // start address
  d |= uint64_t(1) << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= uint64_t((8 * SW) >> 4) << 32;      // stride byte offset: next 8-row group
  d |= uint64_t(1) << 46;                  // descriptor version
  d |= uint64_t(SW == 128 ? 2 : (SW == 64 ? 4 : 6)) << 61;  // swizzle mode
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Commit arriving on the barrier at the same offset in every CTA of `mask`.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane (one
// load, one wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Store 16 consecutive columns of one output row.  `contig`: the columns'
// offsets are consecutive and 16-byte aligned, so vector stores are used.
__device__ __forceinline__ void store16(const GemmTcArgs& a, uint64_t off, bool contig, const float* f,
                                        const uint64_t* colmap, int64_t col0, uint64_t rbase, int ncols) {
  if (contig && ncols == 16) {
    if (a.kind == OUT_F32) {
      float4* p = reinterpret_cast<float4*>(static_cast<float*>(a.C) + off);
#pragma unroll
      for (int q = 0; q < 4; ++q) p[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
      return;
    }
    if (a.kind == OUT_F64) {
      double2* p = reinterpret_cast<double2*>(static_cast<double*>(a.C) + off);
#pragma unroll
      for (int q = 0; q < 8; ++q) p[q] = make_double2(double(f[2 * q]), double(f[2 * q + 1]));
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j < ncols) store_out_f(a.C, a.kind, a.plane_stride, rbase + colmap[col0 + j], f[j]);
}

// Persistent: grid = min(tiles, SMs); CTA b takes tiles b, b + grid, ...
// The accumulator is double-buffered in TMEM (2 x BN columns) so that the
// epilogue of one tile overlaps the loads and MMAs of the next.
// PAIR: clusters of two CTAs on vertically adjacent tiles (same columns)
// share every B tile: each CTA loads half of its rows and multicasts them to
// both, so B is read from L2 once per pair.  A stage of either CTA is then
// refilled only after both CTAs' MMAs have consumed it (the MMA commits
// arrive on both CTAs' `empty` barriers).  When the pair units leave a last
// wave at most half full, its units are split into two half-width units
// (N = BN / 2, B loaded by rank 0 alone and multicast), so that the tail
// takes about half a unit's time instead of a whole one.
template <class Cfg, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmTcArgs a) {
  constexpr int kBN = Cfg::BN, kBK = Cfg::BK, kStages = Cfg::STAGES;
  constexpr int kTileA = Cfg::kTileA, kTileB = Cfg::kTileB, kStageBytes = Cfg::kStageBytes;
  constexpr int kTmemCols = Cfg::kTmemCols, kSW = Cfg::kSwizzleBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;      // [2]: MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;        // [2]: epilogue -> MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ double red[kThreads / 32];
  __shared__ int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tiles_n = a.Np / kBN;
  const int tn_shift = __ffsll(tiles_n) - 1;
  const int64_t ntiles = (a.Mp / kBM) * tiles_n;
  const int nk = int(a.Kp / kBK);
  // work units: tiles, or (PAIR) pairs of vertically adjacent tiles, this
  // CTA taking the one of its cluster rank
  uint32_t rank = 0;
  if constexpr (PAIR) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const int64_t unit0 = PAIR ? int64_t(blockIdx.x >> 1) : int64_t(blockIdx.x);
  const int64_t unit_step = PAIR ? int64_t(gridDim.x >> 1) : int64_t(gridDim.x);
  const int64_t nwide = PAIR ? ntiles / 2 : ntiles;
  const int64_t tail = nwide % unit_step;
  const bool split = PAIR && tail > 0 && 2 * tail <= unit_step;
  const int64_t wide_end = split ? nwide - tail : nwide;        // units [wide_end, nunits) are half-width
  const int64_t nunits = split ? wide_end + 2 * tail : nwide;
  // unit u -> (tile row origin, column origin, half width)
  auto unit_of = [&](int64_t u, int64_t* m0, int64_t* n0, bool* half) {
    int64_t wu = u, noff = 0;
    *half = u >= wide_end;
    if (*half) {
      wu = wide_end + ((u - wide_end) >> 1);
      noff = ((u - wide_end) & 1) * (kBN / 2);
    }
    *m0 = ((wu >> tn_shift) * (PAIR ? 2 : 1) + rank) * kBM;
    *n0 = (wu & (tiles_n - 1)) * kBN + noff;
  };

  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], PAIR ? 2 : 1);     // PAIR: both CTAs' MMAs
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);    // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // the partner's multicasts and commits target this CTA's barriers: both
  // CTAs' barriers are initialised before either starts
  if constexpr (PAIR) cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  double sum_d = 0.0;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: one continuous ring of stages across all tiles
    int64_t it = 0, issued = 0;
    for (int64_t u = unit0; u < nunits && !failed; u += unit_step) {
      int64_t um0, un0;
      bool half;
      unit_of(u, &um0, &un0, &half);
      const int m0 = int(um0), n0 = int(un0);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = int(it % kStages);
        const int64_t use = it / kStages;
        if (use > 0 && !mbar_wait(&empty[s], uint32_t((use - 1) & 1))) {
          atomicExch(&failed, 1);
          break;
        }
        uint8_t* st = smem + s * kStageBytes;
        // a half-width unit's stage holds the A planes and the first BN / 2
        // rows of each B plane
        mbar_expect_tx(&full[s], half ? 3 * kTileA + 3 * (kTileB / 2) : kStageBytes);
        for (int p = 0; p < 3; ++p) tma_load_3d(st + p * kTileA, &tmA, kb * kBK, m0, p, &full[s]);
        if constexpr (PAIR) {
          if (half) {
            // the unit's BN / 2 B rows (one box of the map), loaded by rank
            // 0 alone, to both CTAs
            if (rank == 0)
              for (int p = 0; p < 3; ++p)
                tma_load_3d_mc(st + 3 * kTileA + p * kTileB, &tmB, kb * kBK, n0, p, &full[s], uint16_t(0x3));
          } else {
            // this CTA's half of the B rows, to both CTAs
            for (int p = 0; p < 3; ++p)
              tma_load_3d_mc(st + 3 * kTileA + p * kTileB + int(rank) * (kTileB / 2), &tmB, kb * kBK,
                             n0 + int(rank) * (kBN / 2), p, &full[s], uint16_t(0x3));
          }
        } else {
          for (int p = 0; p < 3; ++p) tma_load_3d(st + 3 * kTileA + p * kTileB, &tmB, kb * kBK, n0, p, &full[s]);
        }
        issued = it + 1;
      }
    }
    // drain: every stage we filled must have landed before the CTA exits
    for (int64_t j = (issued > kStages ? issued - kStages : 0); j < issued; ++j)
      if (!mbar_wait(&full[j % kStages], uint32_t((j / kStages) & 1))) atomicExch(&failed, 1);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
    constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
    int64_t it = 0, t = 0;
    for (int64_t u = unit0; u < nunits && !failed; u += unit_step, ++t) {
      const uint32_t idesc = u >= wide_end ? Cfg::kIdescHalf : Cfg::kIdesc;
      const int buf = int(t & 1);
      const int64_t use = t >> 1;
      if (use > 0 && !mbar_wait(&acc_empty[buf], uint32_t((use - 1) & 1))) {
        atomicExch(&failed, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dacc = tmem + uint32_t(buf * kTmemCols);
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = int(it % kStages);
        if (!mbar_wait(&full[s], uint32_t((it / kStages) & 1)) || failed) {
          atomicExch(&failed, 1);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t da = smem_desc<kSW>(base + pa[q] * kTileA);
          const uint64_t db = smem_desc<kSW>(base + 3 * kTileA + pb[q] * kTileB);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)   // K = 16 per instruction: +32 bytes = +2 in the address field
            mma_bf16(dacc, da + 2 * kk, db + 2 * kk, idesc, (kb | q | kk) != 0);
        }
        if constexpr (PAIR) mma_commit_mc(&empty[s], uint16_t(0x3));
        else mma_commit(&empty[s]);
      }
      mma_commit(&acc_full[buf]);
      if (!ok) break;
    }
  } else if (warp >= 2) {
    // ---- epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (its rows) and
    // half (w-2)/4 of the tile's columns, 32 columns per TMEM load
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const float alpha_f = float(a.alpha);
    int64_t t = 0;
    for (int64_t u = unit0; u < nunits; u += unit_step, ++t) {
      const int buf = int(t & 1);
      if (!mbar_wait(&acc_full[buf], uint32_t((t >> 1) & 1)) || failed) {
        atomicExch(&failed, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int64_t m0, n0;
      bool half_unit;
      unit_of(u, &m0, &n0, &half_unit);
      const int width = half_unit ? kBN / 2 : kBN;
      const int64_t row = m0 + quad * 32 + lane;
      const bool row_ok = row < a.M;
      const uint64_t rbase = row_ok ? a.rowmap[row] : 0;
      for (int c0 = half * (width / 2); c0 < (half + 1) * (width / 2); c0 += 32) {
        float v[32];
        tmem_ld32(tmem + uint32_t(buf * kTmemCols) + (uint32_t(quad * 32) << 16) + uint32_t(c0), v);
        if (!row_ok) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t col0 = n0 + c0 + 16 * h;
          const int ncols = int(a.N - col0 < 16 ? (a.N - col0 > 0 ? a.N - col0 : 0) : 16);
          if (ncols == 0) continue;
          float* f = v + 16 * h;
          // probability check: the 16 values summed in FP32, the chunks in FP64
          float cs = 0.f;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            f[j] *= alpha_f;
            if (j < ncols) cs += f[j];
          }
          sum_d += double(cs);
          const uint64_t c_first = a.colmap[col0];
          store16(a, rbase + c_first, a.contig16 && ncols == 16, f, a.colmap, col0, rbase, ncols);
        }
      }
      // hand the accumulator back to the MMA warp
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // neither CTA leaves while the partner may still signal its barriers
  if constexpr (PAIR) cluster_sync();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols) : "memory");
  }
  if (failed && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
  if (a.partials) finish_total(sum_d, a.partials, a.counter, a.total, red);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  // looked up once per process (thread-safe initialisation)
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return EncodeTiledFn(nullptr);
  }();
  return fn;
}

// 3-D map over BF16 planes [3][rows][Kp], box bk x box_rows x 1, with the
// swizzle of a bk-wide row (128 or 64 bytes).
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t Kp, int bk, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {cuuint64_t(Kp), cuuint64_t(rows), 3};
  const cuuint64_t strides[2] = {cuuint64_t(Kp) * 2, cuuint64_t(rows) * cuuint64_t(Kp) * 2};
  const cuuint32_t box[3] = {cuuint32_t(bk), cuuint32_t(box_rows), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE,
            bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B),
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class Cfg>
cudaError_t launch_cfg(const GemmTcArgs& a, cudaStream_t s) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, a.A, a.Mp, a.Kp, Cfg::BK, kBM) || !make_map(&mb, a.B, a.Np, a.Kp, Cfg::BK, Cfg::BN))
    return cudaErrorInvalidValue;
  const int64_t tiles = (a.Mp / kBM) * (a.Np / Cfg::BN);
  const int64_t grid = tiles < 152 ? tiles : 152;    // persistent: at most one CTA per SM
  gemm_tc_kernel<Cfg, false><<<unsigned(grid), kThreads, Cfg::kSmemBytes, s>>>(ma, mb, a);
  return cudaGetLastError();
}

// Co-resident 2-CTA clusters of the pair kernel (0: none), once per process.
int pair_clusters() {
  static const int n = [] {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(152, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = CfgPair::kSmemBytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, gemm_tc_kernel<CfgPair, true>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      c = 0;
    }
    return c < 76 ? c : 76;
  }();
  return n;
}

cudaError_t launch_pair(const GemmTcArgs& a, int clusters, cudaStream_t s) {
  CUtensorMap ma, mb;
  // B is loaded in halves (BN / 2 rows) by the two CTAs of a pair
  if (!make_map(&ma, a.A, a.Mp, a.Kp, CfgPair::BK, kBM) ||
      !make_map(&mb, a.B, a.Np, a.Kp, CfgPair::BK, CfgPair::BN / 2))
    return cudaErrorInvalidValue;
  const int64_t units = (a.Mp / (2 * kBM)) * (a.Np / CfgPair::BN);
  const int64_t nc = units < clusters ? units : clusters;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(unsigned(2 * nc), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = CfgPair::kSmemBytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gemm_tc_kernel<CfgPair, true>, ma, mb, a);
}

}  // namespace

bool gemm_tc_available() { return encode_fn() != nullptr; }

int gemm_tc_min_rows() { return kBM; }
int gemm_tc_k_align() { return kKAlign; }

cudaError_t gemm_tc_configure() {
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<CfgNarrow, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, CfgNarrow::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<CfgWide, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             CfgWide::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<CfgPair, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             CfgPair::kSmemBytes);
  return e;
}

cudaError_t launch_gemm_tc(const GemmTcArgs& a, cudaStream_t s) {
  // shape contract: Mp, Np multiples of 128 (they are the powers of two M, N
  // >= 128), Kp a multiple of 64; checked here so that no TMA coordinate or
  // TMEM lane can leave the operands
  if (a.Mp % kBM || a.Np % 128 || a.Kp % kKAlign || a.Kp <= 0 || a.M > a.Mp || a.N > a.Np || a.K > a.Kp)
    return cudaErrorInvalidValue;
  // TMA wants 16-byte aligned global operands (the 1024-byte alignment the
  // swizzle needs applies to the shared-memory stages only)
  if ((reinterpret_cast<uintptr_t>(a.A) | reinterpret_cast<uintptr_t>(a.B)) & 15) return cudaErrorInvalidValue;
  // 256-wide tiles when they still fill every SM at least once; in pairs
  // sharing B when the row tiles pair up and the pairs fill the clusters
  if (a.Np % 256 == 0 && (a.Mp / kBM) * (a.Np / 256) >= 152) {
    const int clusters = pair_clusters();
    if (a.Mp % (2 * kBM) == 0 && clusters > 0 && (a.Mp / (2 * kBM)) * (a.Np / 256) >= clusters)
      return launch_pair(a, clusters, s);
    return launch_cfg<CfgWide>(a, s);
  }
  return launch_cfg<CfgNarrow>(a, s);
}

}  // namespace sqc
