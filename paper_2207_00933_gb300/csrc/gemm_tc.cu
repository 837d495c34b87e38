// One contraction step (Section 6.1: C = A B^T over the shared cut-edge
// index) on the tcgen05 tensor cores in split-BF16.
//
// Every operand is held as three BF16 planes x = hi + mid + lo (each plane
// the round-to-nearest of what the previous ones left).  The product keeps
// the six terms of order <= 2 -- hi*hi, hi*mid, mid*hi, hi*lo, mid*mid,
// lo*hi -- all accumulated in one FP32 accumulator in tensor memory, which
// gives about FP32 accuracy for the signed I/X/Y/Z sums.
//
// Persistent CTAs (one per SM) walk the output units; 10 warps:
//   warp 0 (one thread): TMA producer -- for each BK-wide block of the
//     shared index it loads the three A planes and three B planes into one
//     of the pipeline stages;
//   warp 1: allocates 2 x BN TMEM columns; one thread issues tcgen05.mma
//     (kind::f16, BF16 x BF16 -> FP32, K = 16 per instruction): 6 plane pairs
//     per 16-wide slice of the shared index, commits each stage back to the
//     producer and each accumulator pass to the epilogue;
//   warps 2-9: epilogue -- wait for a pass, read the accumulator rows with
//     tcgen05.ld (warp w reads TMEM lanes 32*(w%4) .. +31 and half of the
//     columns), scale by alpha, write through rowmap/colmap (vector stores
//     where 16 columns are contiguous; FP32, FP64 or BF16 planes), add the
//     written values into the per-CTA probability sum, and hand the TMEM
//     buffer back.  Two accumulator buffers let the epilogue of one pass
//     run under the MMAs of the next.
//
// Cross-chunk FP64 sum (Section 6.3, the 4^K edge terms for K >= 12): with
// `chunk` > 0 a unit's shared index is summed in passes of `chunk` terms,
// each pass accumulating in FP32 in TMEM; the epilogue adds every pass into
// the FP64 output (the first pass stores, later passes read-add-write; a
// unit's passes all run on one CTA, one after another, and each output
// element is always handled by the same thread, so the additions are
// ordered).  `accumulate` adds the step's result into C instead of
// overwriting it (first-level slices).
//
// Pairs (Cfg::PAIR): clusters of two CTAs compute one 256 x BN unit with
// tcgen05.mma.cta_group::2 (M = 256): each CTA loads its own 128 rows of A
// and its own half of the B rows into its own shared memory by TMA; the
// MMA, issued by the even CTA, reads both halves and leaves each
// CTA's 128 output rows in that CTA's TMEM.  The odd CTA's loads complete on
// the even CTA's stage barrier (the cta_group::2 form of the TMA load), its
// epilogue warps return the accumulator to the even CTA's barrier, and the
// even CTA's commits arrive on the barriers of both.
//
// Tail: when the units leave a last wave at most half full, that wave runs
// as half-width units (N = BN / 2), so that the busiest CTA does half a
// unit less.
//
// Every mbarrier wait is bounded in time; on timeout the CTA (and its pair
// partner) records an error code, waits (bounded) for its own copies in
// flight and frees its TMEM before returning.
#include <cuda.h>

#include "common.cuh"

namespace sqc {

namespace {

constexpr int kBM = 128;
constexpr int kKAlign = 64;        // the shared index is padded to a multiple of this
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, each half of the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr unsigned long long kWaitNs = 2000000000ull;   // default limit of one wait: 2 s

constexpr uint32_t make_idesc(int m, int n) {
  // D = FP32, A = B = BF16, both K-major, M x N
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

// Tile configurations: BN output columns per unit, BK shared-index columns
// per stage (BK BF16 = one swizzle row: 64 -> 128-byte swizzle, 32 ->
// 64-byte swizzle), STAGES pipeline stages.
//   128 x 128, BK 64, 2 stages of 96 KB (narrow steps)
//   128 x 256, BK 32, 3 stages of 72 KB: 25% less operand traffic per flop
//   256 x 256 in 2-CTA pairs, BK 32, 4 stages of 48 KB per CTA
template <int BN_, int BK_, int STAGES_, bool PAIR_>
struct TcCfg {
  static constexpr int BN = BN_, BK = BK_, STAGES = STAGES_;
  static constexpr bool PAIR = PAIR_;
  static constexpr int kRowsB = PAIR ? BN / 2 : BN;   // B rows one CTA holds per plane
  static constexpr int kBoxB = PAIR ? BN / 4 : BN / 2;  // rows per B load (a half-width unit loads one box)
  static constexpr int kTileA = kBM * BK * 2;
  static constexpr int kTileB = kRowsB * BK * 2;
  static constexpr int kStageBytes = 3 * kTileA + 3 * kTileB;
  // guard band after the stages: every operand read of the pair's MMA
  // stays inside this CTA's allocation even for a full-height B tile
  static constexpr int kGuardBytes = PAIR ? 16384 : 0;
  static constexpr int kTmemCols = BN;          // one FP32 accumulator buffer
  static constexpr int kSmemBytes = STAGES * kStageBytes + kGuardBytes + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int kSwizzleBytes = BK * 2;
  static constexpr uint32_t kIdesc = make_idesc(PAIR ? 2 * kBM : kBM, BN);
  static constexpr uint32_t kIdescHalf = make_idesc(PAIR ? 2 * kBM : kBM, BN / 2);
};
using CfgNarrow = TcCfg<128, 64, 2, false>;
using CfgWide = TcCfg<256, 32, 3, false>;
using CfgPair = TcCfg<256, 32, 4, true>;
static_assert(CfgPair::kSmemBytes <= 227 * 1024, "pair stages exceed shared memory");
static_assert(CfgWide::kSmemBytes <= 227 * 1024, "wide stages exceed shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Arrive on a barrier of another CTA of the cluster (release at cluster scope).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}

template <bool CLUSTER>
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if constexpr (CLUSTER) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  } else {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return ok != 0;
}

// Wait for the phase of `parity` to complete, at most limit_ns; gives up
// early when `failed` is set (unless drain: waits for own copies ignore it).
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* failed,
                                          uint64_t limit_ns, bool drain = false) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_test<CLUSTER>(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (!drain && *failed) return false;
      const uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
      __nanosleep(64);
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// The same load by the odd CTA of a pair: the data lands in this CTA's
// shared memory and the completion is counted on the even CTA's barrier
// (`bar` is its shared::cluster address), whose MMAs read both CTAs' stages.
__device__ __forceinline__ void tma_load_3d_peer(void* dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, %3, "
      "%4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
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

template <bool PAIR>
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  if constexpr (PAIR) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// Commit: the barrier at `addr` (shared::cluster; this CTA's or the pair
// partner's) receives one arrival when the MMAs issued so far complete.
template <bool PAIR>
__device__ __forceinline__ void mma_commit(uint32_t addr) {
  if constexpr (PAIR)
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(addr)
                 : "memory");
  else
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(addr)
                 : "memory");
}

// Start loading 32 consecutive accumulator columns of this thread's TMEM
// lane into r; the values may be read only after tmem_wait(r).
__device__ __forceinline__ void tmem_ld32_start(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Wait for every TMEM load of this thread; r is passed through the wait so
// that no read of it can be scheduled before the data has arrived.
__device__ __forceinline__ void tmem_wait(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
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
// 32 bytes from registers to global memory in one 256-bit store (a whole
// sector: a lane's row segment no longer reaches L2 as two half-sector
// writes).  p must be 32-byte aligned.
__device__ __forceinline__ void st_v8(float* p, const float* f) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(f[0]), "f"(f[1]), "f"(f[2]),
               "f"(f[3]), "f"(f[4]), "f"(f[5]), "f"(f[6]), "f"(f[7])
               : "memory");
}
__device__ __forceinline__ void st_v4d(double* p, double x0, double x1, double x2, double x3) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(x0), "d"(x1), "d"(x2), "d"(x3) : "memory");
}

// The output format is a template parameter of the kernel (one
// instantiation per format): only its store path is compiled in, which
// keeps the epilogue's code small in the instruction cache.
template <int KIND>
__device__ __forceinline__ void store16(const GemmTcArgs& a, uint64_t off, bool contig, const float* f,
                                        const uint64_t* colmap, int64_t col0, uint64_t rbase, int ncols) {
  if (contig && ncols == 16) {
    if constexpr (KIND == OUT_F32) {
      float* c = static_cast<float*>(a.C) + off;
      if ((reinterpret_cast<uintptr_t>(c) & 31) == 0) {
        st_v8(c, f);
        st_v8(c + 8, f + 8);
        return;
      }
      float4* p = reinterpret_cast<float4*>(c);
#pragma unroll
      for (int q = 0; q < 4; ++q) p[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
      return;
    }
    if constexpr (KIND == OUT_F64) {
      double* c = static_cast<double*>(a.C) + off;
      if ((reinterpret_cast<uintptr_t>(c) & 31) == 0) {
        // the hardware conversion here (exact, as any FP32 -> FP64 one):
        // 16 per thread and group cost the FP64 pipe less than the bit
        // moves' instructions cost issue slots (measured 8% faster on the
        // 1024 x 4096 x 64 FP64-output step)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          st_v4d(c + 4 * q, double(f[4 * q]), double(f[4 * q + 1]), double(f[4 * q + 2]), double(f[4 * q + 3]));
        return;
      }
      double2* p = reinterpret_cast<double2*>(c);
#pragma unroll
      for (int q = 0; q < 8; ++q) p[q] = make_double2(f2d(f[2 * q]), f2d(f[2 * q + 1]));
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j < ncols) store_out_f(a.C, KIND, a.plane_stride, rbase + colmap[col0 + j], f[j]);
}

// Add 16 consecutive columns of one output row into C (FP32 or FP64
// output), or store them (load_old false; FP64 only: the first pass of a
// chunked unit).  Returns the sum of the values now in C.
template <int KIND>
__device__ __forceinline__ double add16(const GemmTcArgs& a, uint64_t off, bool contig, const float* f,
                                        const uint64_t* colmap, int64_t col0, uint64_t rbase, int ncols,
                                        bool load_old) {
  double s = 0.0;
  if constexpr (KIND == OUT_BF16X3) {
    return s;                                   // never reached: BF16 planes are written, not added
  } else if constexpr (KIND == OUT_F64) {
    double* C = static_cast<double*>(a.C);
    if (contig && ncols == 16) {
      double2* p = reinterpret_cast<double2*>(C + off);
      double2 o[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q] = make_double2(f2d(f[2 * q]), f2d(f[2 * q + 1]));
      if (load_old) {
        double2 old[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) old[q] = p[q];          // all loads in flight together
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          o[q].x += old[q].x;
          o[q].y += old[q].y;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        p[q] = o[q];
        s += o[q].x + o[q].y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < ncols) {
          double* d = C + rbase + colmap[col0 + j];
          const double v = load_old ? *d + f2d(f[j]) : f2d(f[j]);
          *d = v;
          s += v;
        }
    }
  } else {
    float* C = static_cast<float*>(a.C);
    float sf = 0.f;
    if (contig && ncols == 16) {
      float4* p = reinterpret_cast<float4*>(C + off);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float4 o = load_old ? p[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        o.x += f[4 * q]; o.y += f[4 * q + 1]; o.z += f[4 * q + 2]; o.w += f[4 * q + 3];
        p[q] = o;
        sf += (o.x + o.y) + (o.z + o.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < ncols) {
          float* d = C + rbase + colmap[col0 + j];
          const float v = (load_old ? *d : 0.f) + f[j];
          *d = v;
          sf += v;
        }
    }
    s = double(sf);
  }
  return s;
}

// Persistent: CTA (or pair) b takes units b, b + grid, ...  The
// accumulator is double-buffered in TMEM (2 x BN columns).
template <class Cfg, int KIND>
__global__ void __launch_bounds__(kThreads, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmTcArgs a) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  constexpr bool PAIR = Cfg::PAIR;
  constexpr int kBN = Cfg::BN, kBK = Cfg::BK, kStages = Cfg::STAGES;
  constexpr int kTileA = Cfg::kTileA, kTileB = Cfg::kTileB, kStageBytes = Cfg::kStageBytes;
  constexpr int kTmemCols = Cfg::kTmemCols, kSW = Cfg::kSwizzleBytes;
  constexpr int kSlices = kBK / 16;          // 16-wide shared-index slices per stage
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + Cfg::kGuardBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;      // [2]: MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;        // [2]: epilogue -> MMA
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ double red[kThreads / 32];
  __shared__ int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t rank = 0;
  if constexpr (PAIR) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  const bool leader = rank == 0;
  const uint64_t wlim = a.wait_ns ? a.wait_ns : kWaitNs;
  const int64_t tiles_n = a.Np / kBN;
  const int tn_shift = __ffsll(tiles_n) - 1;
  const int64_t nwide = (a.Mp / (PAIR ? 2 * kBM : kBM)) * tiles_n;
  const int nk = int(a.Kp / kBK);
  const int64_t unit0 = PAIR ? int64_t(blockIdx.x >> 1) : int64_t(blockIdx.x);
  const int64_t unit_step = PAIR ? int64_t(gridDim.x >> 1) : int64_t(gridDim.x);
  const int64_t tail = nwide % unit_step;
  const bool split = tail > 0 && 2 * tail <= unit_step;
  const int64_t wide_end = split ? nwide - tail : nwide;        // units [wide_end, nunits) are half-width
  const int64_t nunits = split ? wide_end + 2 * tail : nwide;
  // accumulator passes per unit: the shared index in chunks of `chunk`
  // terms (16-wide slices), each summed in FP32 and added in FP64
  const int nsl = int(a.Kp / 16);
  const int sl_chunk = (a.chunk > 0 && a.chunk / 16 < nsl) ? int(a.chunk / 16) : nsl;
  const int npass = nsl / sl_chunk;
  // unit u -> (this CTA's first row, the unit's first column, half width)
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
  // record a failure here and, in a pair, in the partner
  auto set_failed = [&]() {
    atomicExch(&failed, 1);
    if constexpr (PAIR)
      asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr(&failed, rank ^ 1u)), "r"(1) : "memory");
  };

  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < kStages; ++s) {
      // pair: only the even CTA's stage barriers count (both CTAs' bytes)
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], PAIR ? 2 * kEpiWarps : kEpiWarps);   // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(2 * kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(2 * kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // a pair's barriers receive the partner's arrivals: both are initialised
  // (and both TMEM allocations done) before either CTA starts
  if constexpr (PAIR) cluster_sync();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  double sum_d = 0.0;
  float sum_hi = 0.f, sum_lo = 0.f;       // plain FP32 groups, as an FP32 pair

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: one continuous ring of stages across all units
    int64_t it = 0, issued = 0;
    bool ok = true;
    for (int64_t u = unit0; u < nunits && ok; u += unit_step) {
      int64_t um0, un0;
      bool half;
      unit_of(u, &um0, &un0, &half);
      const int m0 = int(um0), n0 = int(un0);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = int(it % kStages);
        const int64_t use = it / kStages;
        if (use > 0 && !mbar_wait<PAIR>(&empty[s], uint32_t((use - 1) & 1), &failed, wlim)) {
          set_failed();
          ok = false;
          break;
        }
        uint8_t* st = smem + s * kStageBytes;
        uint8_t* stb = st + 3 * kTileA;
        if constexpr (PAIR) {
          // this CTA's A rows and B rows (half of the unit's columns: two
          // boxes of BN / 4 rows, one for a half-width unit); the even CTA's
          // barrier expects both CTAs' bytes, the odd CTA's loads count on it
          const uint32_t bytes = 3 * kTileA + 3 * (half ? kTileB / 2 : kTileB);
          const uint32_t lead_full = cluster_addr(&full[s], 0);
          auto load = [&](void* dst, const CUtensorMap* map, int x, int y, int z) {
            if (leader) tma_load_3d(dst, map, x, y, z, &full[s]);
            else tma_load_3d_peer(dst, map, x, y, z, lead_full);
          };
          if (leader) mbar_expect_tx(&full[s], 2 * bytes);
          for (int p = 0; p < 3; ++p) load(st + p * kTileA, &tmA, kb * kBK, m0, p);
          if (half) {
            for (int p = 0; p < 3; ++p) load(stb + p * kTileB, &tmB, kb * kBK, n0 + int(rank) * (kBN / 4), p);
          } else {
            for (int p = 0; p < 3; ++p)
              for (int h = 0; h < 2; ++h)
                load(stb + p * kTileB + h * (kTileB / 2), &tmB, kb * kBK, n0 + int(rank) * (kBN / 2) + h * (kBN / 4),
                     p);
          }
        } else {
          // the unit's B rows: two boxes of BN / 2 rows (half width: one)
          mbar_expect_tx(&full[s], 3 * kTileA + 3 * (half ? kTileB / 2 : kTileB));
          for (int p = 0; p < 3; ++p) tma_load_3d(st + p * kTileA, &tmA, kb * kBK, m0, p, &full[s]);
          for (int p = 0; p < 3; ++p)
            for (int h = 0; h < (half ? 1 : 2); ++h)
              tma_load_3d(stb + p * kTileB + h * (kTileB / 2), &tmB, kb * kBK, n0 + h * (kBN / 2), p, &full[s]);
        }
        issued = it + 1;
      }
    }
    // drain: every copy this CTA issued has landed (a pair's odd CTA: the
    // commit that frees a stage follows the even CTA's wait for both CTAs'
    // bytes), and (normal end) every commit that frees a stage has arrived,
    // before the CTA exits
    const int64_t j0 = issued > kStages ? issued - kStages : 0;
    if (leader)
      for (int64_t j = j0; j < issued; ++j)
        if (!mbar_wait<PAIR>(&full[j % kStages], uint32_t((j / kStages) & 1), &failed, wlim, true)) set_failed();
    if (!failed)
      for (int64_t j = j0; j < issued; ++j)
        if (!mbar_wait<PAIR>(&empty[j % kStages], uint32_t((j / kStages) & 1), &failed, wlim)) set_failed();
  } else if (warp == 1 && lane == 0 && leader) {
    // ---- MMA issuer (the pair's even CTA)
    constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
    constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
    const uint32_t peer = rank ^ 1u;
    int64_t it = 0, t = 0;
    bool ok = true;
    for (int64_t u = unit0; u < nunits && ok; u += unit_step) {
      const uint32_t idesc = u >= wide_end ? Cfg::kIdescHalf : Cfg::kIdesc;
      for (int sl = 0; sl < nsl; ++sl) {
        const int kk = sl % kSlices;
        const int cs = sl % sl_chunk;
        if (cs == 0) {
          const int64_t use = t >> 1;
          if (use > 0 && !mbar_wait<PAIR>(&acc_empty[t & 1], uint32_t((use - 1) & 1), &failed, wlim)) {
            set_failed();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const int s = int(it % kStages);
        if (kk == 0) {
          if (!mbar_wait<PAIR>(&full[s], uint32_t((it / kStages) & 1), &failed, wlim)) {
            set_failed();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const uint32_t base = smem_u32(smem + s * kStageBytes);
        const uint32_t dacc = tmem + uint32_t((t & 1) * kTmemCols);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t da = smem_desc<kSW>(base + pa[q] * kTileA);
          const uint64_t db = smem_desc<kSW>(base + 3 * kTileA + pb[q] * kTileB);
          // K = 16 per instruction: +32 bytes = +2 in the address field
          mma_bf16<PAIR>(dacc, da + 2 * kk, db + 2 * kk, idesc, (cs | q) != 0);
        }
        if (kk == kSlices - 1) {
          mma_commit<PAIR>(smem_u32(&empty[s]));
          if constexpr (PAIR) mma_commit<PAIR>(cluster_addr(&empty[s], peer));
          ++it;
        }
        if (cs == sl_chunk - 1) {
          mma_commit<PAIR>(smem_u32(&acc_full[t & 1]));
          if constexpr (PAIR) mma_commit<PAIR>(cluster_addr(&acc_full[t & 1], peer));
          ++t;
        }
      }
    }
    // normal end: the epilogues (a pair: both CTAs') have released the last
    // accumulator buffers, so no arrival is still on its way here
    if (ok && !failed)
      for (int64_t j = t > 2 ? t - 2 : 0; j < t; ++j)
        if (!mbar_wait<PAIR>(&acc_empty[j & 1], uint32_t((j >> 1) & 1), &failed, wlim)) set_failed();
  } else if (warp >= 2) {
    // ---- epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (its rows) and
    // half (w-2)/4 of the unit's columns, 32 columns per TMEM load; the next
    // 32 columns load while the current ones are stored
    constexpr int kChunks = kBN / 64;          // 32-column chunks in a warp's half of a full-width unit
    const int quad = warp & 3;
    const int hc = (warp - 2) >> 2;
    const float alpha_f = pow2_to_float(a.alpha);   // a power of two
    const bool plain = npass == 1 && !a.accumulate;
    int64_t t = 0;
    bool ok = true;
    for (int64_t u = unit0; u < nunits && ok; u += unit_step) {
      int64_t m0, n0;
      bool half_unit;
      unit_of(u, &m0, &n0, &half_unit);
      const int cw = (half_unit ? kBN / 2 : kBN) / 2;      // this warp's columns
      const int nchunk = cw / 32;
      const int64_t c_lo = n0 + int64_t(hc) * cw;
      const int64_t row = m0 + quad * 32 + lane;
      const bool row_ok = row < a.M;
      // the row's and the columns' offsets, loaded together before the
      // accumulator is ready (one memory latency per unit, not one per group)
      const uint64_t rbase = row_ok ? a.rowmap[row] : 0;
      uint64_t cb[2 * kChunks];
#pragma unroll
      for (int g = 0; g < 2 * kChunks; ++g) {
        const int64_t col0 = c_lo + 16 * g;
        cb[g] = (g < 2 * nchunk && col0 < a.N) ? a.colmap[col0] : 0;
      }
      for (int pass = 0; pass < npass; ++pass, ++t) {
        const int buf = int(t & 1);
        if (!mbar_wait<PAIR>(&acc_full[buf], uint32_t((t >> 1) & 1), &failed, wlim)) {
          set_failed();
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool load_old = pass > 0 || a.accumulate;
        const bool last_pass = pass == npass - 1;
        const uint32_t tbase = tmem + uint32_t(buf * kTmemCols) + (uint32_t(quad * 32) << 16) +
                               uint32_t(hc * cw);
        uint32_t r[2][32];
        tmem_ld32_start(tbase, r[0]);
        tmem_wait(r[0]);
#pragma unroll
        for (int i = 0; i < kChunks; ++i) {
          if (i >= nchunk) break;
          uint32_t* cur = r[i & 1];
          if (i + 1 < nchunk) tmem_ld32_start(tbase + uint32_t(32 * (i + 1)), r[(i + 1) & 1]);
          if (row_ok) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int64_t col0 = c_lo + 32 * i + 16 * h;
              const int ncols = int(a.N - col0 < 16 ? (a.N - col0 > 0 ? a.N - col0 : 0) : 16);
              if (ncols == 0) continue;
              float f[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) f[j] = __uint_as_float(cur[16 * h + j]) * alpha_f;   // exact: 2^-K
              const uint64_t c_first = cb[2 * i + h];
              const bool contig = a.contig16 && ncols == 16;
              if (plain) {
                // probability check: the 16 values summed in FP32, the groups
                // added into an FP32 pair (no FP64 instruction per group)
                float cs = 0.f;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  if (j < ncols) cs += f[j];
                two_sum_add(sum_hi, sum_lo, cs);
                store16<KIND>(a, rbase + c_first, contig, f, a.colmap, col0, rbase, ncols);
              } else {
                const double sv = add16<KIND>(a, rbase + c_first, contig, f, a.colmap, col0, rbase, ncols, load_old);
                if (last_pass) sum_d += sv;
              }
            }
          }
          if (i + 1 < nchunk) tmem_wait(r[(i + 1) & 1]);
        }
        // hand the accumulator back to the MMA thread
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          if (PAIR && !leader) mbar_arrive_cluster(cluster_addr(&acc_empty[buf], 0));
          else mbar_arrive_local(&acc_empty[buf]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // neither CTA of a pair leaves (or frees TMEM) while the partner may
  // still use it or signal its barriers
  if constexpr (PAIR) cluster_sync();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols)
                   : "memory");
  }
  if (failed && threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
  if (a.partials) finish_total(sum_d + (double(sum_hi) + double(sum_lo)), a.partials, a.counter, a.total, red);
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
  if (!make_map(&ma, a.A, a.Mp, a.Kp, Cfg::BK, kBM) || !make_map(&mb, a.B, a.Np, a.Kp, Cfg::BK, Cfg::kBoxB))
    return cudaErrorInvalidValue;
  const int64_t tiles = (a.Mp / kBM) * (a.Np / Cfg::BN);
  const int64_t grid = tiles < 152 ? tiles : 152;    // persistent: at most one CTA per SM
  auto go = [&](auto kernel) {
    return launch_k(kernel, dim3(unsigned(grid)), dim3(kThreads), size_t(Cfg::kSmemBytes), s, false, ma, mb, a);
  };
  if (a.kind == OUT_F32) return go(gemm_tc_kernel<Cfg, OUT_F32>);
  if (a.kind == OUT_F64) return go(gemm_tc_kernel<Cfg, OUT_F64>);
  return go(gemm_tc_kernel<Cfg, OUT_BF16X3>);
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
    if (cudaOccupancyMaxActiveClusters(&c, gemm_tc_kernel<CfgPair, OUT_F32>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      c = 0;
    }
    return c < 76 ? c : 76;
  }();
  return n;
}

cudaError_t launch_pair(const GemmTcArgs& a, int clusters, cudaStream_t s) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, a.A, a.Mp, a.Kp, CfgPair::BK, kBM) ||
      !make_map(&mb, a.B, a.Np, a.Kp, CfgPair::BK, CfgPair::kBoxB))
    return cudaErrorInvalidValue;
  const int64_t units = (a.Mp / (2 * kBM)) * (a.Np / CfgPair::BN);
  const int64_t nc = units < clusters ? units : clusters;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(unsigned(2 * nc), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = CfgPair::kSmemBytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_flag() ? 2 : 1;
  auto go = [&](auto kernel) {
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, ma, mb, a);
    if (e != cudaSuccess && cfg.numAttrs == 2) {
      cudaGetLastError();
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, kernel, ma, mb, a);
    }
    return e;
  };
  if (a.kind == OUT_F32) return go(gemm_tc_kernel<CfgPair, OUT_F32>);
  if (a.kind == OUT_F64) return go(gemm_tc_kernel<CfgPair, OUT_F64>);
  return go(gemm_tc_kernel<CfgPair, OUT_BF16X3>);
}

}  // namespace

bool gemm_tc_available() { return encode_fn() != nullptr; }

int gemm_tc_min_rows() { return kBM; }
int gemm_tc_k_align() { return kKAlign; }

namespace {
template <class Cfg>
cudaError_t configure_cfg() {
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<Cfg, OUT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Cfg::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<Cfg, OUT_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gemm_tc_kernel<Cfg, OUT_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Cfg::kSmemBytes);
  return e;
}
}  // namespace

cudaError_t gemm_tc_configure() {
  cudaError_t e = configure_cfg<CfgNarrow>();
  if (e == cudaSuccess) e = configure_cfg<CfgWide>();
  if (e == cudaSuccess) e = configure_cfg<CfgPair>();
  return e;
}

cudaError_t launch_gemm_tc(const GemmTcArgs& a, cudaStream_t s) {
  // shape contract: Mp, Np multiples of 128 (they are the powers of two M, N
  // >= 128), Kp a multiple of 64; checked here so that no TMA coordinate or
  // TMEM lane can leave the operands
  if (a.Mp % kBM || a.Np % 128 || a.Kp % kKAlign || a.Kp <= 0 || a.M > a.Mp || a.N > a.Np || a.K > a.Kp)
    return cudaErrorInvalidValue;
  // chunked passes: a power of two >= 16 terms, FP64 output only
  if (a.chunk < 0 || (a.chunk > 0 && (a.chunk < 16 || (a.chunk & (a.chunk - 1)) || a.kind != OUT_F64)))
    return cudaErrorInvalidValue;
  if (a.accumulate && a.kind != OUT_F32 && a.kind != OUT_F64) return cudaErrorInvalidValue;
  // TMA wants 16-byte aligned global operands (the 1024-byte alignment the
  // swizzle needs applies to the shared-memory stages only)
  if ((reinterpret_cast<uintptr_t>(a.A) | reinterpret_cast<uintptr_t>(a.B)) & 15) return cudaErrorInvalidValue;
  // 256-wide units when they still fill every SM at least once; in 2-SM
  // pairs when allowed, the row tiles pair up and the pairs fill the clusters
  if (a.Np % 256 == 0 && (a.Mp / kBM) * (a.Np / 256) >= 152) {
    const int clusters = a.pairs ? pair_clusters() : 0;
    if (a.Mp % (2 * kBM) == 0 && clusters > 0 && (a.Mp / (2 * kBM)) * (a.Np / 256) >= clusters)
      return launch_pair(a, clusters, s);
    return launch_cfg<CfgWide>(a, s);
  }
  return launch_cfg<CfgNarrow>(a, s);
}

}  // namespace sqc
