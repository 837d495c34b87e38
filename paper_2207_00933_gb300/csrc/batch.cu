// Batched recursion level: many queries (bins of possibly different
// circuits, uneven active-qubit counts) reconstructed by ONE persistent
// kernel launch.
//
// The host flattens every query's merge blocks and contraction-step tiles
// into one work list ordered by dependency level (all merge blocks first,
// then the steps level by level).  Persistent CTAs take items in list order
// from a global head counter.  Every tensor has a completion counter; an
// item waits (bounded) until the counters of its input tensors reach their
// expected item counts, does its work, then bumps the counter of the tensor
// it wrote.  An item only ever waits for items earlier in the list, which
// were taken by CTAs that are running, so the schedule cannot deadlock.
// The last CTA to leave re-arms the head and the counters, so the same
// launch can be replayed (e.g. from a CUDA graph).  On a wait timeout the
// kernel raises an abort flag that makes every CTA drain quickly and
// records an error code.
#include "device_ops.cuh"

namespace sqc {

namespace {

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Per-query FP64 probability sum over the final step's tiles: each tile
// stores its partial, the last one adds them in tile order into *total.
__device__ __forceinline__ void finish_query_total(double mine, const BatchStep& st, int64_t tile, double* total,
                                                   double* red) {
  __shared__ bool is_last;
  const double bs = block_sum(mine, red);
  if (threadIdx.x == 0) {
    st.partials[tile] = bs;
    __threadfence();
    const unsigned t = atomicAdd(st.counter, 1u);
    is_last = (t == unsigned(st.ntiles - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < st.ntiles; i += blockDim.x) s += static_cast<volatile double*>(st.partials)[i];
  const double tot = block_sum(s, red);
  if (threadIdx.x == 0) {
    *total = tot;
    *st.counter = 0u;
  }
}

template <int BM, int BN, int TM, int TN, bool CH, int BK>
__device__ __forceinline__ double run_tile(const BatchStep& st, int64_t tile, float* smem, void* C) {
  const int64_t tiles_n = (st.a.N + BN - 1) / BN;
  const int tn_shift = __ffsll(tiles_n) - 1;
  const int64_t m0 = (tile >> tn_shift) * BM;
  const int64_t n0 = (tile & (tiles_n - 1)) * BN;
  // operands written by other CTAs of this launch: read from L2, not
  // through the read-only path
  return gemm_tile<BM, BN, TM, TN, CH, BK, kOpThreads, true>(st.a, m0, n0, smem, smem + BK * (BM + 4), C);
}

__global__ void __launch_bounds__(kOpThreads, 2) batch_kernel(BatchLaunch L) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  extern __shared__ __align__(16) float smem[];
  __shared__ MergeDesc md;
  __shared__ BatchItem item;
  __shared__ int64_t my;
  __shared__ double red[kOpThreads / 32];
  __shared__ bool is_last;
  __shared__ int skip;
  for (;;) {
    if (threadIdx.x == 0) {
      my = (*static_cast<volatile int*>(L.abort)) ? L.n_items : int64_t(atomicAdd(reinterpret_cast<unsigned long long*>(L.head), 1ull));
      if (my < L.n_items) item = L.items[my];
    }
    __syncthreads();
    if (my >= L.n_items) break;
    if (threadIdx.x == 0) {
      // wait for the input tensors (bounded; abort on timeout)
      for (int k = 0; k < 2; ++k) {
        const int dep = k ? item.dep1 : item.dep0;
        if (dep < 0) continue;
        uint32_t i = 0;
        uint64_t t0 = 0;
        while (ld_acquire(L.counts + dep) < L.expected[dep]) {
          if (*static_cast<volatile int*>(L.abort)) break;     // another CTA gave up: drain
          if ((++i & 31) == 0) {
            const uint64_t now = global_ns();
            if (t0 == 0) {
              t0 = now;
            } else if (now - t0 > L.wait_ns) {
              atomicExch(L.abort, 1);
              atomicExch(L.err, 1);
              break;
            }
          }
          if (i > 32) __nanosleep(64);
        }
      }
      if (item.type == kItemMerge) md = L.mdescs[item.idx];
      skip = *static_cast<volatile int*>(L.abort);    // one decision for the whole CTA
    }
    __syncthreads();
    if (!skip) {
      if (item.type == kItemMerge) {
        merge_block(md, item.tile);
      } else {
        const BatchStep& st = L.steps[item.idx];
        // a single-query launch names its output and probability sum per
        // run; a batch baked them into its steps
        void* C = st.from_launch ? L.out : st.a.C;
        double* total = st.from_launch ? L.total : st.total;
        double mine;
        switch (st.cfg) {
          case 0: mine = run_tile<32, 32, 2, 2, false, 16>(st, item.tile, smem, C); break;
          case 1: mine = run_tile<64, 64, 4, 4, false, 16>(st, item.tile, smem, C); break;
          case 2: mine = run_tile<128, 64, 8, 4, false, 16>(st, item.tile, smem, C); break;
          case 3: mine = run_tile<32, 32, 2, 2, false, 64>(st, item.tile, smem, C); break;
          case 4: mine = run_tile<64, 64, 4, 4, false, 64>(st, item.tile, smem, C); break;
          case 5: mine = run_tile<32, 32, 2, 2, true, 16>(st, item.tile, smem, C); break;
          default: mine = run_tile<64, 64, 4, 4, true, 16>(st, item.tile, smem, C); break;
        }
        if (st.a.partials && total) finish_query_total(mine, st, item.tile, total, red);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && item.out >= 0) {
      __threadfence();
      atomicAdd(L.counts + item.out, 1u);
    }
  }
  // the last CTA out re-arms the schedule for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(L.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    for (int64_t i = threadIdx.x; i < L.n_slots; i += blockDim.x) L.counts[i] = 0u;
    if (threadIdx.x == 0) {
      *L.head = 0ull;
      *L.done = 0u;
      *L.abort = 0;
    }
  }
}

}  // namespace

int batch_smem_bytes() {
  // largest tile stage among the configurations above (64x64 with BK = 64)
  return int(sizeof(float)) * gemm_tile_smem_floats<64, 64, 64>();
}

cudaError_t batch_configure() {
  return cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem_bytes());
}

cudaError_t launch_batch(const BatchLaunch& L, int grid, cudaStream_t s) {
  if (L.n_items <= 0) return cudaSuccess;
  return launch_k(batch_kernel, dim3(unsigned(grid)), dim3(kOpThreads), size_t(batch_smem_bytes()), s, false, L);
}

// Tile configuration ids of the batch kernel for one step, under a tile
// policy: 0 = by occupancy (the default), 1 = small tiles (32 x 32: the
// most work items, best balance for many uneven queries), 2 = large tiles
// (64 x 64 or 128 x 64 wherever a step has enough of them: fewer operand
// reloads).  Every configuration sums each bin in the same order, so the
// bins do not depend on the policy.
int batch_tile_cfg(int64_t M, int64_t N, int64_t K, bool chunked, int64_t chunk, int64_t* bm, int64_t* bn,
                   int policy) {
  auto tiles = [&](int64_t a, int64_t b) { return ((M + a - 1) / a) * ((N + b - 1) / b); };
  (void)chunk;
  const bool deep = K >= 64;
  if (policy == 1) {
    *bm = 32; *bn = 32;
    return chunked ? 5 : (deep ? 3 : 0);
  }
  if (policy == 2) {
    if (chunked) {
      if (tiles(64, 64) >= 4) { *bm = 64; *bn = 64; return 6; }
      *bm = 32; *bn = 32;
      return 5;
    }
    if (!deep && tiles(128, 64) >= 16) { *bm = 128; *bn = 64; return 2; }
    if (tiles(64, 64) >= 4) { *bm = 64; *bn = 64; return deep ? 4 : 1; }
    *bm = 32; *bn = 32;
    return deep ? 3 : 0;
  }
  if (chunked) {
    if (tiles(64, 64) >= 64) { *bm = 64; *bn = 64; return 6; }
    *bm = 32; *bn = 32;
    return 5;
  }
  if (tiles(128, 64) >= 152 && !deep) { *bm = 128; *bn = 64; return 2; }
  if (tiles(64, 64) >= 64) { *bm = 64; *bn = 64; return deep ? 4 : 1; }
  *bm = 32; *bn = 32;
  return deep ? 3 : 0;
}

}  // namespace sqc
