// States merging (Section 4, Algorithm 2): for every subcircuit,
//
//   T_i[e][b] = sum_{x : zoom bits of x fixed, active bits of x = b} A_i[e][x]
//
// One launch covers all subcircuits of a query (a descriptor per
// subcircuit, a contiguous CTA range per descriptor).  It is an HBM-bound
// streaming reduction: with the recursion's roles the merged data qubits are
// the low bits of the bit-reversed storage index, so each bin is a
// contiguous run read with 128-bit loads, `lanes` threads per bin and a
// shuffle tree.  Other role patterns take the generic bit-deposit path.
// The result goes straight into the layout the first contraction step reads
// (rowmap/colmap), in FP32, FP64 or as three BF16 planes.
#include "device_ops.cuh"

namespace sqc {

namespace {

// Persistent: CTAs walk the blocks of all descriptors in order; a CTA
// reads a descriptor (and where the next one starts) only when it crosses
// into it.
__global__ void __launch_bounds__(256) merge_kernel(const MergeDesc* __restrict__ descs, int n,
                                                    int64_t total_blocks) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  __shared__ MergeDesc d;
  __shared__ int cur;
  __shared__ int64_t next_begin;
  if (threadIdx.x == 0) {
    cur = -1;
    next_begin = 0;
  }
  __syncthreads();
  for (int64_t blk = blockIdx.x; blk < total_blocks; blk += gridDim.x) {
    if (threadIdx.x == 0 && blk >= next_begin) {
      int i = cur < 0 ? 0 : cur;
      while (i + 1 < n && descs[i + 1].block_begin <= blk) ++i;
      d = descs[i];
      cur = i;
      next_begin = i + 1 < n ? descs[i + 1].block_begin : total_blocks;
    }
    __syncthreads();
    merge_block(d, blk - d.block_begin);
    __syncthreads();
  }
}

// Levels s+1 .. s+c of the merge pyramid from level s: a CTA takes chunks
// of 2^c consecutive values of one row, halves them c times in shared
// memory (pairwise sums) and writes every level's share.
__global__ void __launch_bounds__(256) pyramid_kernel(const float* __restrict__ src, float* pyr, int64_t V, int n,
                                                      int s, int c) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  __shared__ float buf[1 << kPyramidLevelsPerPass];
  const int C = 1 << c;
  const int row_shift = n - s - c;                   // chunks per row = 2^row_shift
  const int64_t total = V << row_shift;
  for (int64_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int64_t e = b >> row_shift;
    const int64_t ch = b & ((int64_t(1) << row_shift) - 1);
    const float* in = src + (e << (n - s)) + (ch << c);
    for (int i = threadIdx.x; i < C; i += blockDim.x) buf[i] = in[i];
    __syncthreads();
    for (int l = 1; l <= c; ++l) {
      const int half = C >> l;
      const int m = s + l;
      float* out = pyr + V * ((int64_t(1) << n) - (int64_t(1) << (n - m + 1))) + (e << (n - m)) + (ch << (c - l));
      float t[(1 << kPyramidLevelsPerPass) / 2 / 256];
#pragma unroll
      for (int k = 0; k < int(sizeof(t) / sizeof(float)); ++k) {
        const int i = int(threadIdx.x) + k * 256;
        t[k] = i < half ? buf[2 * i] + buf[2 * i + 1] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < int(sizeof(t) / sizeof(float)); ++k) {
        const int i = int(threadIdx.x) + k * 256;
        if (i < half) {
          buf[i] = t[k];
          out[i] = t[k];
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace

cudaError_t launch_pyramid(const float* A, float* pyr, int64_t V, int n, cudaStream_t s) {
  for (int lev = 0; lev < n;) {
    const int c = n - lev < kPyramidLevelsPerPass ? n - lev : kPyramidLevelsPerPass;
    const float* src = lev == 0 ? A : pyr + V * ((int64_t(1) << n) - (int64_t(1) << (n - lev + 1)));
    const int64_t total = V << (n - lev - c);
    const int64_t grid = total < 152 * 8 ? total : 152 * 8;
    cudaError_t e = launch_k(pyramid_kernel, dim3(unsigned(grid)), dim3(256), 0, s, false, src, pyr, V, n, lev, c);
    if (e != cudaSuccess) return e;
    lev += c;
  }
  return cudaSuccess;
}

cudaError_t launch_merge_blocks(const MergeDesc* d_descs, int n, int64_t total_blocks, cudaStream_t s) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  // 8 CTAs of 256 threads per SM
  const int64_t grid = total_blocks < 152 * 8 ? total_blocks : 152 * 8;
  return launch_k(merge_kernel, dim3(unsigned(grid)), dim3(256), 0, s, false, d_descs, n, total_blocks);
}

}  // namespace sqc
