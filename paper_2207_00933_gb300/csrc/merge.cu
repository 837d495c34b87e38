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

}  // namespace

cudaError_t launch_merge_blocks(const MergeDesc* d_descs, int n, int64_t total_blocks, cudaStream_t s) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  // 8 CTAs of 256 threads per SM
  const int64_t grid = total_blocks < 152 * 8 ? total_blocks : 152 * 8;
  merge_kernel<<<unsigned(grid), 256, 0, s>>>(d_descs, n, total_blocks);
  return cudaGetLastError();
}

}  // namespace sqc
