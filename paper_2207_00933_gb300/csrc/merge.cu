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

__global__ void __launch_bounds__(256) merge_kernel(const MergeDesc* __restrict__ descs, int n) {
  __shared__ MergeDesc d;
  if (threadIdx.x == 0) {
    int lo = 0;
    for (int i = 1; i < n; ++i)
      if (descs[i].block_begin <= int64_t(blockIdx.x)) lo = i;
    d = descs[lo];
  }
  __syncthreads();
  merge_block(d, int64_t(blockIdx.x) - d.block_begin);
}

}  // namespace

cudaError_t launch_merge_blocks(const MergeDesc* d_descs, int n, int64_t total_blocks, cudaStream_t s) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  merge_kernel<<<unsigned(total_blocks), 256, 0, s>>>(d_descs, n);
  return cudaGetLastError();
}

}  // namespace sqc
