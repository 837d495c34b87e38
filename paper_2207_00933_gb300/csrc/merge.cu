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
#include "common.cuh"

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
  const int lanes = d.lanes;                       // power of two
  const int lshift = __ffs(lanes) - 1;
  const int64_t o = ((int64_t(blockIdx.x) - d.block_begin) << (8 - lshift)) + (threadIdx.x >> lshift);
  const int lane = threadIdx.x & (lanes - 1);
  const int64_t total = d.rows << d.a;
  const bool valid = o < total;
  float acc = 0.f;
  if (valid) {
    const int64_t e = o >> d.a;
    const uint32_t b = uint32_t(o & ((int64_t(1) << d.a) - 1));
    const float* row = d.A + (e << d.n);
    const uint32_t run = 1u << d.m;
    if (d.fast) {
      const float* src = row + (d.zoom_val | (b << d.m));
      if (run >= 4u * lanes) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        for (uint32_t r = lane; r < run / 4; r += lanes) {
          const float4 q = __ldg(s4 + r);
          acc += (q.x + q.y) + (q.z + q.w);
        }
      } else {
        for (uint32_t r = lane; r < run; r += lanes) acc += __ldg(src + r);
      }
    } else {
      const uint32_t xb = deposit(b, d.act_mask) | d.zoom_val;
      for (uint32_t r = lane; r < run; r += lanes) acc += __ldg(row + (xb | deposit(r, d.mer_mask)));
    }
  }
  for (int off = lanes >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (valid && lane == 0) {
    const int64_t e = o >> d.a;
    const uint32_t b = uint32_t(o & ((int64_t(1) << d.a) - 1));
    store_out_f(d.dst, d.kind, d.plane_stride, d.rowmap[e] + d.colmap[b], acc * float(d.alpha));
  }
}

}  // namespace

cudaError_t launch_merge_blocks(const MergeDesc* d_descs, int n, int64_t total_blocks, cudaStream_t s) {
  if (n <= 0 || total_blocks <= 0) return cudaSuccess;
  merge_kernel<<<unsigned(total_blocks), 256, 0, s>>>(d_descs, n);
  return cudaGetLastError();
}

}  // namespace sqc
