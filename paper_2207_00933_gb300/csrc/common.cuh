// Device helpers shared by the library's kernels.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "internal.h"
#include "launch.cuh"

namespace sqc {

// Exact widening of an FP32 value to FP64 by moving its bits (IEEE 754
// binary32 -> binary64: same sign, exponent rebiased from 127 to 1023, the
// 23 fraction bits at the top of the 52-bit fraction; subnormals
// normalised; infinities and NaNs keep their payload).  Integer operations
// only: the FP64 pipe of this GPU is narrow, and an FP64 output would
// otherwise spend it on one conversion per element.
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t e = (u >> 23) & 0xffu;
  const uint32_t m = u & 0x7fffffu;
  uint32_t hi, lo;
  if (e - 1u < 0xfeu) {                      // normal: 1 <= e <= 254
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (e == 0xffu) {                   // infinity or NaN
    hi = sign | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else if (m == 0u) {                      // signed zero
    hi = sign;
    lo = 0u;
  } else {                                   // subnormal: m 2^-149, leading one at bit p
    const int p = 31 - __clz(m);
    const uint64_t f52 = uint64_t(m ^ (1u << p)) << (52 - p);
    hi = sign | (uint32_t(p + 874) << 20) | uint32_t(f52 >> 32);
    lo = uint32_t(f52);
  }
  return __hiloint2double(int(hi), int(lo));
}

// FP32 value of a power of two held in FP64 (2^e with -126 <= e <= 127, as
// every scale of the method is: 2^-K or 1) by moving its exponent field:
// exact, integer operations only (a conversion would take the narrow FP64
// pipe once per thread).
__device__ __forceinline__ float pow2_to_float(double d) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  const int e = int((u >> 52) & 0x7ffu) - 1023;
  return __uint_as_float(unsigned(u >> 63) << 31 | unsigned(e + 127) << 23);
}

// s_hi + s_lo += v with the rounding error of the high part kept (Knuth's
// TwoSum: t + e = s_hi + v exactly).  Sums of FP32 values kept as such a
// pair and converted to FP64 once cost no FP64 instruction per value (the
// FP64 pipe of this GPU is narrow).
__device__ __forceinline__ void two_sum_add(float& s_hi, float& s_lo, float v) {
  const float t = s_hi + v;
  const float bp = t - s_hi;
  const float ap = t - bp;
  s_lo += (s_hi - ap) + (v - bp);
  s_hi = t;
}

// Write one result element in the destination's number format: FP32, FP64,
// or three BF16 planes hi + mid + lo (each the round-to-nearest of what the
// previous planes left), the operand format of the split-BF16 steps.
__device__ __forceinline__ void store_out(void* dst, int kind, int64_t plane_stride, uint64_t off, double v) {
  if (kind == OUT_F32) {
    static_cast<float*>(dst)[off] = float(v);
  } else if (kind == OUT_F64) {
    static_cast<double*>(dst)[off] = v;
  } else {
    const float f = float(v);
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(dst);
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const float r1 = f - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    p[off] = hi;
    p[off + plane_stride] = mid;
    p[off + 2 * plane_stride] = lo;
  }
}

// FP32 result: FP64 conversion only when the destination is FP64 (the FP64
// pipe is narrow on this GPU).
__device__ __forceinline__ void store_out_f(void* dst, int kind, int64_t plane_stride, uint64_t off, float f) {
  if (kind == OUT_F32) {
    static_cast<float*>(dst)[off] = f;
  } else if (kind == OUT_F64) {
    static_cast<double*>(dst)[off] = f2d(f);
  } else {
    __nv_bfloat16* p = static_cast<__nv_bfloat16*>(dst);
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const float r1 = f - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    p[off] = hi;
    p[off + plane_stride] = mid;
    p[off + 2 * plane_stride] = lo;
  }
}

// Scatter the low bits of src to the set bits of mask (bit deposit).
__device__ __forceinline__ uint32_t deposit(uint32_t src, uint32_t mask) {
  uint32_t r = 0;
  for (uint32_t bit = 1; mask; bit <<= 1) {
    const uint32_t low = mask & (0u - mask);
    if (src & bit) r |= low;
    mask &= mask - 1;
  }
  return r;
}

// Block-wide FP64 sum in a fixed order; the result is valid in thread 0.
// Every thread of the block must call it.  red: blockDim/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < int(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// Each CTA stores its partial sum; the CTA that finishes last adds all
// partials in CTA order (so the total does not depend on scheduling),
// writes *total and re-arms the counter for the next launch.
__device__ __forceinline__ void finish_total(double mine, double* partials, unsigned* counter, double* total,
                                             double* red) {
  __shared__ bool is_last;
  const double bs = block_sum(mine, red);
  const unsigned nblocks = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    partials[bid] = bs;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    is_last = (t == nblocks - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s = 0.0;
  for (unsigned i = threadIdx.x; i < nblocks; i += blockDim.x) s += static_cast<volatile double*>(partials)[i];
  const double tot = block_sum(s, red);
  if (threadIdx.x == 0) {
    *total = tot;
    *counter = 0u;
  }
}

}  // namespace sqc
