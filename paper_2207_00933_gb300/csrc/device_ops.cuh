// Device-side bodies shared by the per-step kernels and the persistent
// batched kernel: one merge CTA-block and one SIMT contraction tile.
#pragma once
#include "common.cuh"

namespace sqc {

constexpr int kOpThreads = 256;

// One CTA-block of the merge of descriptor d (Section 4, Algorithm 2):
// blk is the block index relative to the descriptor's first block.
__device__ __forceinline__ void merge_block(const MergeDesc& d, int64_t blk) {
  const int lanes = d.lanes;                       // power of two
  const int lshift = __ffs(lanes) - 1;
  const int64_t o = (blk << (8 - lshift)) + (threadIdx.x >> lshift);
  const int lane = threadIdx.x & (lanes - 1);
  const int64_t total = d.rows << d.a;
  const bool valid = o < total;
  float acc = 0.f;
  if (valid) {
    const int64_t e = o >> d.a;
    const uint32_t b = uint32_t(o & ((int64_t(1) << d.a) - 1));
    const int64_t er = d.rowsel ? int64_t(d.rowsel[e]) + d.row_add : e;
    const float* row = d.A + (er << d.n);
    const uint32_t run = 1u << d.m;
    if (d.fast) {
      const float* src = row + (d.zoom_val | (b << d.m));
      if (run >= 4u * lanes) {
        // four independent 16-byte loads in flight per lane and round
        const float4* s4 = reinterpret_cast<const float4*>(src);
        const uint32_t nv = run / 4;
        uint32_t r = lane;
        for (; r + 3u * lanes < nv; r += 4u * lanes) {
          const float4 q0 = __ldg(s4 + r), q1 = __ldg(s4 + r + lanes);
          const float4 q2 = __ldg(s4 + r + 2u * lanes), q3 = __ldg(s4 + r + 3u * lanes);
          acc += (((q0.x + q0.y) + (q0.z + q0.w)) + ((q1.x + q1.y) + (q1.z + q1.w))) +
                 (((q2.x + q2.y) + (q2.z + q2.w)) + ((q3.x + q3.y) + (q3.z + q3.w)));
        }
        for (; r < nv; r += lanes) {
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
    store_out_f(d.dst, d.kind, d.plane_stride, d.rowmap[e] + d.colmap[b], acc * pow2_to_float(d.alpha));
  }
}

// Shared memory (floats) one SIMT tile needs for its A and B stages.
template <int BM, int BN, int kBK>
constexpr int gemm_tile_smem_floats() {
  return kBK * (BM + 4) + kBK * (BN + 4);
}

// Operand load: through the read-only path, or from L2 only (CG) for
// operands that other CTAs of the same launch wrote.
template <bool CG>
__device__ __forceinline__ float ld_operand(const float* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

// One BM x BN tile (origin m0, n0) of C = A B^T (Section 6.1) on NT threads
// (256 unless a launch gives the whole CTA to one tile), epilogue through
// the layout maps into Cout (the step's own output, or the one a
// single-query launch names); returns this thread's sum of the values it
// wrote (for the probability check).  smem_a / smem_b: kBK x (BM+4) and
// kBK x (BN+4) floats of shared memory.  CG: read the operands from L2 (they
// were written earlier in the same launch).
template <int BM, int BN, int TM, int TN, bool CHUNKED, int kBK, int NT = kOpThreads, bool CG = false>
__device__ __forceinline__ double gemm_tile(const GemmArgs& a, int64_t m0, int64_t n0, float* smem_a,
                                            float* smem_b, void* Cout) {
  constexpr int kThreads = NT;
  static_assert((BM / TM) * (BN / TN) == kThreads, "tile shape");
  constexpr int TX = BN / TN;
  float (*As)[BM + 4] = reinterpret_cast<float (*)[BM + 4]>(smem_a);
  float (*Bs)[BN + 4] = reinterpret_cast<float (*)[BN + 4]>(smem_b);

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  // alpha is a power of two: scaling an FP32 partial by it is exact
  const float alpha_f = pow2_to_float(a.alpha);
  float acc[TM][TN];
  double acc64[CHUNKED ? TM : 1][CHUNKED ? TN : 1];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  if constexpr (CHUNKED) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc64[i][j] = 0.0;
  }

  // the operand loads of a stage are issued in groups of four before their
  // shared-memory stores, so that four are in flight together (one memory
  // round trip per group instead of one per load; four keeps the registers
  // of the deep tile shapes in bounds)
  constexpr int kLA = (BM * kBK + kThreads - 1) / kThreads;
  constexpr int kLB = (BN * kBK + kThreads - 1) / kThreads;
  constexpr int kG = 4;
  for (int64_t k0 = 0; k0 < a.K; k0 += kBK) {
#pragma unroll
    for (int g0 = 0; g0 < kLA; g0 += kG) {
      float rv[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int idx = tid + (g0 + u) * kThreads;
        const int r = idx / kBK, kk = idx % kBK;
        rv[u] = 0.f;
        if (g0 + u < kLA && idx < BM * kBK && m0 + r < a.M && k0 + kk < a.K)
          rv[u] = ld_operand<CG>(a.A + (m0 + r) * a.K + k0 + kk);
      }
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int idx = tid + (g0 + u) * kThreads;
        if (g0 + u < kLA && idx < BM * kBK) As[idx % kBK][idx / kBK] = rv[u];
      }
    }
#pragma unroll
    for (int g0 = 0; g0 < kLB; g0 += kG) {
      float rv[kG];
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int idx = tid + (g0 + u) * kThreads;
        const int r = idx / kBK, kk = idx % kBK;
        rv[u] = 0.f;
        if (g0 + u < kLB && idx < BN * kBK && n0 + r < a.N && k0 + kk < a.K)
          rv[u] = ld_operand<CG>(a.B + (n0 + r) * a.K + k0 + kk);
      }
#pragma unroll
      for (int u = 0; u < kG; ++u) {
        const int idx = tid + (g0 + u) * kThreads;
        if (g0 + u < kLB && idx < BN * kBK) Bs[idx % kBK][idx / kBK] = rv[u];
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float af[TM], bf[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) af[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bf[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(af[i], bf[j], acc[i][j]);
    }
    __syncthreads();
    if constexpr (CHUNKED) {
      const int64_t done = k0 + kBK;
      if ((done & (a.chunk - 1)) == 0 || done >= a.K) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            acc64[i][j] += f2d(acc[i][j] * alpha_f);
            acc[i][j] = 0.f;
          }
      }
    }
  }

  // FP32 outputs are scaled and summed in FP32; only FP64 outputs use the
  // FP64 pipe per element
  float sum_f = 0.f;
  double sum_d = 0.0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t row = m0 + ty * TM + i;
    if (row >= a.M) continue;
    const uint64_t rbase = a.rowmap[row];
    const int64_t c0 = n0 + tx * TN;
    if (!CHUNKED && a.kind == OUT_F32) {
      if (a.vec4 && (TN % 4) == 0 && c0 + TN <= a.N) {
#pragma unroll
        for (int j = 0; j < TN; j += 4) {
          float4 q;
          q.x = acc[i][j] * alpha_f; q.y = acc[i][j + 1] * alpha_f;
          q.z = acc[i][j + 2] * alpha_f; q.w = acc[i][j + 3] * alpha_f;
          sum_f += (q.x + q.y) + (q.z + q.w);
          float4* dst = reinterpret_cast<float4*>(static_cast<float*>(Cout) + rbase + a.colmap[c0 + j]);
          if (a.accumulate) {
            const float4 o = *dst;
            q.x += o.x; q.y += o.y; q.z += o.z; q.w += o.w;
          }
          *dst = q;
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int64_t col = c0 + j;
          if (col >= a.N) continue;
          const float v = acc[i][j] * alpha_f;
          sum_f += v;
          float* dst = static_cast<float*>(Cout) + rbase + a.colmap[col];
          *dst = a.accumulate ? *dst + v : v;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t col = c0 + j;
        if (col >= a.N) continue;
        double v;
        if constexpr (CHUNKED) v = acc64[i][j]; else v = f2d(acc[i][j] * alpha_f);
        if (a.kind == OUT_F64) sum_d += v; else sum_f += float(v);
        if (a.accumulate && a.kind == OUT_F64) {
          double* dst = static_cast<double*>(Cout) + rbase + a.colmap[col];
          *dst += v;                          // slices add up in FP64
        } else if (a.accumulate && a.kind == OUT_F32) {
          float* dst = static_cast<float*>(Cout) + rbase + a.colmap[col];
          *dst += float(v);
        } else {
          store_out(Cout, a.kind, a.plane_stride, rbase + a.colmap[col], v);
        }
      }
    }
  }
  return sum_d + double(sum_f);
}


}  // namespace sqc
