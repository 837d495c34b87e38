// One contraction step of the compute graph in FP32 on the SIMT cores
// (Section 6.1: contracting two tensors over their shared cut edges is the
// matrix product C = A B^T with both operands K-contiguous).
//
// Register-tiled: a CTA computes a BM x BN tile with 256 threads, each a
// TM x TN block of outputs, staging BK = 16 columns of A and B through
// shared memory.  The epilogue scales by alpha (2^-K on the last step),
// writes every element to rowmap[i] + colmap[j] of its destination (the
// layout the next step reads, or the canonical bin order), in FP32, FP64
// or three BF16 planes, and adds the written values into per-CTA FP64
// partial sums that the last CTA reduces in a fixed order (the probability
// check).  With `chunk` > 0 the shared index is summed in FP32 chunks of
// `chunk` terms that are added up in FP64 registers (the cross-chunk sum).
#include "common.cuh"

namespace sqc {

namespace {

constexpr int kThreads = 256;

template <int BM, int BN, int TM, int TN, bool CHUNKED, int kBK>
__global__ void __launch_bounds__(kThreads) gemm_simt_kernel(GemmArgs a) {
  static_assert((BM / TM) * (BN / TN) == kThreads, "tile shape");
  constexpr int TX = BN / TN;
  __shared__ __align__(16) float As[kBK][BM + 4];
  __shared__ __align__(16) float Bs[kBK][BN + 4];
  __shared__ double red[kThreads / 32];

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  // M, N, BM, BN are powers of two: tile coordinates by shifts (64-bit
  // division is a long software sequence)
  const int64_t tiles_n = (a.N + BN - 1) / BN;
  const int tn_shift = __ffsll(tiles_n) - 1;
  const int64_t tile = int64_t(blockIdx.y) * gridDim.x + blockIdx.x;
  const int64_t m0 = (tile >> tn_shift) * BM;
  const int64_t n0 = (tile & (tiles_n - 1)) * BN;

  // alpha is a power of two: scaling an FP32 partial by it is exact
  const float alpha_f = float(a.alpha);
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

  for (int64_t k0 = 0; k0 < a.K; k0 += kBK) {
    for (int idx = tid; idx < BM * kBK; idx += kThreads) {
      const int r = idx / kBK, kk = idx % kBK;
      float v = 0.f;
      if (m0 + r < a.M && k0 + kk < a.K) v = __ldg(a.A + (m0 + r) * a.K + k0 + kk);
      As[kk][r] = v;
    }
    for (int idx = tid; idx < BN * kBK; idx += kThreads) {
      const int r = idx / kBK, kk = idx % kBK;
      float v = 0.f;
      if (n0 + r < a.N && k0 + kk < a.K) v = __ldg(a.B + (n0 + r) * a.K + k0 + kk);
      Bs[kk][r] = v;
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
            acc64[i][j] += double(acc[i][j] * alpha_f);
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
          *reinterpret_cast<float4*>(static_cast<float*>(a.C) + rbase + a.colmap[c0 + j]) = q;
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int64_t col = c0 + j;
          if (col >= a.N) continue;
          const float v = acc[i][j] * alpha_f;
          sum_f += v;
          static_cast<float*>(a.C)[rbase + a.colmap[col]] = v;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t col = c0 + j;
        if (col >= a.N) continue;
        double v;
        if constexpr (CHUNKED) v = acc64[i][j]; else v = double(acc[i][j] * alpha_f);
        if (a.kind == OUT_F64) sum_d += v; else sum_f += float(v);
        store_out(a.C, a.kind, a.plane_stride, rbase + a.colmap[col], v);
      }
    }
  }
  const double mysum = sum_d + double(sum_f);
  if (a.partials) finish_total(mysum, a.partials, a.counter, a.total, red);
}

template <int BM, int BN, int TM, int TN, bool CH, int BK = 16>
cudaError_t launch_cfg(const GemmArgs& a, cudaStream_t s) {
  const int64_t tiles = ((a.M + BM - 1) / BM) * ((a.N + BN - 1) / BN);
  const int64_t gx = tiles < 65535 ? tiles : 65535;
  const int64_t gy = (tiles + gx - 1) / gx;
  if (gx * gy != tiles) {
    // tiles is a product of powers of two: gx = 65535 never divides it, so
    // fall back to an exact power-of-two split
    int64_t x = 32768;
    while (tiles % x) x >>= 1;
    gemm_simt_kernel<BM, BN, TM, TN, CH, BK><<<dim3(unsigned(x), unsigned(tiles / x)), kThreads, 0, s>>>(a);
  } else {
    gemm_simt_kernel<BM, BN, TM, TN, CH, BK><<<dim3(unsigned(gx), unsigned(gy)), kThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_simt(const GemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaErrorInvalidValue;
  const bool chunked = a.chunk > 0;
  const bool wide = !chunked && a.kind == OUT_F32;
  auto tiles = [&](int bm, int bn) { return ((a.M + bm - 1) / bm) * ((a.N + bn - 1) / bn); };
  const int64_t want = 152;   // at least one full wave of CTAs
  if (wide && tiles(128, 128) >= want) return launch_cfg<128, 128, 8, 8, false>(a, s);
  if (!wide && tiles(128, 64) >= want) {
    if (chunked) return launch_cfg<128, 64, 8, 4, true>(a, s);
    return launch_cfg<128, 64, 8, 4, false>(a, s);
  }
  // small steps: few CTAs, so stage up to 64 shared-index columns per
  // round (fewer dependent load rounds)
  const bool deep = a.K >= 64 && (!chunked || a.chunk % 64 == 0);
  if (tiles(64, 64) >= want) {
    if (chunked) return deep ? launch_cfg<64, 64, 4, 4, true, 64>(a, s) : launch_cfg<64, 64, 4, 4, true>(a, s);
    return deep ? launch_cfg<64, 64, 4, 4, false, 64>(a, s) : launch_cfg<64, 64, 4, 4, false>(a, s);
  }
  if (chunked) return deep ? launch_cfg<32, 32, 2, 2, true, 64>(a, s) : launch_cfg<32, 32, 2, 2, true>(a, s);
  return deep ? launch_cfg<32, 32, 2, 2, false, 64>(a, s) : launch_cfg<32, 32, 2, 2, false>(a, s);
}

}  // namespace sqc
