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
#include "device_ops.cuh"

namespace sqc {

namespace {

constexpr int kThreads = kOpThreads;

template <int BM, int BN, int TM, int TN, bool CHUNKED, int kBK>
__global__ void __launch_bounds__(kThreads, 2) gemm_simt_kernel(GemmArgs a) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  __shared__ __align__(16) float As[kBK * (BM + 4)];
  __shared__ __align__(16) float Bs[kBK * (BN + 4)];
  __shared__ double red[kThreads / 32];
  // M, N, BM, BN are powers of two: tile coordinates by shifts (64-bit
  // division is a long software sequence)
  const int64_t tiles_n = (a.N + BN - 1) / BN;
  const int tn_shift = __ffsll(tiles_n) - 1;
  const int64_t tile = int64_t(blockIdx.y) * gridDim.x + blockIdx.x;
  const int64_t m0 = (tile >> tn_shift) * BM;
  const int64_t n0 = (tile & (tiles_n - 1)) * BN;
  const double mysum = gemm_tile<BM, BN, TM, TN, CHUNKED, kBK>(a, m0, n0, As, Bs, a.C);
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
    return launch_k(gemm_simt_kernel<BM, BN, TM, TN, CH, BK>, dim3(unsigned(x), unsigned(tiles / x)), dim3(kThreads),
                    0, s, false, a);
  }
  return launch_k(gemm_simt_kernel<BM, BN, TM, TN, CH, BK>, dim3(unsigned(gx), unsigned(gy)), dim3(kThreads), 0, s,
                  false, a);
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
