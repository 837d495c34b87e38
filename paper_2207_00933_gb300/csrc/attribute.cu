// Attribution of subcircuit variant outputs to cut-edge labels (Eq. 1 with
// the I/X/Y/Z expansion of each cut wire, Section 2.1):
//
//   A_i[e][x] = sum_{s,c} prod_{in-edges t} D[e_t][s_t]
//                         prod_{out-edges u} W[e_u][c_u]  p_i[v(s, e)][x | c << n]
//
// evaluated in two HBM/L2-streaming passes: `fold` sums the outcomes c of
// the outgoing cut wires (the basis is already the variant digit), and `mix`
// combines the prepared states s of the incoming cut wires.  The data index
// is stored bit-reversed so that, under the recursion's roles (zoomed =
// low data qubits, merged = high), a bin's states are one contiguous run.
#include "internal.h"

namespace sqc {

namespace {

__device__ __forceinline__ uint32_t rev_bits(uint32_t x, int n) {
  return n == 0 ? 0u : (__brev(x) >> (32 - n));
}

template <typename T>
__global__ void __launch_bounds__(256) fold_kernel(FoldArgs a) {
  const T* p = static_cast<const T*>(a.p);
  const int64_t X = int64_t(1) << a.n;
  const int64_t total = a.V * X;
  const int64_t row_len = X << a.kout;
  const int nc = 1 << a.kout;
  for (int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; o < total;
       o += int64_t(gridDim.x) * blockDim.x) {
    const int64_t v = o >> a.n;
    const uint32_t x = uint32_t(o & (X - 1));
    // outgoing edges measured in X, Y or Z weigh outcome 1 by -1
    uint32_t signed_mask = 0;
    for (int u = 0; u < a.kout; ++u)
      if ((v >> a.outshift[u]) & 3) signed_mask |= 1u << u;
    const T* row = p + v * row_len + x;
    float acc = 0.f;
    for (int c = 0; c < nc; ++c) {
      const float val = float(row[int64_t(c) << a.n]);
      acc += (__popc(uint32_t(c) & signed_mask) & 1) ? -val : val;
    }
    a.B[v * X + rev_bits(x, a.n)] = acc;
  }
}

__global__ void __launch_bounds__(256) mix_kernel(MixArgs a) {
  const int64_t X = int64_t(1) << a.n;
  const int64_t total = a.rows * X;
  for (int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; o < total;
       o += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = o >> a.n;
    const int64_t xs = o & (X - 1);
    // radix of each incoming edge: I, Z expand over |0>,|1>; X, Y also over |+>/|+i>
    int radix[16];
    int64_t combos = 1;
    int64_t base = e;
    for (int t = 0; t < a.kin; ++t) {
      const int d = int((e >> a.inshift[t]) & 3);
      radix[t] = (d == 1 || d == 2) ? 3 : 2;
      combos *= radix[t];
      base &= ~(int64_t(3) << a.inshift[t]);
    }
    float acc = 0.f;
    for (int64_t cidx = 0; cidx < combos; ++cidx) {
      int64_t rem = cidx;
      int64_t v = base;
      float coef = 1.f;
      for (int t = 0; t < a.kin; ++t) {
        const int opt = int(rem % radix[t]);
        rem /= radix[t];
        const int d = int((e >> a.inshift[t]) & 3);
        int s;
        float w;
        if (d == 0) {            // I = |0><0| + |1><1|
          s = opt; w = 1.f;
        } else if (d == 3) {     // Z = |0><0| - |1><1|
          s = opt; w = opt ? -1.f : 1.f;
        } else if (opt < 2) {    // X = 2|+><+| - I,  Y = 2|+i><+i| - I
          s = opt; w = -1.f;
        } else {
          s = (d == 1) ? 2 : 3; w = 2.f;
        }
        v |= int64_t(s) << a.inshift[t];
        coef *= w;
      }
      acc = fmaf(coef, a.B[v * X + xs], acc);
    }
    a.A[o] = acc;
  }
}

__device__ __forceinline__ int64_t variant_of(const AttrDesc& d, int64_t vbase, int s) {
  int64_t v = vbase;
  for (int q = 0; q < d.kin; ++q) v |= int64_t((s >> (2 * q)) & 3) << d.inshift[q];
  return v;
}

__device__ __forceinline__ int64_t x_in_tile(const AttrDesc& d, int64_t xm, int j) {
  const int64_t jl = j & ((1 << d.L1) - 1);
  const int64_t jh = j >> d.L1;
  return jl | (xm << d.L1) | (jh << (d.n - d.L2));
}

// Phase 1 of the fused attribution: fold the outcomes of the outgoing wires
// for every (s, x) of the tile into shared memory.  NC = outcomes handled per
// round (all of them when 2^kout <= 8); kU entries per thread per round, so
// that NC x kU independent loads are in flight.
template <int NC, bool F64>
__device__ __forceinline__ void fold_phase(const AttrDesc& d, float* val, int S, int lt, int64_t vbase,
                                           uint32_t signed_mask) {
  constexpr int kU = NC >= 8 ? 2 : (NC >= 4 ? 4 : 8);
  // tiles are (x middle bits) x (4^kout outgoing bases): shifts, no division
  const int64_t xm = (int64_t(blockIdx.x) - d.block_begin) >> (2 * d.kout);
  const int n = d.n;
  const int64_t row_len = (int64_t(1) << n) << d.kout;
  const int nc = 1 << d.kout;
  const int total = S << lt;
  const float* p32 = static_cast<const float*>(d.p);
  const double* p64 = static_cast<const double*>(d.p);
  for (int b0 = 0; b0 < total; b0 += int(blockDim.x) * kU) {
    int64_t base[kU];
    float acc[kU];
    bool ok[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int idx = b0 + u * int(blockDim.x) + int(threadIdx.x);
      ok[u] = idx < total;
      const int s = ok[u] ? idx >> lt : 0, j = ok[u] ? idx & ((1 << lt) - 1) : 0;
      base[u] = variant_of(d, vbase, s) * row_len + x_in_tile(d, xm, j);
      acc[u] = 0.f;
    }
    for (int c0 = 0; c0 < nc; c0 += NC) {
      float w[NC][kU];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int64_t a = base[u] + (int64_t(c0 + cc) << n);
          // the input type is a template parameter: FP64 conversions (a
          // narrow pipe on this GPU) exist only in the FP64-input variant
          if constexpr (F64)
            w[cc][u] = ok[u] ? float(__ldg(p64 + a)) : 0.f;
          else
            w[cc][u] = ok[u] ? __ldg(p32 + a) : 0.f;
        }
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) {
        const bool neg = __popc(uint32_t(c0 + cc) & signed_mask) & 1;
#pragma unroll
        for (int u = 0; u < kU; ++u) acc[u] += neg ? -w[cc][u] : w[cc][u];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (ok[u]) val[b0 + u * int(blockDim.x) + int(threadIdx.x)] = acc[u];
  }
}

// Fused attribution for subcircuits with at most kMaxFusedIn incoming cut
// edges.  A CTA owns one tile of data states x (2^L1 consecutive low values
// times 2^L2 values of the top bits, so that both the reads of p and the
// bit-reversed writes of A touch whole 32-byte sectors) for one combination
// o of outgoing-edge bases and all 4^kin prepared-state combinations s:
//   1. load and fold the outcomes c of the outgoing wires into shared memory,
//   2. apply the incoming-edge expansion one edge at a time in place:
//      (|0>,|1>,|+>,|+i>) -> (I, X, Y, Z) = (a+b, 2c-(a+b), 2d-(a+b), a-b),
//   3. write the 4^kin labelled rows to A (data index bit-reversed).
// Every variant output is read once.
__global__ void __launch_bounds__(256) attr_fused_kernel(AttrLaunch L) {
  extern __shared__ float val[];
  // the descriptor of this CTA, copied with constant parameter offsets only
  // (a dynamic index into the parameter block would copy all of it to local
  // memory in every thread)
  __shared__ AttrDesc d;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < kAttrPerLaunch; ++i)
      if (i < L.n && L.d[i].block_begin <= int64_t(blockIdx.x)) d = L.d[i];
  }
  __syncthreads();
  const int64_t t = int64_t(blockIdx.x) - d.block_begin;
  const int64_t o = t & ((int64_t(1) << (2 * d.kout)) - 1);
  const int64_t xm = t >> (2 * d.kout);
  const int S = 1 << (2 * d.kin);
  const int TX = 1 << (d.L1 + d.L2);
  const int n = d.n;
  const int64_t X = int64_t(1) << n;
  // base variant index: the outgoing edges' bases from o
  int64_t vbase = 0;
  uint32_t signed_mask = 0;
  for (int u = 0; u < d.kout; ++u) {
    const int64_t dig = (o >> (2 * u)) & 3;
    vbase |= dig << d.outshift[u];
    if (dig) signed_mask |= 1u << u;
  }
  // phase 1, specialised on the number of outcomes so that no load slot is
  // predicated away
  const int lt = d.L1 + d.L2;
  if (d.in_f64) {
    switch (d.kout) {
      case 0: fold_phase<1, true>(d, val, S, lt, vbase, signed_mask); break;
      case 1: fold_phase<2, true>(d, val, S, lt, vbase, signed_mask); break;
      case 2: fold_phase<4, true>(d, val, S, lt, vbase, signed_mask); break;
      default: fold_phase<8, true>(d, val, S, lt, vbase, signed_mask); break;
    }
  } else {
    switch (d.kout) {
      case 0: fold_phase<1, false>(d, val, S, lt, vbase, signed_mask); break;
      case 1: fold_phase<2, false>(d, val, S, lt, vbase, signed_mask); break;
      case 2: fold_phase<4, false>(d, val, S, lt, vbase, signed_mask); break;
      default: fold_phase<8, false>(d, val, S, lt, vbase, signed_mask); break;
    }
  }
  __syncthreads();
  for (int q = 0; q < d.kin; ++q) {
    const int lowmask = (1 << (2 * q)) - 1;
    for (int idx = threadIdx.x; idx < (S / 4) * TX; idx += blockDim.x) {
      const int g = idx >> lt, j = idx & (TX - 1);
      const int s0 = ((g & ~lowmask) << 2) | (g & lowmask);
      const int st = 1 << (2 * q);
      float* a = val + s0 * TX + j;
      const float v0 = a[0], v1 = a[st * TX], v2 = a[2 * st * TX], v3 = a[3 * st * TX];
      const float sum = v0 + v1;
      a[0] = sum;                       // I
      a[st * TX] = 2.f * v2 - sum;      // X
      a[2 * st * TX] = 2.f * v3 - sum;  // Y
      a[3 * st * TX] = v0 - v1;         // Z
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < S * TX; idx += blockDim.x) {
    const int s = idx >> lt, jr = idx & (TX - 1);
    const int jh = jr & ((1 << d.L2) - 1), jl = jr >> d.L2;
    const int j = jl | (jh << d.L1);
    const int64_t e = variant_of(d, vbase, s);
    d.A[e * X + rev_bits(uint32_t(x_in_tile(d, xm, j)), n)] = val[s * TX + j];
  }
}

inline int grid_for(int64_t total) {
  int64_t g = (total + 255) / 256;
  const int64_t cap = 152 * 16;
  return int(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_fold(const FoldArgs& a, cudaStream_t s) {
  const int64_t total = a.V << a.n;
  if (a.in_f64)
    fold_kernel<double><<<grid_for(total), 256, 0, s>>>(a);
  else
    fold_kernel<float><<<grid_for(total), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_attr_fused(const AttrLaunch& L, int64_t blocks, int smem_bytes, cudaStream_t s) {
  if (L.n <= 0 || blocks <= 0) return cudaSuccess;
  attr_fused_kernel<<<unsigned(blocks), 256, smem_bytes, s>>>(L);
  return cudaGetLastError();
}

cudaError_t attr_configure() {
  return cudaFuncSetAttribute(attr_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kAttrSmemMax);
}

cudaError_t launch_mix(const MixArgs& a, cudaStream_t s) {
  const int64_t total = a.rows << a.n;
  mix_kernel<<<grid_for(total), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sqc
