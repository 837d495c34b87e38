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

cudaError_t launch_mix(const MixArgs& a, cudaStream_t s) {
  const int64_t total = a.rows << a.n;
  mix_kernel<<<grid_for(total), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sqc
