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
#include "common.cuh"

#include <atomic>

namespace sqc {

namespace {

__device__ __forceinline__ uint32_t rev_bits(uint32_t x, int n) {
  return n == 0 ? 0u : (__brev(x) >> (32 - n));
}

template <typename T>
__global__ void __launch_bounds__(256) fold_kernel(FoldArgs a) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
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
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
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

// ---- fused attribution -------------------------------------------------------
// For subcircuits with at most kMaxFusedIn incoming cut edges.  A CTA owns
// one tile: 2^L1 consecutive low values of the data state x times 2^L2
// values of its top bits (so that the reads of p run over 2^L1 consecutive
// x and the bit-reversed writes of A over 2^L2 consecutive storage
// addresses), for one combination o of outgoing-edge bases and all 4^kin
// prepared-state combinations s:
//   1. fold the outcomes c of the outgoing wires into shared memory,
//   2. expand the incoming edges one at a time in place:
//      (|0>,|1>,|+>,|+i>) -> (I, X, Y, Z) = (a+b, 2c-(a+b), 2d-(a+b), a-b),
//   3. write the 4^kin labelled rows to A (data index bit-reversed).
// Every variant output is read once.
//
// A tile holds TX = 2^(L1+L2) <= 256 states, so with 256 threads every
// thread keeps the same state slot j in all three phases and only steps
// through the rows s; the per-element work is a table lookup, an OR and a
// shift.  The slot's shared-memory position is XOR-swizzled so that phase
// 3, which reads the slots in storage order (top bits fastest), hits 32
// distinct banks.
struct AttrTileCtx {
  uint64_t vlo[256];   // variant-index contribution of the low 4 in-edge digits of s
  uint64_t vhi[64];    // ... of the digits above them
};

__device__ __forceinline__ uint64_t in_digits(const AttrTileCtx& t, int s) {
  return t.vlo[s & 255] | t.vhi[s >> 8];
}

// shared-memory position of slot j = jl | jh << L1 within a row
__device__ __forceinline__ int slot_pos(int j, int L1, int L2) {
  if (L1 + L2 <= 5) return j;
  const int jh = j >> L1;
  const int m = L1 >= 5 ? jh : (jh >> (5 - L1));
  return j ^ ((m << (5 - L2)) & ((1 << L1) - 1));
}

// Shared-memory slot of state j in the 4-states-per-thread forms: the 5/3
// tile shape (128-byte reads, 32-byte write runs) swizzles as slot_pos
// does; the 4/4 shape (64-byte reads and write runs) needs no swizzle
// (phase 3 then reads with at most 2-way bank conflicts).
template <int L1>
__device__ __forceinline__ int v4_pos(int j) {
  if constexpr (L1 == 5) return slot_pos(j, 5, 3);
  else return j;
}

template <int NC, bool F64, class Desc>
__device__ __forceinline__ void fold_phase(const Desc& d, const AttrTileCtx& t, float* val, int S, int lt,
                                           uint64_t x, int pos, uint64_t vbase, uint32_t signed_mask) {
  constexpr int kU = NC >= 8 ? 2 : (NC >= 4 ? 4 : 8);
  const int n = d.n;
  const int row_shift = n + d.kout;
  const int nc = 1 << d.kout;
  const int TX = 1 << lt;
  const int step = int(blockDim.x) >> lt;
  const float* p32 = static_cast<const float*>(d.p);
  const double* p64 = static_cast<const double*>(d.p);
  for (int s0 = int(threadIdx.x) >> lt; s0 < S; s0 += step * kU) {
    uint64_t base[kU];
    float acc[kU];
    bool ok[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int s = s0 + u * step;
      ok[u] = s < S;
      base[u] = ((in_digits(t, ok[u] ? s : 0) | vbase) << row_shift) + x;
      acc[u] = 0.f;
    }
    for (int c0 = 0; c0 < nc; c0 += NC) {
      float w[NC][kU];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const uint64_t a = base[u] + (uint64_t(c0 + cc) << n);
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
      if (ok[u]) val[(s0 + u * step) * TX + pos] = acc[u];
  }
}

// One tile (index t relative to the descriptor's first tile).  F64: the
// FP64-input folds are compiled in.
template <bool F64>
__device__ __forceinline__ void attr_tile(const AttrDesc& d, const AttrTileCtx& tc, int64_t t, float* val) {
  // tiles are (x middle bits) x (4^kout outgoing bases): shifts, no division
  const uint64_t o = uint64_t(t) & ((uint64_t(1) << (2 * d.kout)) - 1);
  const uint64_t xm = uint64_t(t) >> (2 * d.kout);
  const int S = 1 << (2 * d.kin);
  const int L1 = d.L1, L2 = d.L2, lt = L1 + L2;
  const int TX = 1 << lt;
  const int n = d.n;
  const int step = int(blockDim.x) >> lt;
  // the outgoing edges' bases from o
  uint64_t vbase = 0;
  uint32_t signed_mask = 0;
  for (int u = 0; u < d.kout; ++u) {
    const uint64_t dig = (o >> (2 * u)) & 3;
    vbase |= dig << d.outshift[u];
    if (dig) signed_mask |= 1u << u;
  }
  // this thread's slot in phases 1-2: j = low bits of the thread index
  const int j = int(threadIdx.x) & (TX - 1);
  auto x_of = [&](int jj) -> uint64_t {
    const uint64_t jl = uint64_t(jj & ((1 << L1) - 1)), jh = uint64_t(jj >> L1);
    return jl | (xm << L1) | (jh << (n - L2));
  };
  const int pos = slot_pos(j, L1, L2);
  if (F64 && d.in_f64) {
    switch (d.kout) {
      case 0: fold_phase<1, true>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
      case 1: fold_phase<2, true>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
      case 2: fold_phase<4, true>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
      default: fold_phase<8, true>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
    }
  } else {
    switch (d.kout) {
      case 0: fold_phase<1, false>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
      case 1: fold_phase<2, false>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
      case 2: fold_phase<4, false>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
      default: fold_phase<8, false>(d, tc, val, S, lt, x_of(j), pos, vbase, signed_mask); break;
    }
  }
  __syncthreads();
  for (int q = 0; q < d.kin; ++q) {
    const int lowmask = (1 << (2 * q)) - 1;
    const int st = TX << (2 * q);
    for (int g = int(threadIdx.x) >> lt; g < (S >> 2); g += step) {
      const int s0 = ((g & ~lowmask) << 2) | (g & lowmask);
      float* a = val + s0 * TX + pos;
      const float v0 = a[0], v1 = a[st], v2 = a[2 * st], v3 = a[3 * st];
      const float sum = v0 + v1;
      a[0] = sum;                 // I
      a[st] = 2.f * v2 - sum;     // X
      a[2 * st] = 2.f * v3 - sum; // Y
      a[3 * st] = v0 - v1;        // Z
    }
    __syncthreads();
  }
  // phase 3: slot order with the top bits fastest, so that consecutive
  // threads write consecutive (bit-reversed) storage addresses
  const int jh = j & ((1 << L2) - 1), jl = j >> L2;
  const int jw = jl | (jh << L1);
  const int posw = slot_pos(jw, L1, L2);
  const uint64_t xw = rev_bits(uint32_t(x_of(jw)), n);
  for (int s = int(threadIdx.x) >> lt; s < S; s += step)
    d.A[((in_digits(tc, s) | vbase) << n) + xw] = val[s * TX + posw];
}


// The same tile for the largest tile shape (32 x 8 states, TX = 256) with
// FP32 input: every thread handles 4 consecutive states (one 16-byte load
// per row and outcome, 16-byte shared-memory and global accesses).  64
// threads cover a row, so 4 rows are in flight per pass.  In phase 3 a
// thread writes 4 consecutive storage addresses of A: the same low state
// bits with the top bits jh = rev3(r), r = r0 .. r0+3 (the top 3 state
// bits are the low 3 storage bits, reversed).
template <int NC>
__device__ __forceinline__ void fold_phase_v4(const AttrDesc& d, const AttrTileCtx& t, float* val, int S,
                                              uint64_t x0, int pos, uint64_t vbase, uint32_t signed_mask) {
  constexpr int kU = NC >= 4 ? 1 : (NC >= 2 ? 2 : 4);   // rows per thread per round
  const int n = d.n;
  const int row_shift = n + d.kout;
  const int nc = 1 << d.kout;
  const float* p = static_cast<const float*>(d.p);
  for (int s0 = int(threadIdx.x) >> 6; s0 < S; s0 += 4 * kU) {
    uint64_t base[kU];
    float4 acc[kU];
    bool ok[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int s = s0 + 4 * u;
      ok[u] = s < S;
      base[u] = ((in_digits(t, ok[u] ? s : 0) | vbase) << row_shift) + x0;
      acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int c0 = 0; c0 < nc; c0 += NC) {
      float4 w[NC][kU];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
#pragma unroll
        for (int u = 0; u < kU; ++u)
          w[cc][u] = ok[u] ? __ldg(reinterpret_cast<const float4*>(p + base[u] + (uint64_t(c0 + cc) << n)))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) {
        const float sg = (__popc(uint32_t(c0 + cc) & signed_mask) & 1) ? -1.f : 1.f;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          acc[u].x = fmaf(sg, w[cc][u].x, acc[u].x);
          acc[u].y = fmaf(sg, w[cc][u].y, acc[u].y);
          acc[u].z = fmaf(sg, w[cc][u].z, acc[u].z);
          acc[u].w = fmaf(sg, w[cc][u].w, acc[u].w);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (ok[u]) *reinterpret_cast<float4*>(val + (s0 + 4 * u) * 256 + pos) = acc[u];
  }
}

template <int L1>
__device__ __forceinline__ void attr_tile_v4(const AttrDesc& d, const AttrTileCtx& tc, int64_t t, float* val) {
  constexpr int L2 = 8 - L1;
  const uint64_t o = uint64_t(t) & ((uint64_t(1) << (2 * d.kout)) - 1);
  const uint64_t xm = uint64_t(t) >> (2 * d.kout);
  const int S = 1 << (2 * d.kin);
  const int n = d.n;
  uint64_t vbase = 0;
  uint32_t signed_mask = 0;
  for (int u = 0; u < d.kout; ++u) {
    const uint64_t dig = (o >> (2 * u)) & 3;
    vbase |= dig << d.outshift[u];
    if (dig) signed_mask |= 1u << u;
  }
  const int g = int(threadIdx.x) & 63;
  const int j0 = 4 * g;                              // 4 consecutive low bits, one jh
  const uint64_t x0 = uint64_t(j0 & ((1 << L1) - 1)) | (xm << L1) | (uint64_t(j0 >> L1) << (n - L2));
  const int pos = v4_pos<L1>(j0);                    // a multiple of 4
  switch (d.kout) {
    case 0: fold_phase_v4<1>(d, tc, val, S, x0, pos, vbase, signed_mask); break;
    case 1: fold_phase_v4<2>(d, tc, val, S, x0, pos, vbase, signed_mask); break;
    case 2: fold_phase_v4<4>(d, tc, val, S, x0, pos, vbase, signed_mask); break;
    default: fold_phase_v4<8>(d, tc, val, S, x0, pos, vbase, signed_mask); break;
  }
  __syncthreads();
  for (int q = 0; q < d.kin; ++q) {
    const int lowmask = (1 << (2 * q)) - 1;
    const int st = 256 << (2 * q);
    for (int gg = int(threadIdx.x) >> 6; gg < (S >> 2); gg += 4) {
      const int s0 = ((gg & ~lowmask) << 2) | (gg & lowmask);
      float* a = val + s0 * 256 + pos;
      const float4 v0 = *reinterpret_cast<const float4*>(a);
      const float4 v1 = *reinterpret_cast<const float4*>(a + st);
      const float4 v2 = *reinterpret_cast<const float4*>(a + 2 * st);
      const float4 v3 = *reinterpret_cast<const float4*>(a + 3 * st);
      const float4 sm = make_float4(v0.x + v1.x, v0.y + v1.y, v0.z + v1.z, v0.w + v1.w);
      *reinterpret_cast<float4*>(a) = sm;                                                     // I
      *reinterpret_cast<float4*>(a + st) =
          make_float4(2.f * v2.x - sm.x, 2.f * v2.y - sm.y, 2.f * v2.z - sm.z, 2.f * v2.w - sm.w);   // X
      *reinterpret_cast<float4*>(a + 2 * st) =
          make_float4(2.f * v3.x - sm.x, 2.f * v3.y - sm.y, 2.f * v3.z - sm.z, 2.f * v3.w - sm.w);   // Y
      *reinterpret_cast<float4*>(a + 3 * st) =
          make_float4(v0.x - v1.x, v0.y - v1.y, v0.z - v1.z, v0.w - v1.w);                   // Z
    }
    __syncthreads();
  }
  // phase 3: thread g writes storage offsets r0 .. r0+3 of low state bits
  // jl (top state bits jh = the L2-bit reversal of the offset)
  constexpr int kPerJl = (1 << L2) / 4;
  const int jl = g / kPerJl, r0 = (g % kPerJl) * 4;
  int pw[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) pw[q] = v4_pos<L1>(jl | (int(__brev(uint32_t(r0 + q)) >> (32 - L2)) << L1));
  const uint64_t xw = rev_bits(uint32_t(uint64_t(jl) | (xm << L1)), n) + uint64_t(r0);
  for (int s = int(threadIdx.x) >> 6; s < S; s += 4) {
    const float* v = val + s * 256;
    *reinterpret_cast<float4*>(d.A + ((in_digits(tc, s) | vbase) << n) + xw) =
        make_float4(v[pw[0]], v[pw[1]], v[pw[2]], v[pw[3]]);
  }
}

// No incoming edges (a single prepared-state row): work unit t is the four
// tiles 4t .. 4t+3, one per 64-thread group, each group folding the
// outcomes of its 256 states (4 per thread) and writing them through its
// own 256-float region of shared memory.
template <int L1>
__device__ __forceinline__ void attr_tiles_v4_kin0(const AttrDesc& d, int64_t t, float* val) {
  constexpr int L2 = 8 - L1;
  const int g4 = int(threadIdx.x) >> 6;
  const uint64_t tt = uint64_t(t) * 4 + uint64_t(g4);
  const uint64_t o = tt & ((uint64_t(1) << (2 * d.kout)) - 1);
  const uint64_t xm = tt >> (2 * d.kout);
  const int n = d.n;
  uint64_t vbase = 0;
  uint32_t signed_mask = 0;
  for (int u = 0; u < d.kout; ++u) {
    const uint64_t dig = (o >> (2 * u)) & 3;
    vbase |= dig << d.outshift[u];
    if (dig) signed_mask |= 1u << u;
  }
  const int g = int(threadIdx.x) & 63;
  const int j0 = 4 * g;
  const uint64_t x0 = uint64_t(j0 & ((1 << L1) - 1)) | (xm << L1) | (uint64_t(j0 >> L1) << (n - L2));
  const int pos = v4_pos<L1>(j0);
  float* mine = val + g4 * 256;
  const float* p = static_cast<const float*>(d.p) + (vbase << (n + d.kout)) + x0;
  const int nc = 1 << d.kout;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int c0 = 0; c0 < nc; c0 += 4) {
    float4 w[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
      w[cc] = c0 + cc < nc ? __ldg(reinterpret_cast<const float4*>(p + (uint64_t(c0 + cc) << n)))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const float sg = (__popc(uint32_t(c0 + cc) & signed_mask) & 1) ? -1.f : 1.f;
      acc.x = fmaf(sg, w[cc].x, acc.x);
      acc.y = fmaf(sg, w[cc].y, acc.y);
      acc.z = fmaf(sg, w[cc].z, acc.z);
      acc.w = fmaf(sg, w[cc].w, acc.w);
    }
  }
  *reinterpret_cast<float4*>(mine + pos) = acc;
  __syncthreads();
  constexpr int kPerJl = (1 << L2) / 4;
  const int jl = g / kPerJl, r0 = (g % kPerJl) * 4;
  float o4[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) o4[q] = mine[v4_pos<L1>(jl | (int(__brev(uint32_t(r0 + q)) >> (32 - L2)) << L1))];
  const uint64_t xw = rev_bits(uint32_t(uint64_t(jl) | (xm << L1)), n) + uint64_t(r0);
  *reinterpret_cast<float4*>(d.A + (vbase << n) + xw) = make_float4(o4[0], o4[1], o4[2], o4[3]);
}

// ---- double-buffered form (no outgoing edges, 4^kin <= 32): the rows of
// the next tiles are copied into other buffers of a ring in shared memory
// by cp.async while this tile is expanded and written.  A tile is 2^L1 low
// x 2^L2 top data states (4 consecutive states per thread and row), so the
// reads of p run over 2^L1 consecutive states and the bit-reversed writes
// of A over 2^L2 consecutive storage addresses.  This form writes as many
// bytes as it reads, and its write runs set its speed.  Measured at 592 MB
// per step with one side of the traffic cut out: the writes alone took 115
// us in 64-byte runs and 95 us in 128- or 256-byte runs; the reads alone 95
// us in 64- or 128-byte runs, 110 us in 32-byte and 124 us in 16-byte runs.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(uint32_t(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// the 4^kin rows of tile t into buf, state j of a row at buf + row * 2^(L1+L2) + j
template <int L1, int L2>
__device__ __forceinline__ void ring_issue(const AttrDesc& d, const AttrTileCtx& tc, int64_t t, float* buf) {
  constexpr int TS = 1 << (L1 + L2);                // states per tile
  constexpr int TPR = TS / 4;                       // threads per row
  constexpr int RPP = 256 / TPR;                    // rows per pass of 256 threads
  const uint64_t xm = uint64_t(t);                  // no outgoing edges: tile = x middle bits
  const int S = 1 << (2 * d.kin), n = d.n;
  const int j0 = 4 * (int(threadIdx.x) % TPR);
  const uint64_t x0 = uint64_t(j0 & ((1 << L1) - 1)) | (xm << L1) | (uint64_t(j0 >> L1) << (n - L2));
  const float* p = static_cast<const float*>(d.p);
  for (int s = int(threadIdx.x) / TPR; s < S; s += RPP) cp_async16(buf + s * TS + j0, p + (in_digits(tc, s) << n) + x0);
}

// the incoming edges' expansion of one state slot held in registers: the
// 4^KIN values of slot p (stride TS), each digit q in turn, with the same
// operations per element as the shared-memory passes
template <int KIN, int TS>
__device__ __forceinline__ void ring_expand_slot(float* val, int p) {
  constexpr int S = 1 << (2 * KIN);
  float v[S];
#pragma unroll
  for (int s = 0; s < S; ++s) v[s] = val[s * TS + p];
#pragma unroll
  for (int q = 0; q < KIN; ++q) {
    const int st = 1 << (2 * q);
#pragma unroll
    for (int g = 0; g < S / 4; ++g) {
      const int lowmask = st - 1;
      const int s0 = ((g & ~lowmask) << 2) | (g & lowmask);
      const float v0 = v[s0], v1 = v[s0 + st], v2 = v[s0 + 2 * st], v3 = v[s0 + 3 * st];
      const float sum = v0 + v1;
      v[s0] = sum;                  // I
      v[s0 + st] = 2.f * v2 - sum;  // X
      v[s0 + 2 * st] = 2.f * v3 - sum;  // Y
      v[s0 + 3 * st] = v0 - v1;     // Z
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s) val[s * TS + p] = v[s];
}

// expansion of the incoming edges and the bit-reversed write of tile t
template <int L1, int L2>
__device__ __forceinline__ void ring_finish(const AttrDesc& d, const AttrTileCtx& tc, int64_t t, float* val) {
  constexpr int TS = 1 << (L1 + L2);
  constexpr int TPR = TS / 4;
  constexpr int RPP = 256 / TPR;
  const uint64_t xm = uint64_t(t);
  const int S = 1 << (2 * d.kin), n = d.n;
  // thread i expands the 4^kin values of state slots i, i + 256, ... in
  // registers, one CTA barrier in all
  for (int j = int(threadIdx.x); j < TS; j += 256) {
    if (d.kin == 1) ring_expand_slot<1, TS>(val, j);
    else ring_expand_slot<2, TS>(val, j);
  }
  __syncthreads();
  // thread g writes storage offsets r0 .. r0+3 (top state bits jh = the
  // L2-bit reversal of the offset) of the low state bits jl
  constexpr int kPerJl = (1 << L2) / 4;             // threads per low-bit value
  const int g = int(threadIdx.x) % TPR;
  const int jl = g / kPerJl, r0 = (g % kPerJl) * 4;
  int pw[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) pw[q] = jl | (int(__brev(uint32_t(r0 + q)) >> (32 - L2)) << L1);
  const uint64_t xw = rev_bits(uint32_t(uint64_t(jl) | (xm << L1)), n) + uint64_t(r0);
  for (int s = int(threadIdx.x) / TPR; s < S; s += RPP) {
    const float* v = val + s * TS;
    *reinterpret_cast<float4*>(d.A + (in_digits(tc, s) << n) + xw) = make_float4(v[pw[0]], v[pw[1]], v[pw[2]], v[pw[3]]);
  }
}

template <class Desc>
__device__ void fill_tile_ctx(const Desc& d, AttrTileCtx& t) {
  for (int i = threadIdx.x; i < 256 + 64; i += blockDim.x) {
    const int s = i < 256 ? i : ((i - 256) << 8);
    uint64_t v = 0;
    for (int q = 0; q < d.kin; ++q) v |= uint64_t((s >> (2 * q)) & 3) << d.inshift[q];
    if (i < 256) t.vlo[i] = v;
    else t.vhi[i - 256] = v;
  }
}

// Persistent: CTAs walk the tiles of all descriptors; a CTA copies a
// descriptor into shared memory only when it crosses into it (constant
// parameter offsets only: a dynamic index into the parameter block would copy
// all of it to local memory in every thread).
// MODE selects the forms compiled in, so that a launch runs the smallest
// kernel that covers its descriptors (fewer registers, and for small
// subcircuits fewer instruction-cache misses):
//   kAttrAll  -- every form;
//   kAttrVec  -- every descriptor takes a 4-state-per-thread form (at most
//                40 registers, for six CTAs per SM);
//   kAttrVec3 -- the same forms, for launches whose shared memory allows
//                three CTAs per SM at most (the double-buffered form's
//                ring): up to 80 registers, where kAttrVec spills (at 592
//                MB per step 125.5 us against 134.1 us);
//   kAttrOne  -- every descriptor takes the one-state form with FP32 input.
enum : int { kAttrAll = 0, kAttrVec = 1, kAttrOne = 2, kAttrVec3 = 3 };
template <int MODE>
__global__ void __launch_bounds__(256, MODE == kAttrVec ? 6 : (MODE == kAttrVec3 ? 3 : 4))
    attr_fused_kernel(AttrLaunch L, int64_t total_tiles) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  extern __shared__ float val[];
  __shared__ AttrDesc d;
  __shared__ AttrTileCtx tc;
  __shared__ int cur, changed;
  if (threadIdx.x == 0) cur = -1;
  __syncthreads();
  // the ring-buffered form: tiles of this CTA already requested (the
  // current one included) and the ring slot of the current one
  int ahead = 0;
  int head = 0;
  for (int64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
    if (threadIdx.x == 0) {
      // the descriptor search (parameter reads) only when the tile leaves
      // the current descriptor's range
      if (cur >= 0 && tile >= d.block_begin && tile < d.block_end) {
        changed = 0;
      } else {
      int di = 0;
#pragma unroll
      for (int i = 1; i < kAttrPerLaunch; ++i)
        if (i < L.n && L.d[i].block_begin <= tile) di = i;
      changed = di != cur;
      if (changed) {
        switch (di) {
#define SQC_ATTR_CASE(k) case k: d = L.d[k]; break;
          SQC_ATTR_CASE(0) SQC_ATTR_CASE(1) SQC_ATTR_CASE(2) SQC_ATTR_CASE(3) SQC_ATTR_CASE(4) SQC_ATTR_CASE(5)
          SQC_ATTR_CASE(6) SQC_ATTR_CASE(7) SQC_ATTR_CASE(8) SQC_ATTR_CASE(9) SQC_ATTR_CASE(10) SQC_ATTR_CASE(11)
          SQC_ATTR_CASE(12) SQC_ATTR_CASE(13) SQC_ATTR_CASE(14) SQC_ATTR_CASE(15)
#undef SQC_ATTR_CASE
          default: break;
        }
        cur = di;
      }
      }
    }
    __syncthreads();
    if (changed) {
      fill_tile_ctx(d, tc);
      __syncthreads();
    }
    if (MODE == kAttrOne) {
      attr_tile<false>(d, tc, tile - d.block_begin, val);
    } else if (d.async2) {
      // a ring of kAttrRing tile buffers: the CTA's next tiles of the same
      // subcircuit are requested (cp.async) before the current one is
      // expanded, so up to kAttrRing - 1 loads are in flight meanwhile
      const int64_t t = tile - d.block_begin;
      const int rows = (1 << (2 * d.kin)) << (kRingL1 + kRingL2);
      while (ahead < kAttrRing && tile + int64_t(ahead) * gridDim.x < d.block_end) {
        float* b = val + ((head + ahead) % kAttrRing) * rows;
        const int64_t ta = t + int64_t(ahead) * gridDim.x;
        ring_issue<kRingL1, kRingL2>(d, tc, ta, b);
        cp_async_commit();
        ++ahead;
      }
      // the current tile's group is complete once at most ahead - 1 remain
      if (ahead >= 3) cp_async_wait<2>();
      else if (ahead == 2) cp_async_wait<1>();
      else cp_async_wait<0>();
      __syncthreads();
      float* cur_buf = val + head * rows;
      ring_finish<kRingL1, kRingL2>(d, tc, t, cur_buf);
      head = (head + 1) % kAttrRing;
      --ahead;
    } else if (d.vec && d.kin == 0) {
      // (the host gives the 16 x 32 split to the double-buffered form only)
      attr_tiles_v4_kin0<5>(d, tile - d.block_begin, val);
    } else if (MODE == kAttrVec || MODE == kAttrVec3 || d.vec) {
      // (with incoming edges the host gives the 16 x 16 split)
      attr_tile_v4<4>(d, tc, tile - d.block_begin, val);
    } else {
      attr_tile<true>(d, tc, tile - d.block_begin, val);
    }
    __syncthreads();
  }
}

// One tile of the fused attribution + merge (AttrMergeDesc): phases 1-2 as
// attr_tile over the kept states x = zval | jl << z | xa << (z + L1) |
// jh << (n - L2), then every (row, active value) sums its 2^L2 merged
// slots in ascending order and writes T through the maps.
template <bool F64>
__device__ __forceinline__ void attr_merge_tile(const AttrMergeDesc& d, const AttrTileCtx& tc, int64_t t,
                                                float* val) {
  const uint64_t o = uint64_t(t) & ((uint64_t(1) << (2 * d.kout)) - 1);
  const uint64_t xa = uint64_t(t) >> (2 * d.kout);
  const int S = 1 << (2 * d.kin);
  const int L1 = d.L1, L2 = d.L2, lt = L1 + L2;
  const int TX = 1 << lt;
  const int n = d.n, z = d.z;
  const int step = int(blockDim.x) >> lt;
  uint64_t vbase = 0;
  uint32_t signed_mask = 0;
  for (int u = 0; u < d.kout; ++u) {
    const uint64_t dig = (o >> (2 * u)) & 3;
    vbase |= dig << d.outshift[u];
    if (dig) signed_mask |= 1u << u;
  }
  const int j = int(threadIdx.x) & (TX - 1);
  const uint64_t jl = uint64_t(j & ((1 << L1) - 1)), jh = uint64_t(j >> L1);
  const uint64_t x = uint64_t(d.zval) | (jl << z) | (xa << (z + L1)) | (jh << (n - L2));
  const int pos = slot_pos(j, L1, L2);
  if (F64 && d.in_f64) {
    switch (d.kout) {
      case 0: fold_phase<1, true>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
      case 1: fold_phase<2, true>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
      case 2: fold_phase<4, true>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
      default: fold_phase<8, true>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
    }
  } else {
    switch (d.kout) {
      case 0: fold_phase<1, false>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
      case 1: fold_phase<2, false>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
      case 2: fold_phase<4, false>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
      default: fold_phase<8, false>(d, tc, val, S, lt, x, pos, vbase, signed_mask); break;
    }
  }
  __syncthreads();
  for (int q = 0; q < d.kin; ++q) {
    const int lowmask = (1 << (2 * q)) - 1;
    const int st = TX << (2 * q);
    for (int g = int(threadIdx.x) >> lt; g < (S >> 2); g += step) {
      const int s0 = ((g & ~lowmask) << 2) | (g & lowmask);
      float* a = val + s0 * TX + pos;
      const float v0 = a[0], v1 = a[st], v2 = a[2 * st], v3 = a[3 * st];
      const float sum = v0 + v1;
      a[0] = sum;                 // I
      a[st] = 2.f * v2 - sum;     // X
      a[2 * st] = 2.f * v3 - sum; // Y
      a[3 * st] = v0 - v1;        // Z
    }
    __syncthreads();
  }
  // merge: the merged slots of (row s, active value jl), in ascending order
  const int na = 1 << L1, nm = 1 << L2;
  for (int idx = int(threadIdx.x); idx < (S << L1); idx += int(blockDim.x)) {
    const int s = idx >> L1, l = idx & (na - 1);
    const float* row = val + s * TX;
    float acc = 0.f;
    for (int h = 0; h < nm; ++h) acc += row[slot_pos(l | (h << L1), L1, L2)];
    const uint64_t e = in_digits(tc, s) | vbase;
    const uint32_t b = rev_bits(uint32_t(uint64_t(l) | (xa << L1)), d.a);
    store_out_f(d.dst, d.kind, d.plane_stride, d.rowmap[e] + d.colmap[b], acc * d.alpha);
  }
}

// Persistent over the tiles of up to kAttrPerLaunch subcircuits (the same
// walk as attr_fused_kernel).
template <bool F64>
__global__ void __launch_bounds__(256, 4) attr_merge_kernel(AttrMergeLaunch L, int64_t total_tiles) {
  // the first descriptor and tile context (parameters and shared memory
  // only) are set up before waiting on the previous kernel (programmatic
  // dependent launch); the variant outputs are read after the wait
  bool waited = false;
  extern __shared__ float val[];
  __shared__ AttrMergeDesc d;
  __shared__ AttrTileCtx tc;
  __shared__ int cur, changed, sdi;
  if (threadIdx.x == 0) cur = -1;
  __syncthreads();
  for (int64_t tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
    if (threadIdx.x == 0) {
      int di = 0;
#pragma unroll
      for (int i = 1; i < kAttrPerLaunch; ++i)
        if (i < L.n && L.d[i].block_begin <= tile) di = i;
      changed = di != cur;
      sdi = di;
      cur = di;
    }
    __syncthreads();
    if (changed) {
      // the descriptor copied by all threads at once (its parameter words
      // are fetched together), and its layout maps -- read at the end of
      // the tile, cold at the start of a step -- requested into L2 now
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&L.d[sdi]);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&d);
      for (int i = int(threadIdx.x); i < int(sizeof(AttrMergeDesc) / 8); i += int(blockDim.x)) dst[i] = src[i];
      __syncthreads();
      const int rows_lines = int(((int64_t(1) << (2 * (d.kin + d.kout))) + 15) >> 4);
      const int cols_lines = int(((int64_t(1) << d.a) + 15) >> 4);
      const int t = int(threadIdx.x);
      if (t < 64 && t < rows_lines) asm volatile("prefetch.global.L2 [%0];" ::"l"(d.rowmap + 16 * t));
      else if (t >= 64 && t < 128 && t - 64 < cols_lines) asm volatile("prefetch.global.L2 [%0];" ::"l"(d.colmap + 16 * (t - 64)));
      fill_tile_ctx(d, tc);
      __syncthreads();
    }
    if (!waited) {
      pdl_wait();      // the previous kernel on the stream has completed
      pdl_trigger();   // the next one may start launching
      waited = true;
    }
    attr_merge_tile<F64>(d, tc, tile - d.block_begin, val);
    __syncthreads();
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
  if (a.in_f64) return launch_k(fold_kernel<double>, dim3(grid_for(total)), dim3(256), 0, s, false, a);
  return launch_k(fold_kernel<float>, dim3(grid_for(total)), dim3(256), 0, s, false, a);
}

cudaError_t launch_attr_fused(const AttrLaunch& L, int64_t blocks, int smem_bytes, cudaStream_t s) {
  if (L.n <= 0 || blocks <= 0) return cudaSuccess;
  // persistent grid: exactly as many CTAs as are resident at once (limited
  // by registers and shared memory), so that no CTA's tile list starts
  // after the others have finished theirs
  // (function-local statics: initialised once, thread-safe)
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    return n;
  }();
  bool all_vec = true, all_one = true;
  for (int i = 0; i < L.n; ++i) {
    all_vec = all_vec && L.d[i].vec;
    all_one = all_one && !L.d[i].vec && !L.d[i].async2 && !L.d[i].in_f64;
  }
  const void* fn = all_vec   ? reinterpret_cast<const void*>(attr_fused_kernel<kAttrVec>)
                   : all_one ? reinterpret_cast<const void*>(attr_fused_kernel<kAttrOne>)
                             : reinterpret_cast<const void*>(attr_fused_kernel<kAttrAll>);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem_bytes) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  // shared memory already holds the launch to three CTAs per SM: the
  // variant with more registers costs no occupancy
  const bool vec3 = all_vec && per_sm <= 3;
  if (vec3 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, attr_fused_kernel<kAttrVec3>, 256, smem_bytes) !=
                   cudaSuccess || per_sm < 1))
    per_sm = 1;
  const int64_t grid = blocks < int64_t(sms) * per_sm ? blocks : int64_t(sms) * per_sm;
  const dim3 g(unsigned(grid), 1, 1);
  if (vec3) return launch_k(attr_fused_kernel<kAttrVec3>, g, dim3(256), size_t(smem_bytes), s, false, L, blocks);
  if (all_vec) return launch_k(attr_fused_kernel<kAttrVec>, g, dim3(256), size_t(smem_bytes), s, false, L, blocks);
  if (all_one) return launch_k(attr_fused_kernel<kAttrOne>, g, dim3(256), size_t(smem_bytes), s, false, L, blocks);
  return launch_k(attr_fused_kernel<kAttrAll>, g, dim3(256), size_t(smem_bytes), s, false, L, blocks);
}

namespace {
// Buffer blockIdx.y, CTAs along x striding over its 16-byte words, four
// loads in flight per thread before their stores.
__global__ void __launch_bounds__(256) stage_copy_kernel(StageCopy c) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  const int b = blockIdx.y;
  const uint4* src = static_cast<const uint4*>(c.src[b]);
  uint4* dst = static_cast<uint4*>(c.dst[b]);
  const uint64_t n = c.words[b];
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t w0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; w0 < n; w0 += 4 * stride) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (w0 + u * stride < n) v[u] = src[w0 + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (w0 + u * stride < n) dst[w0 + u * stride] = v[u];
  }
}
}  // namespace

cudaError_t launch_stage_copy(const StageCopy& c, cudaStream_t s) {
  if (c.n <= 0) return cudaSuccess;
  if (c.n > kAttrPerLaunch) return cudaErrorInvalidValue;
  uint64_t most = 0;
  for (int i = 0; i < c.n; ++i) most = c.words[i] > most ? c.words[i] : most;
  // enough CTAs per buffer for every SM to keep loads in flight
  const uint64_t per = (most + 4 * 256 - 1) / (4 * 256);
  const unsigned gx = unsigned(per < 608 ? (per > 0 ? per : 1) : 608);
  return launch_k(stage_copy_kernel, dim3(gx, unsigned(c.n)), dim3(256), 0, s, false, c);
}

int attr_merge_wave(bool f64, int smem_bytes) {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    return n;
  }();
  // per power of two of the shared memory (the tiles' sizes are powers of
  // two): computed once, read by any thread
  static std::atomic<int> cache[2][32];
  int lg = 0;
  while (lg < 31 && (1 << lg) < smem_bytes) ++lg;
  std::atomic<int>& slot = cache[f64 ? 1 : 0][lg];
  int per_sm = slot.load(std::memory_order_relaxed);
  if (per_sm <= 0) {
    const void* fn = f64 ? reinterpret_cast<const void*>(attr_merge_kernel<true>)
                         : reinterpret_cast<const void*>(attr_merge_kernel<false>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 1 << lg) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    slot.store(per_sm, std::memory_order_relaxed);
  }
  return sms * per_sm;
}

cudaError_t launch_attr_merge(const AttrMergeLaunch& L, int64_t blocks, int smem_bytes, cudaStream_t s) {
  if (L.n <= 0 || blocks <= 0) return cudaSuccess;
  bool any64 = false;
  for (int i = 0; i < L.n; ++i) any64 = any64 || L.d[i].in_f64;
  const int64_t wave = attr_merge_wave(any64, smem_bytes);
  const int64_t grid = blocks < wave ? blocks : wave;
  if (any64)
    return launch_k(attr_merge_kernel<true>, dim3(unsigned(grid)), dim3(256), size_t(smem_bytes), s, false, L, blocks);
  return launch_k(attr_merge_kernel<false>, dim3(unsigned(grid)), dim3(256), size_t(smem_bytes), s, false, L, blocks);
}

cudaError_t attr_configure() {
  cudaError_t e = cudaFuncSetAttribute(attr_fused_kernel<kAttrAll>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kAttrSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(attr_fused_kernel<kAttrVec>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAttrSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(attr_fused_kernel<kAttrOne>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAttrSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(attr_fused_kernel<kAttrVec3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAttrSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(attr_merge_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAttrSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(attr_merge_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAttrSmemMax);
  return e;
}

cudaError_t launch_mix(const MixArgs& a, cudaStream_t s) {
  const int64_t total = a.rows << a.n;
  return launch_k(mix_kernel, dim3(grid_for(total)), dim3(256), 0, s, false, a);
}

}  // namespace sqc
