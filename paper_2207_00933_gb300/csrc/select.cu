// Bin selection and the probability check.
//
// Algorithm 1 keeps the largest bins of each recursion ("append the largest
// bins ... sort and truncate").  Selection here is exact and deterministic:
// among the values >= threshold, the k largest, ordered by value descending
// and bin index ascending.
//
//  1. radix passes (8 bits per pass, most significant first) over
//     order-preserving 64-bit keys find the bucket that holds the k-th
//     largest key; each pass is one launch whose last CTA scans the
//     histogram, and the passes stop early (device-side flag) once that
//     bucket holds at most `cap` values;
//  2. compaction copies every value above the bucket and every value in it
//     to a candidate list;
//  3. if more than `cap` values share the exact k-th key, those ties are
//     taken in ascending bin order by an ordered block scan instead;
//  4. every candidate finds its rank in the final order by counting the
//     candidates ahead of it (many CTAs, shared-memory tiles) and the
//     first k are written at their ranks.
// The FP64 probability sum is a grid reduction with a fixed summation
// order (per-CTA partials added by the last CTA in CTA order).
#include <cmath>
#include <cstring>
#include <limits>
#include <mutex>

#include "device_ops.cuh"

namespace sqc {

namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kPasses = 8;          // 64-bit keys
constexpr int kSelThreads = 256;
constexpr int kMaxSort = 8192;      // candidates sorted in shared memory

// control block layout (unsigned long long words)
enum : int {
  ST_PREFIX = 0,     // determined high bits of the k-th key
  ST_BITS,           // how many high bits are determined
  ST_KREM,           // how many more to take from the current bucket
  ST_DONE,           // 0 = refining, 1 = bucket fits, 2 = take every filtered value, 3 = exact ties > cap
  ST_TAKE,           // number of bins to output: min(k, #values >= threshold)
  ST_NCAND,          // candidates written
  ST_COUNTER,        // last-CTA counter
  ST_WORDS = 8
};

__device__ __forceinline__ unsigned long long key_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned k = (u >> 31) ? ~u : (u | 0x80000000u);
  return (unsigned long long)k << 32;
}

__device__ __forceinline__ unsigned long long key_f64(double v) {
  const unsigned long long u = __double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ unsigned long long key_of(const void* x, int is_f64, uint64_t i, double* val) {
  if (is_f64) {
    const double v = static_cast<const double*>(x)[i];
    *val = v;
    return key_f64(v);
  }
  const float f = static_cast<const float*>(x)[i];
  *val = double(f);
  return key_f32(f);
}

// Values i0 .. i0+kVec-1 (fewer at the tail) with one or two vector loads,
// so that every thread keeps kVec independent loads in flight.  The
// threshold test is done on the order-preserving keys (integer compares,
// no FP64 pipe): ok = !isnan(v) && key(v) >= key_thr, where key_thr is the
// key of the smallest value of the input's type that is >= threshold.
constexpr int kVec = 4;
struct Chunk {
  unsigned long long key[kVec];
  bool ok[kVec];
  int cnt;
};

template <bool is_f64>
__device__ __forceinline__ void load_chunk(const void* x, int aligned, uint64_t n, uint64_t i0,
                                           unsigned long long key_thr, Chunk* c) {
  c->cnt = 0;
#pragma unroll
  for (int q = 0; q < kVec; ++q) {
    c->ok[q] = false;
    c->key[q] = 0ull;
  }
  if (i0 >= n) return;
  const int cnt = (n - i0 >= kVec) ? kVec : int(n - i0);
  c->cnt = cnt;
  if constexpr (is_f64) {
    const double* p = static_cast<const double*>(x) + i0;
    double v[kVec];
    if (aligned && cnt == kVec) {
      const double2 a = __ldg(reinterpret_cast<const double2*>(p));
      const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    } else {
      for (int q = 0; q < cnt; ++q) v[q] = p[q];
    }
#pragma unroll
    for (int q = 0; q < kVec; ++q) {
      const unsigned long long u = __double_as_longlong(v[q]);
      const bool nan = (u & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
      c->key[q] = key_f64(v[q]);
      c->ok[q] = q < cnt && !nan && c->key[q] >= key_thr;
    }
  } else {
    const float* p = static_cast<const float*>(x) + i0;
    float f[kVec];
    if (aligned && cnt == kVec) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p));
      f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
    } else {
      for (int q = 0; q < cnt; ++q) f[q] = p[q];
    }
#pragma unroll
    for (int q = 0; q < kVec; ++q) {
      const unsigned u = __float_as_uint(f[q]);
      const bool nan = (u & 0x7fffffffu) > 0x7f800000u;
      c->key[q] = key_f32(f[q]);
      c->ok[q] = q < cnt && !nan && c->key[q] >= key_thr;
    }
  }
}

// Add one digit per lane to a histogram in shared memory.  `sh` is this
// warp's private copy (kRadix counters), so lanes of other warps never
// contend; when every active lane has the same digit (the exponent bytes of
// probabilities) one lane adds the whole count.
__device__ __forceinline__ void warp_hist_add(unsigned* sh, bool ok, unsigned dig, int lane) {
  const unsigned active = __ballot_sync(0xffffffffu, ok);
  if (!active) return;
  const int leader = __ffs(active) - 1;
  const unsigned d0 = __shfl_sync(0xffffffffu, dig, leader);
  if (__all_sync(0xffffffffu, !ok || dig == d0)) {
    if (lane == leader) atomicAdd(&sh[d0], unsigned(__popc(active)));
    return;
  }
  if (ok) atomicAdd(&sh[dig], 1u);
}

template <bool is_f64>
__global__ void __launch_bounds__(kSelThreads)
radix_pass(const void* x, int aligned, uint64_t n, unsigned long long key_thr, int k, int pass,
           int last_pass, int cap, unsigned* hist_all, unsigned long long* st) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  __shared__ unsigned shw[kSelThreads / 32][kRadix];   // one histogram per warp
  unsigned* sh = shw[0];
  __shared__ bool is_last;
  if (st[ST_DONE] != 0) return;
  for (int d = threadIdx.x; d < kRadix * (kSelThreads / 32); d += blockDim.x) (&shw[0][0])[d] = 0;
  __syncthreads();
  const int shift = 64 - kRadixBits * (pass + 1);
  const unsigned long long prefix = st[ST_PREFIX];
  const int lane = threadIdx.x & 31;
  const uint64_t span = uint64_t(blockDim.x) * kVec;
  const uint64_t stride = uint64_t(gridDim.x) * span * 2;
  // the loop bound is uniform across the block, so whole warps iterate
  // together and can aggregate equal digits into one shared atomic; two
  // chunks per iteration keep 2 x kVec loads in flight per thread
  for (uint64_t base = uint64_t(blockIdx.x) * span * 2; base < n; base += stride) {
    Chunk c[2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
      load_chunk<is_f64>(x, aligned, n, base + h * span + uint64_t(threadIdx.x) * kVec, key_thr, &c[h]);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < kVec; ++q) {
        const unsigned long long key = c[h].key[q];
        const bool ok =
            c[h].ok[q] && (pass == 0 || (key >> (shift + kRadixBits)) == (prefix >> (shift + kRadixBits)));
        warp_hist_add(shw[threadIdx.x >> 5], ok, unsigned((key >> shift) & (kRadix - 1)), lane);
      }
  }
  __syncthreads();
  unsigned* hist = hist_all + pass * kRadix;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    unsigned v = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) v += shw[w][d];
    if (v) atomicAdd(&hist[d], v);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long t = atomicAdd(&st[ST_COUNTER], 1ull);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  // the last CTA: copy the global histogram (and re-arm it), then one warp
  // finds the digit holding the k-th largest value with a suffix scan
  __threadfence();
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
    sh[d] = static_cast<volatile unsigned*>(hist)[d];
    hist[d] = 0;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  constexpr int kPer = kRadix / 32;
  unsigned long long part = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) part += sh[lane * kPer + q];
  unsigned long long suf = part;              // sum over lanes >= this lane
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long t = __shfl_down_sync(0xffffffffu, suf, off);
    if (lane + off < 32) suf += t;
  }
  const unsigned long long total = __shfl_sync(0xffffffffu, suf, 0);
  const unsigned long long krem = (pass == 0) ? (unsigned long long)k : st[ST_KREM];
  if (pass == 0 && lane == 0) {
    st[ST_TAKE] = total < (unsigned long long)k ? total : (unsigned long long)k;
    if (total <= (unsigned long long)k) st[ST_DONE] = 2;
  }
  __syncwarp();
  const bool refine = !(pass == 0 && total <= (unsigned long long)k);
  // digits are scanned from the top: the k-th largest lies in the highest
  // lane whose suffix count reaches krem
  const unsigned reach = __ballot_sync(0xffffffffu, suf >= krem);
  const int L = reach ? 31 - __clz(reach) : 0;
  if (refine && lane == L) {
    unsigned long long cum = suf - part;
    int d = lane * kPer + kPer - 1;
    for (; d > lane * kPer; --d) {
      if (cum + sh[d] >= krem) break;
      cum += sh[d];
    }
    st[ST_PREFIX] = prefix | ((unsigned long long)d << shift);
    st[ST_BITS] = (unsigned long long)(kRadixBits * (pass + 1));
    st[ST_KREM] = krem - cum;
    if (sh[d] <= (unsigned)cap)
      st[ST_DONE] = 1;
    else if (last_pass)
      st[ST_DONE] = 3;
  }
  if (lane == 0) st[ST_COUNTER] = 0;
}

// Copy the values that are certainly selected, and the current bucket
// (unless it is an oversized group of exact ties), to the candidate list.
template <bool is_f64>
__global__ void __launch_bounds__(kSelThreads)
compact(const void* x, int aligned, uint64_t n, unsigned long long key_thr, unsigned long long* st,
        unsigned long long* ck, unsigned long long* ci) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  const unsigned long long done = st[ST_DONE];
  const int bits = int(st[ST_BITS]);
  const unsigned long long pv = bits ? (st[ST_PREFIX] >> (64 - bits)) : 0ull;
  const int lane = threadIdx.x & 31;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x * kVec;
  for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x * kVec; base < n; base += stride) {
    Chunk c;
    const uint64_t i0 = base + uint64_t(threadIdx.x) * kVec;
    load_chunk<is_f64>(x, aligned, n, i0, key_thr, &c);
#pragma unroll
    for (int q = 0; q < kVec; ++q) {
      bool take = false;
      if (c.ok[q]) {
        if (done == 2) {
          take = true;
        } else {
          const unsigned long long hb = c.key[q] >> (64 - bits);
          take = (done == 3) ? (hb > pv) : (hb >= pv);
        }
      }
      // one global atomic per warp
      const unsigned m = __ballot_sync(0xffffffffu, take);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long slot = 0;
        if (lane == leader) slot = atomicAdd(&st[ST_NCAND], (unsigned long long)__popc(m));
        slot = __shfl_sync(0xffffffffu, slot, leader);
        if (take) {
          const unsigned long long r = slot + __popc(m & ((1u << lane) - 1u));
          ck[r] = c.key[q];
          ci[r] = i0 + q;
        }
      }
    }
  }
}

// Exact ties beyond capacity: count them per contiguous range ...
__global__ void __launch_bounds__(kSelThreads)
tie_count(const void* x, int is_f64, uint64_t n, unsigned long long key_thr, const unsigned long long* st,
          unsigned* counts, uint64_t range) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  if (st[ST_DONE] != 3) return;
  __shared__ unsigned s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const unsigned long long tkey = st[ST_PREFIX];
  const uint64_t b = uint64_t(blockIdx.x) * range;
  const uint64_t e = (b + range < n) ? b + range : n;
  unsigned c = 0;
  for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    double v;
    const unsigned long long key = key_of(x, is_f64, i, &v);
    if (key >= key_thr && !isnan(v) && key == tkey) ++c;
  }
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// ... then append the first KREM of them in ascending bin order.
__global__ void __launch_bounds__(kSelThreads)
tie_write(const void* x, int is_f64, uint64_t n, unsigned long long key_thr, unsigned long long* st,
          const unsigned* counts, uint64_t range, unsigned long long* ck, unsigned long long* ci) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  if (st[ST_DONE] != 3) return;
  __shared__ unsigned long long base;
  __shared__ unsigned wsum[kSelThreads / 32];
  const unsigned long long tkey = st[ST_PREFIX];
  const unsigned long long need = st[ST_KREM];
  const unsigned long long first = st[ST_NCAND];   // after compact: the values above the ties
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (unsigned b = 0; b < blockIdx.x; ++b) s += counts[b];
    base = s;
  }
  __syncthreads();
  unsigned long long run = base;
  const uint64_t b0 = uint64_t(blockIdx.x) * range;
  const uint64_t e0 = (b0 + range < n) ? b0 + range : n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t t0 = b0; t0 < e0 && run < need; t0 += blockDim.x) {
    const uint64_t i = t0 + threadIdx.x;
    bool tie = false;
    if (i < e0) {
      double v;
      const unsigned long long key = key_of(x, is_f64, i, &v);
      tie = (key >= key_thr && !isnan(v) && key == tkey);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, tie);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, all = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      if (w < warp) before += wsum[w];
      all += wsum[w];
    }
    const unsigned long long rank = run + before + __popc(bal & ((1u << lane) - 1u));
    if (tie && rank < need) {
      ck[first + rank] = tkey;
      ci[first + rank] = i;
    }
    run += all;
    __syncthreads();
  }
}

// Place every candidate by its rank in the order (key descending, index
// ascending): rank = number of candidates that come before it.  The order
// is total (indices are distinct), so ranks are distinct; candidates whose
// rank is below TAKE are written out.  A CTA owns 32 candidates (one per
// lane); each of its warps counts against one slice of all candidates,
// read coalesced and broadcast by shuffles.  The last CTA re-arms the
// control block for the next call.
constexpr int kRankWarps = 8;
constexpr int kRankGrid = kMaxSort / 32;
__global__ void __launch_bounds__(32 * kRankWarps)
rank_emit(const void* x, int is_f64, unsigned long long* st, const unsigned long long* ck,
          const unsigned long long* ci, unsigned long long* bins_out, double* probs_out, int* n_found) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  __shared__ unsigned long long part[kRankWarps][32];
  __shared__ bool is_last;
  const unsigned long long done = st[ST_DONE];
  unsigned long long nc = st[ST_NCAND];
  if (done == 3) nc += st[ST_KREM];
  if (nc > kMaxSort) nc = kMaxSort;
  const unsigned long long take = st[ST_TAKE];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long me = uint64_t(blockIdx.x) * 32 + lane;
  if (uint64_t(blockIdx.x) * 32 < nc) {
    const bool have = me < nc;
    const unsigned long long mk = have ? ck[me] : 0ull, mi = have ? ci[me] : 0ull;
    const unsigned long long per = (nc + kRankWarps - 1) / kRankWarps;
    const unsigned long long j0 = per * warp, j1 = (j0 + per < nc) ? j0 + per : nc;
    unsigned long long rank = 0;
    for (unsigned long long jb = j0; jb < j1; jb += 32) {
      const unsigned long long j = jb + lane;
      const bool ok = j < j1;
      const unsigned long long kj = ok ? ck[j] : 0ull, ij = ok ? ci[j] : 0ull;
      const int m = int((j1 - jb) < 32 ? (j1 - jb) : 32);
      for (int r = 0; r < m; ++r) {
        const unsigned long long kr = __shfl_sync(0xffffffffu, kj, r);
        const unsigned long long ir = __shfl_sync(0xffffffffu, ij, r);
        rank += (kr > mk) || (kr == mk && ir < mi);
      }
    }
    part[warp][lane] = rank;
    __syncthreads();
    if (warp == 0 && have) {
      unsigned long long r = 0;
      for (int w = 0; w < kRankWarps; ++w) r += part[w][lane];
      if (r < take) {
        bins_out[r] = mi;
        probs_out[r] = is_f64 ? static_cast<const double*>(x)[mi] : double(static_cast<const float*>(x)[mi]);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long t = atomicAdd(&st[ST_COUNTER], 1ull);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    *n_found = int(take);
    for (int w = 0; w < ST_WORDS; ++w) st[w] = 0;   // re-arm for the next call
  }
}

__global__ void __launch_bounds__(kSelThreads)
sum_kernel(const void* x, int is_f64, uint64_t n, double* partials, unsigned* counter, double* total) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  __shared__ double red[kSelThreads / 32];
  double s = 0.0;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    s += is_f64 ? static_cast<const double*>(x)[i] : double(static_cast<const float*>(x)[i]);
  finish_total(s, partials, counter, total, red);
}

// Key of the smallest value of the input type that is >= thr (host side,
// same order-preserving transform as the kernels).
unsigned long long threshold_key(int is_f64, double thr) {
  if (is_f64) {
    unsigned long long u;
    std::memcpy(&u, &thr, 8);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
  }
  float f = float(thr);                       // round to nearest, then up if below
  if (double(f) < thr) f = std::nextafter(f, std::numeric_limits<float>::infinity());
  unsigned u;
  std::memcpy(&u, &f, 4);
  const unsigned k = (u >> 31) ? ~u : (u | 0x80000000u);
  return (unsigned long long)k << 32;
}

// Up to two CTAs per SM: every CTA adds its histogram into the global one
// with same-address atomics, so fewer, longer-lived CTAs are cheaper.
inline int vec_grid(uint64_t n) {
  uint64_t g = (n + uint64_t(kSelThreads) * kVec - 1) / (uint64_t(kSelThreads) * kVec);
  if (g < 1) g = 1;
  if (g > 152 * 2) g = 152 * 2;
  return int(g);
}

inline int stream_grid(uint64_t n, int max_blocks) {
  uint64_t g = (n + kSelThreads * 8 - 1) / (kSelThreads * 8);
  if (g < 1) g = 1;
  if (g > uint64_t(max_blocks)) g = max_blocks;
  return int(g);
}

}  // namespace

size_t select_work_bytes(int cap, int max_blocks) {
  const size_t ncand = size_t(kMaxSort);
  (void)cap;
  return sizeof(unsigned) * kPasses * kRadix + sizeof(unsigned long long) * ST_WORDS +
         2 * sizeof(unsigned long long) * ncand + sizeof(unsigned) * size_t(max_blocks) + 256;
}

void select_work_carve(void* base, int cap, int max_blocks, SelectWork* w) {
  char* p = static_cast<char*>(base);
  w->state = reinterpret_cast<unsigned*>(p);                       // ST_WORDS x u64
  p += sizeof(unsigned long long) * ST_WORDS;
  w->cand_key = reinterpret_cast<unsigned long long*>(p);
  p += sizeof(unsigned long long) * kMaxSort;
  w->cand_idx = reinterpret_cast<unsigned long long*>(p);
  p += sizeof(unsigned long long) * kMaxSort;
  w->hist = reinterpret_cast<unsigned*>(p);
  p += sizeof(unsigned) * kPasses * kRadix;
  w->tie_count = reinterpret_cast<unsigned*>(p);
  w->cap = cap;
  w->max_blocks = max_blocks;
}

// The work area must be zero before its first use; every call leaves it
// zeroed again (histograms and the control block are re-armed in-kernel).
cudaError_t launch_select(const SelectWork& w, const void* x, int is_f64, uint64_t n, int k, double threshold,
                          unsigned long long* bins_out, double* probs_out, int* n_found, cudaStream_t s) {
  if (k < 1 || k > kSelectMaxK) return cudaErrorInvalidValue;
  // bucket size at which refinement stops: the sort then sees <= k + cap values
  const int cap = (k > 512 ? k : 512) < kMaxSort - k ? (k > 512 ? k : 512) : kMaxSort - k;
  unsigned long long* st = reinterpret_cast<unsigned long long*>(w.state);
  const int aligned = (reinterpret_cast<uintptr_t>(x) % 16) == 0;
  const unsigned long long kt = threshold_key(is_f64, threshold);
  const int g = vec_grid(n);
  const int passes = is_f64 ? kPasses : 4;
  for (int p = 0; p < passes; ++p) {
    const int last = p == passes - 1;
    const cudaError_t e =
        is_f64 ? launch_k(radix_pass<true>, dim3(g), dim3(kSelThreads), 0, s, false, x, aligned, n, kt, k, p, last,
                          cap, w.hist, st)
               : launch_k(radix_pass<false>, dim3(g), dim3(kSelThreads), 0, s, false, x, aligned, n, kt, k, p, last,
                          cap, w.hist, st);
    if (e != cudaSuccess) return e;
  }
  {
    const cudaError_t e =
        is_f64 ? launch_k(compact<true>, dim3(g), dim3(kSelThreads), 0, s, false, x, aligned, n, kt, st, w.cand_key,
                          w.cand_idx)
               : launch_k(compact<false>, dim3(g), dim3(kSelThreads), 0, s, false, x, aligned, n, kt, st, w.cand_key,
                          w.cand_idx);
    if (e != cudaSuccess) return e;
  }
  const uint64_t range = (n + w.max_blocks - 1) / w.max_blocks;
  const unsigned tb = unsigned((n + range - 1) / (range ? range : 1));
  const uint64_t rng = range ? range : 1;
  const dim3 tg(tb ? tb : 1);
  cudaError_t e = launch_k(tie_count, tg, dim3(kSelThreads), 0, s, false, x, is_f64, n, kt, st, w.tie_count, rng);
  if (e == cudaSuccess)
    e = launch_k(tie_write, tg, dim3(kSelThreads), 0, s, false, x, is_f64, n, kt, st, w.tie_count, rng, w.cand_key,
                 w.cand_idx);
  if (e == cudaSuccess)
    e = launch_k(rank_emit, dim3(kRankGrid), dim3(32 * kRankWarps), 0, s, false, x, is_f64, st, w.cand_key,
                 w.cand_idx, bins_out, probs_out, n_found);
  return e;
}

namespace {

// ---- one cooperative launch ----------------------------------------------------
// The same selection as launch_select, as ONE cooperative kernel: the radix
// passes, the compaction, the (rare) ordered tie pass and the ranking are
// phases separated by grid barriers (bounded spins on a generation counter)
// instead of kernel launches.  Every CTA reads the global histogram after a
// barrier and derives the same radix state, so no CTA has to broadcast it.
constexpr int kCoopThreads = 256;
constexpr int kCoopWarps = kCoopThreads / 32;
constexpr uint32_t kBarrierLimit = 1u << 26;   // ~seconds of polling
constexpr int kCBits = 8;                      // radix digit width of the cooperative passes
constexpr int kCRadix = 1 << kCBits;
constexpr int kCPasses = 8;                    // 8 x 8 = 64 key bits
constexpr int kCSmem = kCoopWarps * kCRadix * 4;  // per-warp histograms
constexpr int kChunks = 4;                     // vector chunks in flight per thread
constexpr int kCopies = 1;                     // global histogram copies

struct CoopWork {
  unsigned* hist;                 // [kCPasses][kCopies][kCRadix]
  unsigned long long* ctl;        // [0] n_cand, [1] barrier count, [2] barrier generation, [3] abort
  unsigned long long* cand_key;   // [kMaxSort]
  unsigned long long* cand_idx;   // [kMaxSort]
  unsigned* rank;                 // [kMaxSort]
  unsigned* tie_count;            // [grid]
};

// Grid barrier: every CTA arrives on one counter, the last one bumps the
// generation the others poll (acquire loads, no sleep: a sleeping poller
// wakes late).  Measured on GB300: ~2.4 us per barrier for 152-304 CTAs, of
// which the same-address arrival chain is a small part; a two-level variant
// (16 group counters) measured ~4 us.  Bounded: gives up (abort flag) after
// kBarrierLimit polls.
__device__ __forceinline__ bool grid_barrier(unsigned long long* ctl, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned long long gen = static_cast<volatile unsigned long long*>(ctl)[2];
    __threadfence();
    if (atomicAdd(&ctl[1], 1ull) == nblocks - 1) {
      ctl[1] = 0ull;
      __threadfence();
      atomicAdd(&ctl[2], 1ull);
    } else {
      uint32_t i = 0;
      for (;;) {
        unsigned long long g;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(g) : "l"(ctl + 2) : "memory");
        if (g != gen) break;
        if (++i > kBarrierLimit || static_cast<volatile unsigned long long*>(ctl)[3]) {
          atomicExch(&ctl[3], 1ull);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// bits [lo, hi) of the key form the digit of pass p
__device__ __forceinline__ int pass_hi(int p) { return 64 - kCBits * p; }
__device__ __forceinline__ int pass_lo(int p) { const int l = 64 - kCBits * (p + 1); return l > 0 ? l : 0; }

template <bool is_f64>
__global__ void __launch_bounds__(kCoopThreads)
select_coop_kernel(const void* x, int aligned, uint64_t n, unsigned long long key_thr, int k, int cap,
                   CoopWork w, unsigned long long* bins_out, double* probs_out, int* n_found, int* err) {
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  extern __shared__ unsigned shw[];               // [kCoopWarps][kCRadix]
  __shared__ unsigned long long s_prefix, s_krem, s_take;
  __shared__ int s_bits, s_done;
  const unsigned nb = gridDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t gtid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t gthreads = uint64_t(nb) * blockDim.x;
  const int passes = is_f64 ? kCPasses : 4;       // FP32 keys hold 32 significant bits
  const uint64_t span = uint64_t(blockDim.x) * kVec;
  // (the histograms, ranks and candidate count start at zero: the previous
  // call cleared them on its way out, and the workspace starts zeroed)
  if (threadIdx.x == 0) {
    s_prefix = 0ull;
    s_krem = (unsigned long long)k;
    s_bits = 0;
    s_done = 0;
    s_take = 0ull;
  }
  __syncthreads();
  for (int pass = 0; pass < passes; ++pass) {
    const int hi = pass_hi(pass), lo = pass_lo(pass);
    const unsigned dmask = (1u << (hi - lo)) - 1u;
    const unsigned long long prefix = s_prefix;
    for (int d = threadIdx.x; d < kCoopWarps * kCRadix; d += blockDim.x) shw[d] = 0;
    __syncthreads();
    unsigned* mine = shw + warp * kCRadix;
    for (uint64_t base = uint64_t(blockIdx.x) * span * kChunks; base < n; base += uint64_t(nb) * span * kChunks) {
      Chunk c[kChunks];
#pragma unroll
      for (int h = 0; h < kChunks; ++h)
        load_chunk<is_f64>(x, aligned, n, base + h * span + uint64_t(threadIdx.x) * kVec, key_thr, &c[h]);
#pragma unroll
      for (int h = 0; h < kChunks; ++h)
#pragma unroll
        for (int q = 0; q < kVec; ++q) {
          const unsigned long long key = c[h].key[q];
          const bool ok = c[h].ok[q] && (pass == 0 || (key >> hi) == (prefix >> hi));
          warp_hist_add(mine, ok, unsigned(key >> lo) & dmask, lane);
        }
    }
    __syncthreads();
    unsigned* hist = w.hist + size_t(pass) * kCopies * kCRadix;
    unsigned* my_copy = hist + (blockIdx.x % kCopies) * kCRadix;
    for (int d = threadIdx.x; d < kCRadix; d += blockDim.x) {
      unsigned v = 0;
      for (int ww = 0; ww < kCoopWarps; ++ww) v += shw[ww * kCRadix + d];
      if (v) atomicAdd(&my_copy[d], v);
    }
    if (!grid_barrier(w.ctl, nb)) goto fail;
    __syncthreads();
    for (int d = threadIdx.x; d < kCRadix; d += blockDim.x) {
      unsigned v = 0;
      for (int cpy = 0; cpy < kCopies; ++cpy) v += static_cast<volatile unsigned*>(hist)[cpy * kCRadix + d];
      shw[d] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      constexpr int kPer = kCRadix / 32;
      unsigned long long part = 0;
      for (int q = 0; q < kPer; ++q) part += shw[lane * kPer + q];
      unsigned long long suf = part;
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, suf, off);
        if (lane + off < 32) suf += t;
      }
      const unsigned long long total = __shfl_sync(0xffffffffu, suf, 0);
      const unsigned long long krem = s_krem;
      bool refine = true;
      if (pass == 0) {
        if (lane == 0) s_take = total < (unsigned long long)k ? total : (unsigned long long)k;
        if (total <= (unsigned long long)k) {
          refine = false;
          if (lane == 0) s_done = 2;
        }
      }
      const unsigned reach = __ballot_sync(0xffffffffu, suf >= krem);
      const int L = reach ? 31 - __clz(reach) : 0;
      if (refine && lane == L) {
        unsigned long long cum = suf - part;
        int d = lane * kPer + kPer - 1;
        for (; d > lane * kPer; --d) {
          if (cum + shw[d] >= krem) break;
          cum += shw[d];
        }
        s_prefix = prefix | ((unsigned long long)d << lo);
        s_bits = 64 - lo;
        s_krem = krem - cum;
        if (shw[d] <= (unsigned)cap) s_done = 1;
        else if (pass == passes - 1) s_done = 3;
      }
    }
    __syncthreads();
    if (s_done) break;
  }
  {
    // compaction: values certainly selected, plus the bucket unless it is an
    // oversized group of exact ties
    const int done = s_done, bits = s_bits;
    const unsigned long long pv = bits ? (s_prefix >> (64 - bits)) : 0ull;
    for (uint64_t base = uint64_t(blockIdx.x) * span * kChunks; base < n; base += uint64_t(nb) * span * kChunks) {
      Chunk c[kChunks];
#pragma unroll
      for (int h = 0; h < kChunks; ++h)
        load_chunk<is_f64>(x, aligned, n, base + h * span + uint64_t(threadIdx.x) * kVec, key_thr, &c[h]);
#pragma unroll
      for (int h = 0; h < kChunks; ++h)
#pragma unroll
        for (int q = 0; q < kVec; ++q) {
          bool take = false;
          if (c[h].ok[q]) {
            if (done == 2) {
              take = true;
            } else {
              const unsigned long long hb = c[h].key[q] >> (64 - bits);
              take = (done == 3) ? (hb > pv) : (hb >= pv);
            }
          }
          const unsigned m = __ballot_sync(0xffffffffu, take);
          if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long slot = 0;
            if (lane == leader) slot = atomicAdd(&w.ctl[0], (unsigned long long)__popc(m));
            slot = __shfl_sync(0xffffffffu, slot, leader);
            if (take) {
              const unsigned long long r = slot + __popc(m & ((1u << lane) - 1u));
              w.cand_key[r] = c[h].key[q];
              w.cand_idx[r] = base + h * span + uint64_t(threadIdx.x) * kVec + q;
            }
          }
        }
    }
    if (!grid_barrier(w.ctl, nb)) goto fail;
    if (done == 3) {
      // exact ties beyond capacity, taken in ascending bin order: count per
      // contiguous range, barrier, then an ordered block scan per range
      const unsigned long long tkey = s_prefix, need = s_krem;
      const uint64_t range = (n + nb - 1) / nb;
      const uint64_t b0 = uint64_t(blockIdx.x) * range;
      const uint64_t e0 = (b0 + range < n) ? b0 + range : n;
      __shared__ unsigned cnt;
      __shared__ unsigned wsum[kCoopWarps];
      if (threadIdx.x == 0) cnt = 0;
      __syncthreads();
      unsigned my = 0;
      for (uint64_t i = b0 + threadIdx.x; i < e0; i += blockDim.x) {
        double v;
        const unsigned long long key = key_of(x, is_f64, i, &v);
        if (key >= key_thr && !isnan(v) && key == tkey) ++my;
      }
      atomicAdd(&cnt, my);
      __syncthreads();
      if (threadIdx.x == 0) w.tie_count[blockIdx.x] = cnt;
      const unsigned long long first = static_cast<volatile unsigned long long*>(w.ctl)[0];
      if (!grid_barrier(w.ctl, nb)) goto fail;
      __shared__ unsigned long long tbase;
      if (threadIdx.x == 0) {
        unsigned long long sacc = 0;
        for (unsigned b = 0; b < blockIdx.x; ++b) sacc += static_cast<volatile unsigned*>(w.tie_count)[b];
        tbase = sacc;
      }
      __syncthreads();
      unsigned long long run = tbase;
      for (uint64_t t0 = b0; t0 < e0 && run < need; t0 += blockDim.x) {
        const uint64_t i = t0 + threadIdx.x;
        bool tie = false;
        if (i < e0) {
          double v;
          const unsigned long long key = key_of(x, is_f64, i, &v);
          tie = (key >= key_thr && !isnan(v) && key == tkey);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, tie);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        unsigned before = 0, all = 0;
        for (int ww = 0; ww < kCoopWarps; ++ww) {
          if (ww < warp) before += wsum[ww];
          all += wsum[ww];
        }
        const unsigned long long rank = run + before + __popc(bal & ((1u << lane) - 1u));
        if (tie && rank < need) {
          w.cand_key[first + rank] = tkey;
          w.cand_idx[first + rank] = i;
        }
        run += all;
        __syncthreads();
      }
      if (!grid_barrier(w.ctl, nb)) goto fail;
    }
  }
  {
    // ranking: every warp of the grid takes one (group of 32 candidates,
    // slice of all candidates) pair and adds its count to the candidates'
    // ranks; the order (key desc, index asc) is total, so ranks are distinct
    unsigned long long nc = static_cast<volatile unsigned long long*>(w.ctl)[0];
    if (s_done == 3) nc += s_krem;
    if (nc > kMaxSort) nc = kMaxSort;
    const unsigned long long groups = (nc + 31) / 32;
    const uint64_t warps = gthreads / 32;
    const uint64_t gw = gtid / 32;
    const uint64_t slices = groups ? (warps / groups > 0 ? warps / groups : 1) : 1;
    for (uint64_t task = gw; task < groups * slices; task += warps) {
      const uint64_t g = task / slices, sl = task % slices;
      const unsigned long long me = g * 32 + lane;
      const bool have = me < nc;
      const unsigned long long mk = have ? w.cand_key[me] : 0ull, mi = have ? w.cand_idx[me] : 0ull;
      const unsigned long long per = (nc + slices - 1) / slices;
      const unsigned long long j0 = per * sl, j1 = (j0 + per < nc) ? j0 + per : nc;
      unsigned cntr = 0;
      for (unsigned long long jb = j0; jb < j1; jb += 32) {
        const unsigned long long j = jb + lane;
        const bool ok = j < j1;
        const unsigned long long kj = ok ? w.cand_key[j] : 0ull, ij = ok ? w.cand_idx[j] : 0ull;
        const int m = int((j1 - jb) < 32 ? (j1 - jb) : 32);
        for (int r = 0; r < m; ++r) {
          const unsigned long long kr = __shfl_sync(0xffffffffu, kj, r);
          const unsigned long long ir = __shfl_sync(0xffffffffu, ij, r);
          cntr += (kr > mk) || (kr == mk && ir < mi);
        }
      }
      if (have && cntr) atomicAdd(&w.rank[me], cntr);
    }
    if (!grid_barrier(w.ctl, nb)) goto fail;
    const unsigned long long take = s_take;
    for (uint64_t i = gtid; i < nc; i += gthreads) {
      const unsigned r = w.rank[i];
      w.rank[i] = 0u;                              // cleared for the next call
      if (r < take) {
        const unsigned long long b = w.cand_idx[i];
        bins_out[r] = b;
        probs_out[r] = is_f64 ? static_cast<const double*>(x)[b] : double(static_cast<const float*>(x)[b]);
      }
    }
    if (gtid == 0) *n_found = int(take);
  }
  // every CTA has read the histograms and the candidate count by now (the
  // ranking barrier); clear them for the next call
  for (uint64_t i = gtid; i < uint64_t(kCPasses) * kCopies * kCRadix; i += gthreads) w.hist[i] = 0u;
  if (gtid == 0) w.ctl[0] = 0ull;
  return;
fail:
  if (threadIdx.x == 0 && err) atomicExch(err, 1);
}


// ---- shared-memory-resident cooperative selection --------------------------------
// For inputs that fit in the shared memory of one CTA per SM (the usual
// recursion level: 2^20 FP32 bins are 27 KB per SM).  Every CTA loads its
// contiguous slice ONCE, as keys, into shared memory and builds the first
// 12-bit histogram on the way; the refinement passes, the compaction and
// the tie scan then read shared memory only.  Grid barriers are a
// monotonic arrival counter (one release-add per CTA, acquire polling, no
// last-arriver step).  The ranking needs no barrier (rank_candidates):
// every CTA groups the candidate list by log-scaled key buckets in shared
// memory, and a warp per owned candidate counts the members of its bucket
// ahead of it.  Control flow is uniform across CTAs
// (every CTA derives the same decisions from the same global histograms),
// so every CTA meets every barrier.
constexpr int kRThreads = 1024;
constexpr int kRWarps = kRThreads / 32;
constexpr int kRBits = 12;
constexpr int kRRadix = 1 << kRBits;
constexpr int kRMaxPasses = 6;                      // 64-bit keys: 5 x 12 + 4 bits
constexpr int kRHistBytes = kRRadix * 4;
constexpr int kRRegionMin = 16 * 1024;              // shared memory after the histogram at least
constexpr int kRSmemMax = 200 * 1024;               // dynamic shared memory per CTA at most
constexpr size_t kRCtlOffset = 128;                 // byte offset of this kernel's control words
constexpr uint32_t kRBarrierLimit = 1u << 21;       // polls (~1-2 s) before a barrier gives up

struct ResWork {
  // [0] barrier word: arrivals (high 32 bits) and candidates (low 32 bits,
  // added at the compaction barrier); [1] exits; [2] abort; [3] slots
  unsigned long long* ctl;
  unsigned* hist;                 // [kRMaxPasses][kRRadix]
  unsigned long long* cand_key;   // [kMaxSort]
  unsigned long long* cand_idx;   // [kMaxSort]
  unsigned* tie_count;            // [grid]
};

// Arrive with `add` (1 << 32 plus any count for the low word) and wait
// until `arrivals` CTAs have arrived; returns the barrier word seen (0 after
// an abort).  The release-add publishes the CTA's writes (ordered before it
// by the CTA barrier), the acquire poll makes the others' visible.
__device__ __forceinline__ unsigned long long res_barrier(unsigned long long* ctl, unsigned long long add,
                                                          unsigned arrivals) {
  __shared__ unsigned long long seen;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(ctl), "l"(add) : "memory");
    uint32_t i = 0;
    for (;;) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctl) : "memory");
      if ((v >> 32) >= arrivals) {
        seen = v;
        break;
      }
      if (++i > kRBarrierLimit || static_cast<volatile unsigned long long*>(ctl)[2]) {
        atomicExch(ctl + 2, 1ull);
        seen = 0ull;
        break;
      }
    }
  }
  __syncthreads();
  return seen;
}

// Decision after a pass: over the pass's global histogram, the digit
// holding the krem-th largest in-scope key is found with a block-wide
// suffix scan (4 bins per thread, one 16-byte load each).  Writes the
// shared decision words; identical in every CTA.
struct ResState {
  unsigned long long prefix;  // determined key bits (as a 64-bit value)
  unsigned long long krem;    // how many to take from the current bucket
  unsigned long long take;    // min(k, values >= threshold)
  int lo;                     // bits below lo are undetermined
  int done;                   // 0 refine, 1 bucket fits, 2 take every value, 3 exact ties > cap
};

__device__ __forceinline__ void res_decide(const unsigned* ghist, int pass, int lo, bool last_pass,
                                           int k, int cap, ResState* st, unsigned long long* wtot) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint4 q4 = __ldcg(reinterpret_cast<const uint4*>(ghist) + t);
  const unsigned v[4] = {q4.x, q4.y, q4.z, q4.w};
  const unsigned long long s = (unsigned long long)v[0] + v[1] + v[2] + v[3];
  // suffix sums over threads: inclusive within the warp from the top lane,
  // then over the warp totals by warp 0
  unsigned long long inc = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, inc, off);
    if (lane + off < 32) inc += o;
  }
  if (lane == 0) wtot[warp] = inc;
  const unsigned long long krem = pass == 0 ? (unsigned long long)k : st->krem;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long mine = wtot[lane];
    unsigned long long suf = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long o = __shfl_down_sync(0xffffffffu, suf, off);
      if (lane + off < 32) suf += o;
    }
    wtot[32 + lane] = suf - mine;                   // keys in the warps above
    if (lane == 0) wtot[64] = suf;                  // all keys in scope
  }
  __syncthreads();
  const unsigned long long total = wtot[64];
  const unsigned long long above = wtot[32 + warp] + inc - s;   // keys in bins above this thread's four
  if (pass == 0 && t == 0) {
    st->take = total < (unsigned long long)k ? total : (unsigned long long)k;
    if (total <= (unsigned long long)k) st->done = 2;
  }
  if (!(pass == 0 && total <= (unsigned long long)k) && above < krem && above + s >= krem) {
    unsigned long long cum = above;
    int j = 3;
    for (; j > 0; --j) {
      if (cum + v[j] >= krem) break;
      cum += v[j];
    }
    st->prefix |= (unsigned long long)(4 * t + j) << lo;
    st->krem = krem - cum;
    st->lo = lo;
    if (v[j] <= unsigned(cap)) st->done = 1;
    else if (last_pass) st->done = 3;
  }
  __syncthreads();
}

// The value a key was made from (the key transform is a bijection).
template <bool F64>
__device__ __forceinline__ double value_of_key(unsigned long long key) {
  if constexpr (F64) {
    const unsigned long long u = (key >> 63) ? (key & 0x7fffffffffffffffull) : ~key;
    return __longlong_as_double((long long)u);
  } else {
    const unsigned k32 = unsigned(key);
    const unsigned u = (k32 >> 31) ? (k32 & 0x7fffffffu) : ~k32;
    return double(__uint_as_float(u));
  }
}

// Sum of the (hi, lo) pairs of a warp, in every lane (butterfly order).
__device__ __forceinline__ void pair_warp_sum(float& h, float& l) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, off);
    const float l2 = __shfl_xor_sync(0xffffffffu, l, off);
    l += l2;
    two_sum_add(h, l, h2);
  }
}

// Bits of b taken run by run (TailPext) and packed into an index (bins
// held in shared memory number fewer than 2^32).
__device__ __forceinline__ uint32_t tail_pext(uint32_t b, const TailPext& r) {
  uint32_t v = 0;
  for (int t = 0; t < r.n; ++t) v |= ((b >> r.pos[t]) & ((1u << r.len[t]) - 1u)) << r.out[t];
  return v;
}

// Shared memory a tile of the steps before the last needs (the largest of
// the three tile shapes: 32 x 32 with 64-deep stages).
constexpr int kTailStageBytes = 64 * (32 + 4) * 2 * 4;
static_assert(kTailStageBytes >= 32 * (64 + 4) * 2 * 4 && kTailStageBytes >= 16 * (128 + 4) * 2 * 4,
              "stage region of the 64 x 64 and 128 x 128 tiles");

// Offset of the staged Y operand in the fused launch's shared memory.
__host__ __device__ __forceinline__ uint64_t tail_y_offset(uint64_t per) {
  uint64_t r = per * 4;
  if (r < uint64_t(kRRegionMin)) r = kRRegionMin;
  if (r < uint64_t(kTailStageBytes)) r = kTailStageBytes;
  return uint64_t(kRHistBytes) + ((r + 15) & ~uint64_t(15));
}

// The contraction steps before the last, level by level: every CTA takes
// tiles of the level's steps (the whole CTA on one tile), then all meet at
// a grid barrier, so the next level reads complete tensors.  Returns false
// when a barrier gave up.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The larger tile shapes of the steps before the last, kept out of line:
// the fused launch is long and its straight-line path should stay compact
// in the instruction cache.
template <int BM, int TMN, int BK>
__device__ __noinline__ void tail_tile_apart(const GemmArgs& a, int64_t m0, int64_t n0, float* stage) {
  gemm_tile<BM, BM, TMN, TMN, false, BK, kRThreads, true>(a, m0, n0, stage, stage + BK * (BM + 4), a.C);
}

// A 32 x 32 tile of an FP32 step with K <= 64 on the whole CTA, one output
// per thread: both operand tiles and the output's two layout-map entries
// are loaded in one round (the general tile loads A, then B, then reads the
// maps in its epilogue: three dependent round trips).  The multiply-adds
// run over k = 0..63 ascending with zeros past K, as the general tile with
// a 64-deep stage does, so the values are the same bit for bit.
__device__ __forceinline__ void tail_tile32(const GemmArgs& a, int64_t m0, int64_t n0, float* stage) {
  static_assert(kRThreads == 1024, "one output per thread");
  float (*As)[32 + 4] = reinterpret_cast<float (*)[32 + 4]>(stage);
  float (*Bs)[32 + 4] = reinterpret_cast<float (*)[32 + 4]>(stage + 64 * (32 + 4));
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  float ra[2], rb[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int idx = tid + u * kRThreads;
    const int r = idx >> 6, kk = idx & 63;
    ra[u] = (m0 + r < a.M && kk < a.K) ? __ldcg(a.A + (m0 + r) * a.K + kk) : 0.f;
    rb[u] = (n0 + r < a.N && kk < a.K) ? __ldcg(a.B + (n0 + r) * a.K + kk) : 0.f;
  }
  const int64_t row = m0 + ty, col = n0 + tx;
  const bool in = row < a.M && col < a.N;
  uint64_t off = 0;
  if (in) off = __ldg(a.rowmap + row) + __ldg(a.colmap + col);
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int idx = tid + u * kRThreads;
    As[idx & 63][idx >> 6] = ra[u];
    Bs[idx & 63][idx >> 6] = rb[u];
  }
  __syncthreads();
  float acc = 0.f;
#pragma unroll
  for (int kk = 0; kk < 64; ++kk) acc = fmaf(As[kk][ty], Bs[kk][tx], acc);
  __syncthreads();
  if (in) {
    const float v = acc * pow2_to_float(a.alpha);
    float* dst = static_cast<float*>(a.C) + off;
    *dst = a.accumulate ? *dst + v : v;
  }
}

__device__ __forceinline__ bool tail_pre_steps(const TailArgs& T, ResWork& w, unsigned nb, unsigned& bar,
                                              float* stage) {
  int lb = 0;
  for (int l = 0; l < T.n_levels; ++l) {
    const int le = T.level_end[l];
    int64_t tot = 0;
    for (int s = lb; s < le; ++s) tot += T.pre[s].ntiles;
    for (int64_t t = blockIdx.x; t < tot; t += nb) {
      int s = lb;
      int64_t tl = t;
      while (tl >= T.pre[s].ntiles) {
        tl -= T.pre[s].ntiles;
        ++s;
      }
      const TailStep& ts = T.pre[s];
      const GemmArgs& a = ts.a;
      const int bshift = 5 + ts.cfg;                       // tile edge 32, 64 or 128
      const int64_t m0 = (tl >> ts.tn_shift) << bshift;
      const int64_t n0 = (tl & ((int64_t(1) << ts.tn_shift) - 1)) << bshift;
      {
        // this tile's layout maps (cold at the start of a step) into L2
        // while its operands load: 16 entries per 128-byte line
        const int64_t r = int64_t(threadIdx.x) * 16, bm = int64_t(1) << bshift;
        if (r < bm && m0 + r < a.M) prefetch_l2(a.rowmap + m0 + r);
        else if (r >= 128 && r - 128 < bm && n0 + r - 128 < a.N) prefetch_l2(a.colmap + n0 + r - 128);
      }
      // operands may come from the level before (written in this launch):
      // read them from L2.  Each stage of gemm_tile ends with a CTA
      // barrier, so the next tile may reuse the shared memory at once.
      if (ts.cfg == 0 && a.K <= 64 && a.kind == OUT_F32)
        tail_tile32(a, m0, n0, stage);
      else if (ts.cfg == 0)
        gemm_tile<32, 32, 1, 1, false, 64, kRThreads, true>(a, m0, n0, stage, stage + 64 * (32 + 4), a.C);
      else if (ts.cfg == 1)
        tail_tile_apart<64, 2, 32>(a, m0, n0, stage);
      else
        tail_tile_apart<128, 4, 16>(a, m0, n0, stage);
    }
    lb = le;
    if (res_barrier(w.ctl, 1ull << 32, nb * ++bar) == 0ull) return false;
  }
  return true;
}

// Bins of a slice for any bit layout of the last step (one bin per thread
// and round: bit runs, Y staged, X staged or read from L2), with their keys
// and the first 12-bit histogram.  Out of line: the fused launch's common
// layout takes the band path.
__device__ __noinline__ void tail_slice_general(const TailArgs& T, const float* ys, const float* xs, uint32_t x0,
                                                bool xst, uint32_t ustart, int cnt, unsigned key_thr,
                                                unsigned* keys, unsigned* sh, float& s_hi, float& s_lo) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int kd = T.Kd;
  const int kd_log2 = __ffs(kd) - 1;
  const int ystride = T.ystride;
  const bool runs1 = T.rows.n <= 1 && T.cols.n <= 1;
  const uint32_t rpos = T.rows.n ? T.rows.pos[0] : 0u, rmask = T.rows.n ? (1u << T.rows.len[0]) - 1u : 0u;
  const uint32_t cpos = T.cols.n ? T.cols.pos[0] : 0u, cmask = T.cols.n ? (1u << T.cols.len[0]) - 1u : 0u;
  const float alpha = T.alpha;
  float* P = T.P;
  // the loop bound is the same for the whole CTA (warp_hist_add)
  for (int i0 = 0; i0 < cnt; i0 += kRThreads) {
    const int i = i0 + tid;
    unsigned kv = 0u;
    if (i < cnt) {
      const uint32_t b = ustart + uint32_t(i);
      uint32_t r, c;
      if (runs1) {
        r = (b >> rpos) & rmask;
        c = (b >> cpos) & cmask;
      } else {
        r = tail_pext(b, T.rows);
        c = tail_pext(b, T.cols);
      }
      float acc = 0.f;
      if (kd >= 4) {
        const float4* yr = reinterpret_cast<const float4*>(ys + c * ystride);
        if (xst) {
          const float4* xr = reinterpret_cast<const float4*>(xs + (r - x0) * ystride);
#pragma unroll 4
          for (int q = 0; q < (kd >> 2); ++q) {
            const float4 xa = xr[q], yb = yr[q];
            acc = fmaf(xa.x, yb.x, acc);
            acc = fmaf(xa.y, yb.y, acc);
            acc = fmaf(xa.z, yb.z, acc);
            acc = fmaf(xa.w, yb.w, acc);
          }
        } else {
          const float4* xr = reinterpret_cast<const float4*>(T.X + (size_t(r) << kd_log2));
#pragma unroll 4
          for (int q = 0; q < (kd >> 2); ++q) {
            const float4 xa = __ldcg(xr + q), yb = yr[q];
            acc = fmaf(xa.x, yb.x, acc);
            acc = fmaf(xa.y, yb.y, acc);
            acc = fmaf(xa.z, yb.z, acc);
            acc = fmaf(xa.w, yb.w, acc);
          }
        }
      } else {
        const float xv = xst ? xs[(r - x0) * ystride] : __ldcg(T.X + r);
        acc = fmaf(xv, ys[c * ystride], acc);
      }
      // the per-step kernel pads a shared index below 16 with zero terms
      // (which turn -0 into +0)
      if (kd < 16) acc = fmaf(0.f, 0.f, acc);
      const float v = acc * alpha;
      P[b] = v;
      two_sum_add(s_hi, s_lo, v);
      const unsigned u = __float_as_uint(v);
      const bool nan = (u & 0x7fffffffu) > 0x7f800000u;
      const unsigned kk = unsigned(key_f32(v) >> 32);
      kv = (!nan && kk >= key_thr) ? kk : 0u;
      keys[i] = kv;
    }
    warp_hist_add(sh, kv != 0, kv >> (32 - kRBits), lane);
  }
}

// Exact ties of the k-th key beyond the candidate capacity (rare): written
// in ascending bin order via per-CTA counts and an ordered scan of each
// slice, after every larger value.  Out of line, like the other rare paths
// of the resident kernel, to keep its common path compact in the
// instruction cache.  Returns false when the grid barrier gave up.
template <bool F64>
__device__ __noinline__ bool tie_scan(ResWork& w, const unsigned* keys, int cnt, uint64_t start, const void* x,
                                      const ResState& st, unsigned* wcnt, unsigned nb, unsigned& bar) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long tkey = st.prefix;
  const unsigned tk_hi = F64 ? unsigned(tkey >> 32) : unsigned(tkey);
  auto is_tie = [&](int i, unsigned kk) -> bool {
    if (kk != tk_hi) return false;
    if constexpr (F64) return unsigned(key_f64(static_cast<const double*>(x)[start + i])) == unsigned(tkey);
    else return true;
  };
  unsigned my = 0;
  for (int i = tid; i < cnt; i += kRThreads) my += is_tie(i, keys[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) my += __shfl_down_sync(0xffffffffu, my, off);
  if (lane == 0) wcnt[warp] = my;
  __syncthreads();
  if (tid == 0) {
    unsigned c = 0;
    for (int ww = 0; ww < kRWarps; ++ww) c += wcnt[ww];
    w.tie_count[blockIdx.x] = c;
  }
  if (res_barrier(w.ctl, 1ull << 32, nb * ++bar) == 0ull) return false;
  __shared__ unsigned long long tbase;
  if (tid == 0) {
    unsigned long long b = 0;
    for (unsigned r = 0; r < blockIdx.x; ++r) b += __ldcg(w.tie_count + r);
    tbase = b;
  }
  __syncthreads();
  const unsigned long long need = st.krem, first = st.take - st.krem;
  unsigned long long run = tbase;
  for (int i0 = 0; i0 < cnt && run < need; i0 += kRThreads) {
    const int i = i0 + tid;
    const bool tie = i < cnt && is_tie(i, keys[i]);
    const unsigned bal = __ballot_sync(0xffffffffu, tie);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, all = 0;
    for (int ww = 0; ww < kRWarps; ++ww) {
      if (ww < warp) before += wcnt[ww];
      all += wcnt[ww];
    }
    const unsigned long long rank = run + before + __popc(bal & ((1u << lane) - 1u));
    if (tie && rank < need) {
      w.cand_key[first + rank] = tkey;
      w.cand_idx[first + rank] = start + i;
    }
    run += all;
    __syncthreads();
  }
  return true;
}

// Bucket of a candidate key for the ranking: a monotone, log-scaled
// function of its distance d = key - tmin above the lowest selectable key
// (the leading-one position of d and the 7 (FP32) or 6 (FP64) bits after
// it), numbered so that bucket 0 holds the largest keys.  Fine steps near
// the selection boundary, where most candidates lie.
template <bool F64>
__device__ __forceinline__ unsigned rank_bucket(unsigned long long key, unsigned long long tmin) {
  const unsigned long long d = key - tmin;
  int val = 0;
  if (d != 0) {
    if constexpr (F64) {
      const int lz = __clzll(static_cast<long long>(d));
      val = 1 + ((63 - lz) << 6) + int(unsigned((d << lz) >> 57) & 63u);
    } else {
      const unsigned d32 = unsigned(d);
      const int lz = __clz(d32);
      val = 1 + ((31 - lz) << 7) + int(((d32 << lz) >> 24) & 127u);
    }
  }
  if (val > kRRadix - 1) val = kRRadix - 1;
  return unsigned(kRRadix - 1 - val);
}

// Bytes of shared memory (after the histogram) the ranking needs: bucket
// starts and the candidates grouped by bucket (FP32: the key packed with
// the bin; FP64: key and bin), FP32 also the whole list's key and bin words
// in list order (read from global memory once).
__host__ __device__ constexpr unsigned rank_region_bytes(bool f64) {
  return unsigned(kRRadix) * 4u + unsigned(kMaxSort) * 16u;
}

// Final order of the nc candidates (value descending, bin ascending) and
// the first `take` written at their ranks.  Every CTA counts the candidates
// per bucket (rank_bucket: bucket order is key order) and groups the whole
// list by bucket in shared memory; then each CTA ranks its share of the
// list, a warp per candidate: rank = candidates in earlier
// buckets + members of its bucket ahead of it.  The work per CTA is its
// share times the bucket sizes, so a bucket of thousands of exact ties
// costs every CTA a little rather than one CTA a lot.  (Ownership is by
// position in the candidate list, which every CTA sees alike.)  With exact ties of
// the k-th key beyond capacity (tie_by_pos), those ties were written in
// ascending bin order right after every larger value: their rank is their
// position in the list.
template <bool F64>
__device__ __forceinline__ void rank_candidates(const ResWork& w, unsigned nc, unsigned long long take,
                                                unsigned long long tmin, bool tie_by_pos,
                                                unsigned long long tie_key, unsigned char* rsm, unsigned* sh,
                                                unsigned* wsum, unsigned long long* bins_out, double* probs_out) {
  const unsigned nb = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* bstart = reinterpret_cast<unsigned*>(rsm + kRHistBytes);                  // [kRRadix]
  unsigned long long* gk = reinterpret_cast<unsigned long long*>(bstart + kRRadix);     // [kMaxSort]
  unsigned long long* gi = gk + kMaxSort;                                               // [kMaxSort] (FP64)
  unsigned* kc = reinterpret_cast<unsigned*>(gi);                                      // [kMaxSort] (FP32)
  unsigned* ic = kc + kMaxSort;                                                         // [kMaxSort] (FP32)
  for (int d = tid; d < kRRadix; d += kRThreads) sh[d] = 0u;
  __syncthreads();
  // the CTAs read the same list: each starts at its own offset.  FP32 keeps
  // the list's key and bin words in shared memory in list order, so that
  // the passes below read global memory no more.
  const unsigned rot = (blockIdx.x * nc) / nb;
  auto at = [&](unsigned e) { const unsigned f = e + rot; return f >= nc ? f - nc : f; };
  for (unsigned e0 = 0; e0 < nc; e0 += 4 * kRThreads) {
    unsigned long long kk[4], ii[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned e = e0 + u * kRThreads + tid;
      if (e < nc) {
        kk[u] = __ldcg(w.cand_key + at(e));
        if (!F64) ii[u] = __ldcg(w.cand_idx + at(e));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned e = e0 + u * kRThreads + tid;
      if (e < nc) {
        atomicAdd(&sh[rank_bucket<F64>(kk[u], tmin)], 1u);
        if constexpr (!F64) {
          kc[at(e)] = unsigned(kk[u]);
          ic[at(e)] = unsigned(ii[u]);
        }
      }
    }
  }
  __syncthreads();
  // exclusive prefix over the buckets: 4 per thread, then warps, then CTA
  {
    const uint4 c4 = reinterpret_cast<const uint4*>(sh)[tid];
    const unsigned own = c4.x + c4.y + c4.z + c4.w;
    unsigned inc = own;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += o;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const unsigned v = wsum[lane];
      unsigned x = v;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += o;
      }
      wsum[lane] = x - v;
    }
    __syncthreads();
    const unsigned b0 = wsum[warp] + inc - own;
    uint4 st4;
    st4.x = b0;
    st4.y = b0 + c4.x;
    st4.z = st4.y + c4.y;
    st4.w = st4.z + c4.z;
    reinterpret_cast<uint4*>(bstart)[tid] = st4;
    reinterpret_cast<uint4*>(sh)[tid] = st4;      // the grouping cursors
  }
  __syncthreads();
  // the whole list grouped by bucket (order within a bucket is arbitrary:
  // ranks compare keys and bins)
  for (unsigned e0 = 0; e0 < nc; e0 += 4 * kRThreads) {
    unsigned long long kk[4], ii[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned e = e0 + u * kRThreads + tid;
      if (e < nc) {
        if constexpr (F64) {
          kk[u] = __ldcg(w.cand_key + at(e));
          ii[u] = __ldcg(w.cand_idx + at(e));
        } else {
          kk[u] = kc[e];
          ii[u] = ic[e];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned e = e0 + u * kRThreads + tid;
      if (e >= nc) continue;
      const unsigned pos = atomicAdd(&sh[rank_bucket<F64>(kk[u], tmin)], 1u);
      if constexpr (F64) {
        gk[pos] = kk[u];
        gi[pos] = ii[u];
      } else {
        gk[pos] = (kk[u] << 32) | (0xffffffffull - ii[u]);
      }
    }
  }
  __syncthreads();
  // this CTA's share of the candidate list (by list position, the same in
  // every CTA; the order inside a grouped bucket differs between CTAs), a
  // warp per candidate
  const unsigned per = (nc + nb - 1) / nb;
  const unsigned p0 = blockIdx.x * per, p1 = p0 + per < nc ? p0 + per : nc;
  for (unsigned f = p0 + unsigned(warp); f < p1; f += kRWarps) {
    const unsigned long long key = F64 ? __ldcg(w.cand_key + f) : (unsigned long long)kc[f];
    const unsigned long long bin = F64 ? __ldcg(w.cand_idx + f) : (unsigned long long)ic[f];
    if (tie_by_pos && key == tie_key) continue;     // written by position below
    const unsigned long long kp = F64 ? key : ((key << 32) | (0xffffffffull - bin));
    const unsigned long long xp = F64 ? bin : 0ull;
    const unsigned q = rank_bucket<F64>(key, tmin);
    const unsigned b = bstart[q], e = sh[q];          // the bucket's segment
    unsigned c = 0;
    for (unsigned j = b + unsigned(lane); j < e; j += 32) {
      if constexpr (F64)
        c += (gk[j] > kp) || (gk[j] == kp && gi[j] < xp);
      else
        c += gk[j] > kp;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    const unsigned rank = b + c;
    if (lane == 0 && rank < take) {
      bins_out[rank] = bin;
      probs_out[rank] = value_of_key<F64>(key);
    }
  }
  if (tie_by_pos) {
    // ties written at their list positions (ascending bins after every
    // larger value), each by one CTA
    for (unsigned f = blockIdx.x + nb * unsigned(tid); f < nc && f < take; f += nb * kRThreads) {
      const unsigned long long kk = __ldcg(w.cand_key + f);
      if (kk != tie_key) continue;
      bins_out[f] = __ldcg(w.cand_idx + f);
      probs_out[f] = value_of_key<F64>(kk);
    }
  }
}

// TAIL: the input is not read but computed -- the query's contraction
// steps before the last run first (tail_pre_steps), then every CTA
// computes its slice of the last step's bins itself (each bin one inner
// product over the shared index, the operands in registers or shared
// memory, the FP32 multiply-adds in the order of the per-step kernel, so
// the bins are the same bit for bit), writes them to T.P in bin order and
// keeps their keys -- the bins are written once and never read back.
template <bool F64, bool TAIL>
__global__ void __launch_bounds__(kRThreads, 1)
select_resident_kernel(const void* x, int aligned, uint64_t n, uint64_t per, unsigned long long key_thr64, int k,
                       int cap, ResWork w, unsigned long long* bins_out, double* probs_out, int* n_found, int* err,
                       TailArgs Tp) {
  static_assert(!(F64 && TAIL), "the fused launch computes FP32 bins");
  // the fused launch reads its arguments from shared memory (one parallel
  // copy of the parameter block instead of scattered parameter loads)
  const TailArgs* tq = &Tp;
  if constexpr (TAIL) {
    __shared__ __align__(16) TailArgs tsh;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&Tp);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&tsh);
    for (int i = int(threadIdx.x); i < int(sizeof(TailArgs) / 8); i += kRThreads) dst[i] = src[i];
    __syncthreads();
    tq = &tsh;
  }
  const TailArgs& T = *tq;
  // Shared memory holds one 32-bit word per value: the whole key of an FP32
  // value, the high word of the 64-bit key of an FP64 value (its low word
  // is read back from the input only for values whose high word equals the
  // determined prefix).  Digits: 12, 12 and 8 bits per word.
  constexpr int KB = F64 ? 64 : 32;
  constexpr int kPasses = F64 ? 6 : 3;
  constexpr int V = F64 ? 2 : 4;                    // values per 16-byte vector
  extern __shared__ __align__(16) unsigned char rsm[];
  unsigned* sh = reinterpret_cast<unsigned*>(rsm);                 // [kRRadix]
  unsigned* keys = reinterpret_cast<unsigned*>(rsm + kRHistBytes); // [per], later the ranking's region
  __shared__ ResState st;
  __shared__ unsigned long long wtot[2 * kRWarps + 1];
  __shared__ unsigned wcnt[kRWarps];
  const unsigned nb = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long key_thr = F64 ? key_thr64 : (key_thr64 >> 32);
  const uint64_t start = uint64_t(blockIdx.x) * per;
  const int cnt = int(start < n ? ((n - start) < per ? (n - start) : per) : 0);
  // low word of the 64-bit key of value i of the slice (FP64 only)
  auto low_word = [&](int i) -> unsigned {
    return unsigned(key_f64(static_cast<const double*>(x)[start + i]));
  };
  auto full_key = [&](int i, unsigned kk) -> unsigned long long {
    if constexpr (F64) return ((unsigned long long)kk << 32) | low_word(i);
    else return (unsigned long long)kk;
  };
  unsigned bar = 0;                                 // barriers met so far
  bool ok = true;
  // the control word and the first two passes' histograms are cold at the
  // start of a step: fetch them into L2 while the slice is produced
  if (tid < 2) {
    const unsigned line = blockIdx.x + unsigned(tid) * nb;          // 32 counters per 128-byte line
    if (line < unsigned(2 * kRRadix / 32)) prefetch_l2(w.hist + size_t(line) * 32);
  } else if (tid == 2 && blockIdx.x == 0) {
    prefetch_l2(w.ctl);
  }
  if (tid == 0) {
    st.prefix = 0ull;
    st.krem = (unsigned long long)k;
    st.take = 0ull;
    st.lo = KB;
    st.done = 0;
  }
  for (int d = tid; d < kRRadix; d += kRThreads) sh[d] = 0u;
  // everything above touches only parameters and shared memory (and L2
  // hints): under a programmatic dependent launch it overlaps the end of
  // the previous kernel
  pdl_wait();      // the previous kernel on the stream has completed
  pdl_trigger();   // the next one may start launching
  if constexpr (TAIL) {
    if (T.n_levels > 0) ok = tail_pre_steps(T, w, nb, bar, reinterpret_cast<float*>(rsm + kRHistBytes));
  }
  __syncthreads();
  // pass 0 with the load: keys of excluded values (NaN or below the
  // threshold) are stored as 0, which no included value has (the smallest
  // included key word is 0x007fffff for FP32, 0x000fffff for FP64)
  if constexpr (TAIL) {
    __shared__ float2 tred[kRWarps];
    // the thread's bins summed as an unevaluated FP32 pair (hi + lo, each
    // addition error-free by Knuth's TwoSum), reduced over the CTA as pairs
    // and converted to FP64 once: the FP64 pipe of this GPU is too narrow
    // for one FP64 addition per bin
    float s_hi = 0.f, s_lo = 0.f;
    if (ok) {
      // stage Y: row j at ys + j * ystride (16-byte aligned rows); and, when
      // the slice's X rows are a range that fits, those rows at xs
      float* ys = reinterpret_cast<float*>(rsm + tail_y_offset(per));
      float* xs = ys + T.N * T.ystride;
      const int kd = T.Kd;
      const int kd_log2 = __ffs(kd) - 1;
      const int ystride = T.ystride;
      const uint32_t ustart = uint32_t(start);
      const bool xst = T.x_rows > 0 && cnt > 0;
      const uint32_t x0 = xst ? tail_pext(ustart, T.rows) : 0u;
      const int nx = xst ? int(tail_pext(ustart + uint32_t(cnt) - 1u, T.rows) - x0) + 1 : 0;
      // four loads in flight per thread and round; every CTA starts at its
      // own offset, so that the CTAs (which all read the same rows) spread
      // their requests over the L2 slices instead of queueing on the same
      // lines at the same time
      auto stage = [&](const float* src, float* dst, int rows) {
        if (kd >= 4) {
          const int q_log2 = kd_log2 - 2;
          const unsigned tot4 = unsigned(rows) << q_log2;
          const unsigned rot = (blockIdx.x * tot4) / nb;
          const float4* s4 = reinterpret_cast<const float4*>(src);
          for (unsigned e0 = 0; e0 < tot4; e0 += 4 * kRThreads) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned e = e0 + u * kRThreads + tid;
              unsigned f = e + rot;
              if (f >= tot4) f -= tot4;
              if (e < tot4) v[u] = __ldcg(s4 + f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const unsigned e = e0 + u * kRThreads + tid;
              unsigned f = e + rot;
              if (f >= tot4) f -= tot4;
              if (e < tot4) *reinterpret_cast<float4*>(dst + (f >> q_log2) * ystride + 4 * (f & ((1u << q_log2) - 1))) = v[u];
            }
          }
        } else {
          for (int e = tid; e < (rows << kd_log2); e += kRThreads)
            dst[(e >> kd_log2) * ystride + (e & (kd - 1))] = __ldcg(src + e);
        }
      };
      // one contiguous bit run per operand (the usual layout): a shift and
      // a mask per index
      const bool runs1 = T.rows.n <= 1 && T.cols.n <= 1;
      const uint32_t rpos = T.rows.n ? T.rows.pos[0] : 0u, rmask = T.rows.n ? (1u << T.rows.len[0]) - 1u : 0u;
      const uint32_t cpos = T.cols.n ? T.cols.pos[0] : 0u, cmask = T.cols.n ? (1u << T.cols.len[0]) - 1u : 0u;
      const float alpha = T.alpha;
      float* P = T.P;
      // the bin is r * N + j (Y owns the low bits, X the rest) and a Y row
      // fits in registers: thread j takes column j for every row of the
      // slice, Y read once into registers, the slice's X rows from shared
      // memory -- no staging of Y
      const bool band = xst && T.rows.n == 1 && T.cols.n == 1 && cpos == 0 && rpos == T.cols.len[0] && kd >= 4 &&
                        kd <= 16;
      if (!band) stage(T.Y, ys, int(T.N));
      if (xst) stage(T.X + (size_t(x0) << kd_log2), xs, nx);
      __syncthreads();
      if (band) {
        const int nbits = T.cols.len[0];
        const uint32_t ncol = 1u << nbits;
        const uint32_t r_hi = (ustart + uint32_t(cnt) - 1u) >> nbits;      // x0 = ustart >> nbits
        const float4* y4 = reinterpret_cast<const float4*>(T.Y);
        const int q4 = kd >> 2;
        for (uint32_t j0 = 0; j0 < ncol; j0 += kRThreads) {
          const uint32_t j = j0 + uint32_t(tid);
          float4 y[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (q < q4 && j < ncol) y[q] = __ldcg(y4 + size_t(j) * q4 + q);
          for (uint32_t r = x0; r <= r_hi; ++r) {
            const uint32_t b = (r << nbits) | j;
            const bool in = j < ncol && b >= ustart && b - ustart < uint32_t(cnt);
            unsigned kv = 0u;
            if (in) {
              const float4* xr = reinterpret_cast<const float4*>(xs + (r - x0) * ystride);
              float acc = 0.f;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if (q < q4) {
                  const float4 xa = xr[q];
                  acc = fmaf(xa.x, y[q].x, acc);
                  acc = fmaf(xa.y, y[q].y, acc);
                  acc = fmaf(xa.z, y[q].z, acc);
                  acc = fmaf(xa.w, y[q].w, acc);
                }
              }
              if (kd < 16) acc = fmaf(0.f, 0.f, acc);
              const float v = acc * alpha;
              P[b] = v;
              two_sum_add(s_hi, s_lo, v);
              const unsigned u = __float_as_uint(v);
              const bool nan = (u & 0x7fffffffu) > 0x7f800000u;
              const unsigned kk = unsigned(key_f32(v) >> 32);
              kv = (!nan && kk >= unsigned(key_thr)) ? kk : 0u;
              keys[b - ustart] = kv;
            }
            warp_hist_add(sh, kv != 0, kv >> (32 - kRBits), lane);
          }
        }
      }
      if (!band)
        tail_slice_general(T, ys, xs, x0, xst, ustart, cnt, unsigned(key_thr), keys, sh, s_hi, s_lo);
    }
    // the CTA's sum as a pair, then one FP64 value per CTA
    pair_warp_sum(s_hi, s_lo);
    if (lane == 0) tred[warp] = make_float2(s_hi, s_lo);
    __syncthreads();
    if (warp == 0) {
      float h = tred[lane].x, l = tred[lane].y;
      pair_warp_sum(h, l);
      if (lane == 0 && T.total) T.partials[blockIdx.x] = double(h) + double(l);
    }
  } else {
    // the loop bound is the same for the whole CTA: warp_hist_add needs
    // every lane of the warp
    for (int b0 = 0; b0 < cnt; b0 += kRThreads * V) {
      const int i0 = b0 + tid * V;
      unsigned kv[V];
      if constexpr (F64) {
        const double* p = static_cast<const double*>(x) + start + i0;
        double a[2];
        if (aligned && i0 + 2 <= cnt) {
          const double2 q = __ldg(reinterpret_cast<const double2*>(p));
          a[0] = q.x; a[1] = q.y;
        } else {
          a[0] = i0 < cnt ? p[0] : __longlong_as_double(0x7ff8000000000000ll);
          a[1] = i0 + 1 < cnt ? p[1] : __longlong_as_double(0x7ff8000000000000ll);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const unsigned long long u = __double_as_longlong(a[q]);
          const bool nan = (u & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
          const unsigned long long kk = key_f64(a[q]);
          kv[q] = (!nan && kk >= key_thr) ? unsigned(kk >> 32) : 0u;
        }
      } else {
        const float* p = static_cast<const float*>(x) + start + i0;
        float a[4];
        if (aligned && i0 + 4 <= cnt) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(p));
          a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = i0 + q < cnt ? p[q] : __uint_as_float(0x7fc00000u);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const unsigned u = __float_as_uint(a[q]);
          const bool nan = (u & 0x7fffffffu) > 0x7f800000u;
          const unsigned kk = unsigned(key_f32(a[q]) >> 32);
          kv[q] = (!nan && kk >= unsigned(key_thr)) ? kk : 0u;
        }
      }
#pragma unroll
      for (int q = 0; q < V; ++q) {
        if (i0 + q < cnt) keys[i0 + q] = kv[q];
        warp_hist_add(sh, kv[q] != 0, kv[q] >> (32 - kRBits), lane);
      }
    }
  }
  // the refinement loop: flush, barrier, decide; then the next digit from
  // shared memory (and, for the low word of FP64 keys, from the input)
  for (int pass = 0; pass < kPasses; ++pass) {
    const int word = pass / 3;                      // 0: the (high) word in shared memory, 1: the low word
    const int hi_w = 32 - kRBits * (pass % 3);      // digit bits [lo_w, hi_w) of the word: 32-20, 20-8, 8-0
    const int lo_w = pass % 3 == 2 ? 0 : hi_w - kRBits;
    const int lo = ((F64 && word == 0) ? 32 : 0) + lo_w;   // bit position in the whole key
    if (pass > 0) {
      const unsigned long long pfx = st.prefix;
      const unsigned pfx_hi = F64 ? unsigned(pfx >> 32) : unsigned(pfx);
      const unsigned pfx_lo = unsigned(pfx);
      const unsigned dmask = (1u << (hi_w - lo_w)) - 1u;
      for (int d = tid; d < kRRadix; d += kRThreads) sh[d] = 0u;
      __syncthreads();
      for (int i0 = 0; i0 < cnt; i0 += kRThreads) {
        const int i = i0 + tid;
        const unsigned kk = i < cnt ? keys[i] : 0u;
        bool in = false;
        unsigned dig = 0;
        if (kk != 0) {
          if (word == 0) {
            in = hi_w >= 32 || (kk >> hi_w) == (pfx_hi >> hi_w);
            dig = (kk >> lo_w) & dmask;
          } else if (kk == pfx_hi) {
            const unsigned lw = low_word(i);
            in = hi_w >= 32 || (lw >> hi_w) == (pfx_lo >> hi_w);
            dig = (lw >> lo_w) & dmask;
          }
        }
        warp_hist_add(sh, in, dig, lane);
      }
    }
    __syncthreads();
    unsigned* gh = w.hist + size_t(pass) * kRRadix;
    for (int d = tid; d < kRRadix; d += kRThreads) {
      const unsigned v = sh[d];
      if (v) atomicAdd(gh + d, v);
    }
    if (!(ok = res_barrier(w.ctl, 1ull << 32, nb * ++bar) != 0ull)) break;
    res_decide(gh, pass, lo, lo == 0, k, cap, &st, wtot);
    if (st.done) break;
  }
  unsigned long long nc = 0;
  if (ok) {
    const int done = st.done, lo = st.lo;
    const unsigned long long pfx = st.prefix;
    // compaction: values above the bucket, and the bucket itself unless it
    // is an oversized group of exact ties.  Counted first (one slot
    // reservation per CTA), then written, each thread its own elements in
    // order.
    auto takes = [&](int i, unsigned kk) -> bool {
      if (kk == 0) return false;
      if (done == 2) return true;
      if (!F64 || lo >= 32) {
        // the bucket is decided within the word in shared memory
        const int l = F64 ? lo - 32 : lo;
        const unsigned pw = F64 ? unsigned(pfx >> 32) : unsigned(pfx);
        const unsigned hb = kk >> l, pv = pw >> l;
        return done == 3 ? hb > pv : hb >= pv;
      }
      // FP64 with the bucket in the low word: every high bit is decided
      const unsigned ph = unsigned(pfx >> 32);
      if (kk != ph) return kk > ph;
      const unsigned hb = low_word(i) >> lo, pv = unsigned(pfx) >> lo;
      return done == 3 ? hb > pv : hb >= pv;
    };
    unsigned mine = 0;
    for (int i = tid; i < cnt; i += kRThreads) mine += takes(i, keys[i]);
    // exclusive prefix of `mine` over the CTA
    unsigned incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) wcnt[warp] = incl;
    __syncthreads();
    __shared__ unsigned cta_taken;
    __shared__ unsigned long long cta_base;
    if (warp == 0) {
      const unsigned wv = wcnt[lane];
      unsigned wi = wv;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += o;
      }
      wcnt[lane] = wi - wv;                          // warps before this one
      if (lane == 31) {
        cta_taken = wi;
        cta_base = wi ? atomicAdd(w.ctl + 3, (unsigned long long)wi) : 0ull;
      }
    }
    __syncthreads();
    {
      unsigned long long r = cta_base + wcnt[warp] + (incl - mine);
      for (int i = tid; i < cnt; i += kRThreads) {
        const unsigned kk = keys[i];
        if (takes(i, kk)) {
          w.cand_key[r] = full_key(i, kk);
          w.cand_idx[r] = start + i;
          ++r;
        }
      }
    }
    __syncthreads();
    if (done == 3) ok = tie_scan<F64>(w, keys, cnt, start, x, st, wcnt, nb, bar);
    // the last barrier also sums the candidate counts into the low word
    if (ok) {
      const unsigned long long word = res_barrier(w.ctl, (1ull << 32) | cta_taken, nb * ++bar);
      ok = word != 0ull;
      nc = word & 0xffffffffull;
    }
  }
  if constexpr (TAIL) {
    // the FP64 probability sum, CTA partials in a fixed order, by the last
    // CTA (which ranks the fewest candidates, if any): every partial was
    // published before the first grid barrier
    if (ok && T.total && blockIdx.x == nb - 1 && warp == 0) {
      double v = 0.0;
      for (unsigned c = lane; c < nb; c += 32) v += __ldcg(T.partials + c);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) *T.total = v;
    }
  }
  if (ok) {
    // the histograms are no longer read by anyone
    for (uint64_t i = uint64_t(blockIdx.x) * kRThreads + tid; i < uint64_t(kRMaxPasses) * kRRadix;
         i += uint64_t(nb) * kRThreads)
      w.hist[i] = 0u;
    // ranking (rank_candidates): the lowest selectable key is the decided
    // bucket's, or the threshold when every value is taken
    const unsigned long long take = st.take;
    if (st.done == 3) nc += st.krem;
    if (nc > (unsigned long long)kMaxSort) nc = kMaxSort;
    const unsigned long long tmin = st.done == 2 ? key_thr : st.prefix;
    if (nc > 0)
      rank_candidates<F64>(w, unsigned(nc), take, tmin, st.done == 3, st.prefix, rsm, sh, wcnt, bins_out,
                           probs_out);
    if (blockIdx.x == 0 && tid == 0) *n_found = int(take);
  } else if (tid == 0 && err) {
    atomicExch(err, 1);
  }
  // the last CTA out re-arms the control words (every CTA has read the
  // candidate count and passed its last barrier by now); after an abort it
  // also clears the histograms, which some CTAs may have left dirty
  __shared__ int last;
  __syncthreads();
  // (no fences: the next launch on the stream starts after this one ends)
  if (tid == 0) last = atomicAdd(w.ctl + 1, 1ull) == nb - 1;
  __syncthreads();
  if (last) {
    if (__ldcg(w.ctl + 2))
      for (int i = tid; i < kRMaxPasses * kRRadix; i += kRThreads) w.hist[i] = 0u;
    if (tid == 0) {
      w.ctl[0] = 0ull;
      w.ctl[1] = 0ull;
      w.ctl[2] = 0ull;
      w.ctl[3] = 0ull;
    }
  }
}

}  // namespace

namespace {
// bytes of the streaming kernel's part of the workspace
size_t coop_part_bytes(int grid) {
  return sizeof(unsigned) * kCPasses * kCopies * kCRadix + sizeof(unsigned long long) * 32 +
         2 * sizeof(unsigned long long) * kMaxSort + sizeof(unsigned) * kMaxSort + sizeof(unsigned) * size_t(grid) +
         256;
}
}  // namespace

// One workspace serves both cooperative kernels: the resident kernel's
// control words sit in unused words of the streaming kernel's control
// block, its histograms after the streaming kernel's part, and both kernels
// leave everything they need zeroed as they found it.
size_t select_coop_bytes(int grid) {
  return coop_part_bytes(grid) + sizeof(unsigned) * kRMaxPasses * kRRadix + 256;
}

int select_coop_grid() {
  // computed once per process (thread-safe initialisation)
  static const int g = [] {
    int dev = 0, sms = 152, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(select_coop_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCSmem);
    cudaFuncSetAttribute(select_coop_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, select_coop_kernel<false>, kCoopThreads, kCSmem);
    int per64 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per64, select_coop_kernel<true>, kCoopThreads, kCSmem);
    per = per < per64 ? per : per64;
    return sms * (per >= 2 ? 2 : (per > 0 ? per : 1));
  }();
  return g;
}

// The resident kernel runs one 1024-thread CTA per SM (0 if it cannot be
// made co-resident with its largest shared-memory size).
int select_resident_grid() {
  static const int g = [] {
    int dev = 0, sms = 152, p32 = 0, p64 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(select_resident_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRSmemMax);
    cudaFuncSetAttribute(select_resident_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRSmemMax);
    cudaFuncSetAttribute(select_resident_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRSmemMax);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p32, select_resident_kernel<false, false>, kRThreads, kRSmemMax);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p64, select_resident_kernel<true, false>, kRThreads, kRSmemMax);
    int pt = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pt, select_resident_kernel<false, true>, kRThreads, kRSmemMax);
    int r = (p32 >= 1 && p64 >= 1 && pt >= 1) ? sms : 0;
    if (r > select_coop_grid()) r = select_coop_grid();   // tie counts live in the streaming part
    return r;
  }();
  return g;
}

// Shared memory the resident kernel needs for n values on `grid` CTAs (0:
// does not fit); *per = values per CTA (a multiple of 4, so every slice
// starts 16-byte aligned).
size_t select_resident_smem(uint64_t n, int is_f64, int grid, uint64_t* per) {
  if (grid <= 0) return 0;
  uint64_t p = (n + uint64_t(grid) - 1) / uint64_t(grid);
  p = (p + 3) & ~uint64_t(3);
  uint64_t region = p * 4;                         // one 32-bit key word per value
  // room for the ranking's bucket starts and owned candidates
  const uint64_t rank = rank_region_bytes(is_f64 != 0);
  if (region < rank) region = rank;
  const uint64_t need = uint64_t(kRHistBytes) + region;
  if (per) *per = p;
  return need <= uint64_t(kRSmemMax) ? size_t(need) : 0;
}

namespace {
// The resident kernel's part of the shared selection workspace.
ResWork resident_work(void* work) {
  char* p = static_cast<char*>(work);
  ResWork w;
  w.ctl = reinterpret_cast<unsigned long long*>(p + kRCtlOffset);
  w.cand_key = reinterpret_cast<unsigned long long*>(p + sizeof(unsigned long long) * 32);
  w.cand_idx = w.cand_key + kMaxSort;
  // the streaming kernel's tie counts (layout of launch_select_coop)
  w.tie_count = reinterpret_cast<unsigned*>(p + sizeof(unsigned long long) * 32 + 2 * sizeof(unsigned long long) * kMaxSort +
                                            sizeof(unsigned) * kCPasses * kCopies * kCRadix + sizeof(unsigned) * kMaxSort);
  w.hist = reinterpret_cast<unsigned*>(p + ((coop_part_bytes(select_coop_grid()) + 255) & ~size_t(255)));
  return w;
}
}  // namespace

cudaError_t launch_select_resident(void* work, int grid, const void* x, int is_f64, uint64_t n, int k,
                                   double threshold, unsigned long long* bins_out, double* probs_out, int* n_found,
                                   int* err, cudaStream_t s) {
  if (k < 1 || k > kSelectMaxK) return cudaErrorInvalidValue;
  uint64_t per = 0;
  const size_t smem = select_resident_smem(n, is_f64, grid, &per);
  if (!smem) return cudaErrorInvalidValue;
  // refinement stops once the k-th value's bucket holds at most cap values:
  // the values above it (< k) and the bucket then fit the ranking's
  // kMaxSort candidates, which costs less than another digit pass and its
  // grid barrier
  const int cap = kMaxSort - k;
  ResWork w = resident_work(work);
  const int aligned = (reinterpret_cast<uintptr_t>(x) % 16) == 0;
  const unsigned long long kt = threshold_key(is_f64, threshold);
  const TailArgs none{};
  if (is_f64)
    return launch_k(select_resident_kernel<true, false>, dim3(grid), dim3(kRThreads), smem, s, true, x, aligned, n,
                    per, kt, k, cap, w, bins_out, probs_out, n_found, err, none);
  return launch_k(select_resident_kernel<false, false>, dim3(grid), dim3(kRThreads), smem, s, true, x, aligned, n,
                  per, kt, k, cap, w, bins_out, probs_out, n_found, err, none);
}

// Rows of X a slice of `per` bins needs when they form a range (x_range):
// at most ceil(per / N) + 1.
int64_t tail_x_rows(const TailArgs& t, uint64_t per) {
  if (!t.x_range || t.N < 1) return 0;
  const int64_t r = int64_t((per + uint64_t(t.N) - 1) / uint64_t(t.N)) + 1;
  return r < t.M ? r : t.M;
}

namespace {
// Shared memory of the fused launch: histogram, slice keys (or the stage of
// the steps before the last), staged Y, staged X rows when they form a
// range and fit, at least the ranking's region.  0: Y does not fit.
size_t tail_layout(uint64_t n, const TailArgs& t, int grid, uint64_t* per, int* x_rows) {
  uint64_t p = 0;
  if (!select_resident_smem(n, 0, grid, &p)) return 0;
  const uint64_t y_end = tail_y_offset(p) + uint64_t(t.N) * uint64_t(t.ystride) * 4;
  if (y_end > uint64_t(kRSmemMax)) return 0;
  const int64_t xr = tail_x_rows(t, p);
  const uint64_t x_end = y_end + uint64_t(xr) * uint64_t(t.ystride) * 4;
  const bool stage_x = xr > 0 && x_end <= uint64_t(kRSmemMax);
  uint64_t need = stage_x ? x_end : y_end;
  const uint64_t rank = uint64_t(kRHistBytes) + rank_region_bytes(false);
  if (need < rank) need = rank;
  if (need > uint64_t(kRSmemMax)) return 0;
  if (per) *per = p;
  if (x_rows) *x_rows = stage_x ? int(xr) : 0;
  return size_t(need);
}
}  // namespace

size_t select_tail_smem(uint64_t n, const TailArgs& t, int grid, uint64_t* per) {
  return tail_layout(n, t, grid, per, nullptr);
}

cudaError_t launch_select_tail(void* work, int grid, const TailArgs& t, uint64_t n, int k, double threshold,
                               unsigned long long* bins_out, double* probs_out, int* n_found, int* err,
                               cudaStream_t s) {
  if (k < 1 || k > kSelectMaxK) return cudaErrorInvalidValue;
  if (t.Kd < 1 || (t.Kd & (t.Kd - 1)) || t.n_levels < 0 || t.n_levels > kTailMaxLevels) return cudaErrorInvalidValue;
  if (t.rows.n > kTailMaxRuns || t.cols.n > kTailMaxRuns || (t.total && !t.partials)) return cudaErrorInvalidValue;
  uint64_t per = 0;
  TailArgs ta = t;
  const size_t smem = tail_layout(n, t, grid, &per, &ta.x_rows);
  if (!smem) return cudaErrorInvalidValue;
  const int cap = kMaxSort - k;
  ResWork w = resident_work(work);
  const unsigned long long kt = threshold_key(0, threshold);
  return launch_k(select_resident_kernel<false, true>, dim3(grid), dim3(kRThreads), smem, s, true,
                  static_cast<const void*>(nullptr), 0, n, per, kt, k, cap, w, bins_out, probs_out, n_found, err, ta);
}

cudaError_t launch_select_coop(void* work, int grid, const void* x, int is_f64, uint64_t n, int k, double threshold,
                               unsigned long long* bins_out, double* probs_out, int* n_found, int* err,
                               cudaStream_t s) {
  if (k < 1 || k > kSelectMaxK) return cudaErrorInvalidValue;
  const int cap = (k > 512 ? k : 512) < kMaxSort - k ? (k > 512 ? k : 512) : kMaxSort - k;
  char* p = static_cast<char*>(work);
  CoopWork w;
  w.ctl = reinterpret_cast<unsigned long long*>(p);
  p += sizeof(unsigned long long) * 32;
  w.cand_key = reinterpret_cast<unsigned long long*>(p);
  p += sizeof(unsigned long long) * kMaxSort;
  w.cand_idx = reinterpret_cast<unsigned long long*>(p);
  p += sizeof(unsigned long long) * kMaxSort;
  w.hist = reinterpret_cast<unsigned*>(p);
  p += sizeof(unsigned) * kCPasses * kCopies * kCRadix;
  w.rank = reinterpret_cast<unsigned*>(p);
  p += sizeof(unsigned) * kMaxSort;
  w.tie_count = reinterpret_cast<unsigned*>(p);
  const int aligned = (reinterpret_cast<uintptr_t>(x) % 16) == 0;
  const unsigned long long kt = threshold_key(is_f64, threshold);
  if (is_f64)
    return launch_k(select_coop_kernel<true>, dim3(grid), dim3(kCoopThreads), size_t(kCSmem), s, true, x, aligned, n,
                    kt, k, cap, w, bins_out, probs_out, n_found, err);
  return launch_k(select_coop_kernel<false>, dim3(grid), dim3(kCoopThreads), size_t(kCSmem), s, true, x, aligned, n,
                  kt, k, cap, w, bins_out, probs_out, n_found, err);
}

// ---- allocation-free variant -------------------------------------------------
// Fixed scratch for sqc_top_bins_noalloc: the same layout launch_select
// carves from a query's workspace (control block, candidate list, radix
// histograms, tie counts), sized for k <= kSelectMaxK and 1024 tie ranges.
constexpr int kStaticSelectBlocks = 1024;
constexpr size_t kStaticSelectBytes = sizeof(unsigned long long) * ST_WORDS +
                                      2 * sizeof(unsigned long long) * kMaxSort +
                                      sizeof(unsigned) * kPasses * kRadix +
                                      sizeof(unsigned) * kStaticSelectBlocks + 256;
static __device__ __align__(256) unsigned char g_select_scratch[kStaticSelectBytes];

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

size_t select_static_bytes() { return kStaticSelectBytes; }

// The caller has made `device` current.  The array's name is only a host
// stand-in for the device symbol, so its device address is looked up once
// per device and cached.
cudaError_t launch_select_static(int device, const void* x, int is_f64, uint64_t n, int k, double threshold,
                                 unsigned long long* bins_out, double* probs_out, int* n_found, cudaStream_t s) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
      if (e != cudaSuccess) return e;
      g_scratch_addr[device] = p;
    }
    base = g_scratch_addr[device];
  }
  SelectWork w{};
  select_work_carve(base, 0, kStaticSelectBlocks, &w);
  // the control block and the histograms must start at zero; the array keeps
  // whatever the previous call left
  cudaError_t e = cudaMemsetAsync(w.state, 0, sizeof(unsigned long long) * ST_WORDS, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.hist, 0, sizeof(unsigned) * kPasses * kRadix, s);
  if (e != cudaSuccess) return e;
  return launch_select(w, x, is_f64, n, k, threshold, bins_out, probs_out, n_found, s);
}

cudaError_t select_configure() { return cudaSuccess; }

cudaError_t launch_sum(const void* x, int is_f64, uint64_t n, double* partials, unsigned* counter, double* total,
                       cudaStream_t s) {
  const int g = stream_grid(n, 1024);
  return launch_k(sum_kernel, dim3(g), dim3(kSelThreads), 0, s, false, x, is_f64, n, partials, counter, total);
}

}  // namespace sqc
