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
//  4. one CTA sorts the candidates (bitonic, in shared memory) and writes
//     the first k.
// The FP64 probability sum is a grid reduction with a fixed summation
// order (per-CTA partials added by the last CTA in CTA order).
#include <mutex>

#include "common.cuh"

namespace sqc {

namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kPasses = 8;          // 64-bit keys
constexpr int kSelThreads = 256;
constexpr int kSortThreads = 1024;
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

__device__ __forceinline__ unsigned long long key_of(const void* x, int is_f64, uint64_t i, double* val) {
  if (is_f64) {
    const double v = static_cast<const double*>(x)[i];
    *val = v;
    const unsigned long long u = __double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
  }
  const float f = static_cast<const float*>(x)[i];
  *val = double(f);
  const unsigned u = __float_as_uint(f);
  const unsigned k = (u >> 31) ? ~u : (u | 0x80000000u);
  return (unsigned long long)k << 32;
}

__global__ void __launch_bounds__(kSelThreads)
radix_pass(const void* x, int is_f64, uint64_t n, double thr, int k, int pass, int last_pass, int cap,
           unsigned* hist_all, unsigned long long* st) {
  __shared__ unsigned sh[kRadix];
  __shared__ bool is_last;
  if (st[ST_DONE] != 0) return;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x) sh[d] = 0;
  __syncthreads();
  const int shift = 64 - kRadixBits * (pass + 1);
  const unsigned long long prefix = st[ST_PREFIX];
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    double v;
    const unsigned long long key = key_of(x, is_f64, i, &v);
    if (!(v >= thr)) continue;
    if (pass > 0 && (key >> (shift + kRadixBits)) != (prefix >> (shift + kRadixBits))) continue;
    atomicAdd(&sh[(key >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  unsigned* hist = hist_all + pass * kRadix;
  for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
    if (sh[d]) atomicAdd(&hist[d], sh[d]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t = atomicAdd(&st[ST_COUNTER], 1ull);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last || threadIdx.x != 0) return;
  __threadfence();
  volatile unsigned* h = hist;
  unsigned long long total = 0;
  for (int d = 0; d < kRadix; ++d) total += h[d];
  unsigned long long krem = (pass == 0) ? (unsigned long long)k : st[ST_KREM];
  if (pass == 0) {
    st[ST_TAKE] = total < (unsigned long long)k ? total : (unsigned long long)k;
    if (total <= (unsigned long long)k) {
      st[ST_DONE] = 2;
    }
  }
  if (st[ST_DONE] == 0) {
    unsigned long long cum = 0;
    int d = kRadix - 1;
    for (; d > 0; --d) {
      if (cum + h[d] >= krem) break;
      cum += h[d];
    }
    st[ST_PREFIX] = prefix | ((unsigned long long)d << shift);
    st[ST_BITS] = (unsigned long long)(kRadixBits * (pass + 1));
    st[ST_KREM] = krem - cum;
    if (h[d] <= (unsigned)cap)
      st[ST_DONE] = 1;
    else if (last_pass)
      st[ST_DONE] = 3;
  }
  for (int d = 0; d < kRadix; ++d) h[d] = 0;
  st[ST_COUNTER] = 0;
}

// Copy the values that are certainly selected, and the current bucket
// (unless it is an oversized group of exact ties), to the candidate list.
__global__ void __launch_bounds__(kSelThreads)
compact(const void* x, int is_f64, uint64_t n, double thr, unsigned long long* st, unsigned long long* ck,
        unsigned long long* ci) {
  const unsigned long long done = st[ST_DONE];
  const int bits = int(st[ST_BITS]);
  const unsigned long long pv = bits ? (st[ST_PREFIX] >> (64 - bits)) : 0ull;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
    double v;
    const unsigned long long key = key_of(x, is_f64, i, &v);
    if (!(v >= thr)) continue;
    bool take;
    if (done == 2) {
      take = true;
    } else {
      const unsigned long long hb = key >> (64 - bits);
      take = (done == 3) ? (hb > pv) : (hb >= pv);
    }
    if (take) {
      const unsigned long long slot = atomicAdd(&st[ST_NCAND], 1ull);
      ck[slot] = key;
      ci[slot] = i;
    }
  }
}

// Exact ties beyond capacity: count them per contiguous range ...
__global__ void __launch_bounds__(kSelThreads)
tie_count(const void* x, int is_f64, uint64_t n, double thr, const unsigned long long* st, unsigned* counts,
          uint64_t range) {
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
    if (v >= thr && key == tkey) ++c;
  }
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// ... then append the first KREM of them in ascending bin order.
__global__ void __launch_bounds__(kSelThreads)
tie_write(const void* x, int is_f64, uint64_t n, double thr, unsigned long long* st, const unsigned* counts,
          uint64_t range, unsigned long long* ck, unsigned long long* ci) {
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
      tie = (v >= thr && key == tkey);
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

// Sort the candidates by (key descending, index ascending) and emit the
// first TAKE as (bin, probability).
__global__ void __launch_bounds__(kSortThreads)
sort_emit(const void* x, int is_f64, unsigned long long* st, const unsigned long long* ck,
          const unsigned long long* ci, unsigned long long* bins_out, double* probs_out, int* n_found) {
  extern __shared__ unsigned long long sm[];
  const unsigned long long done = st[ST_DONE];
  unsigned long long nc = st[ST_NCAND];
  if (done == 3) nc += st[ST_KREM];
  if (nc > kMaxSort) nc = kMaxSort;
  unsigned P = 1;
  while (P < nc) P <<= 1;
  unsigned long long* keys = sm;
  unsigned long long* idx = sm + kMaxSort;
  for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < nc) {
      keys[i] = ck[i];
      idx[i] = ci[i];
    } else {
      keys[i] = 0ull;
      idx[i] = ~0ull;
    }
  }
  __syncthreads();
  // bitonic sort: "a before b" <=> a.key > b.key || (a.key == b.key && a.idx < b.idx)
  for (unsigned size = 2; size <= P; size <<= 1) {
    for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
      for (unsigned i = threadIdx.x; i < P; i += blockDim.x) {
        const unsigned j = i ^ stride;
        if (j > i) {
          const bool up = ((i & size) == 0);
          const unsigned long long ka = keys[i], kb = keys[j];
          const unsigned long long ia = idx[i], ib = idx[j];
          const bool a_first = (ka > kb) || (ka == kb && ia < ib);
          if (a_first != up) {
            keys[i] = kb; keys[j] = ka;
            idx[i] = ib; idx[j] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  const unsigned long long take = st[ST_TAKE];
  for (unsigned i = threadIdx.x; i < take; i += blockDim.x) {
    const unsigned long long b = idx[i];
    bins_out[i] = b;
    probs_out[i] = is_f64 ? static_cast<const double*>(x)[b] : double(static_cast<const float*>(x)[b]);
  }
  if (threadIdx.x == 0) {
    *n_found = int(take);
    for (int w = 0; w < ST_WORDS; ++w) st[w] = 0;   // re-arm for the next call
  }
}

__global__ void __launch_bounds__(kSelThreads)
sum_kernel(const void* x, int is_f64, uint64_t n, double* partials, unsigned* counter, double* total) {
  __shared__ double red[kSelThreads / 32];
  double s = 0.0;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x)
    s += is_f64 ? static_cast<const double*>(x)[i] : double(static_cast<const float*>(x)[i]);
  finish_total(s, partials, counter, total, red);
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
  const int g = stream_grid(n, w.max_blocks);
  const int passes = is_f64 ? kPasses : 4;
  for (int p = 0; p < passes; ++p)
    radix_pass<<<g, kSelThreads, 0, s>>>(x, is_f64, n, threshold, k, p, p == passes - 1, cap, w.hist, st);
  compact<<<g, kSelThreads, 0, s>>>(x, is_f64, n, threshold, st, w.cand_key, w.cand_idx);
  const uint64_t range = (n + w.max_blocks - 1) / w.max_blocks;
  const unsigned tb = unsigned((n + range - 1) / (range ? range : 1));
  const uint64_t rng = range ? range : 1;
  tie_count<<<tb ? tb : 1, kSelThreads, 0, s>>>(x, is_f64, n, threshold, st, w.tie_count, rng);
  tie_write<<<tb ? tb : 1, kSelThreads, 0, s>>>(x, is_f64, n, threshold, st, w.tie_count, rng, w.cand_key,
                                               w.cand_idx);
  const size_t smem = 2 * sizeof(unsigned long long) * kMaxSort;
  sort_emit<<<1, kSortThreads, smem, s>>>(x, is_f64, st, w.cand_key, w.cand_idx, bins_out, probs_out, n_found);
  return cudaGetLastError();
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

cudaError_t select_configure() {
  return cudaFuncSetAttribute(sort_emit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(2 * sizeof(unsigned long long) * kMaxSort));
}

cudaError_t launch_sum(const void* x, int is_f64, uint64_t n, double* partials, unsigned* counter, double* total,
                       cudaStream_t s) {
  const int g = stream_grid(n, 1024);
  sum_kernel<<<g, kSelThreads, 0, s>>>(x, is_f64, n, partials, counter, total);
  return cudaGetLastError();
}

}  // namespace sqc
