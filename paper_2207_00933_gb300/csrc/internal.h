// Internal kernel interfaces of the reconstruction library (not part of the
// C ABI).  Every tensor index here is a plain linear index into a
// power-of-two sized array; layouts are expressed as "maps": an output
// element (row r, column c) of a producer goes to offset rowmap[r] +
// colmap[c] of its destination, which lets each producer write the layout
// its consumer wants (no separate transpose passes).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace sqc {

enum OutKind : int { OUT_F32 = 0, OUT_F64 = 1, OUT_BF16X3 = 2 };

// ---- attribution (Eq. 1, Section 2.1) --------------------------------------
// fold: B[v][rev_n(x)] = sum_c prod_u W[v_u][c_u] * p[v][x | c << n]
//   (outgoing cut wires: outcome weights; the basis is the variant digit)
struct FoldArgs {
  const void* p;
  int in_f64;
  float* B;          // [V][2^n], data index stored bit-reversed
  int64_t V;
  int n;             // data qubits
  int kout;          // outgoing edges
  int outshift[16];  // bit shift of each outgoing edge's digit in v
};
cudaError_t launch_fold(const FoldArgs& a, cudaStream_t s);

// mix: A[e][xs] = sum_s prod_t D[e_t][s_t] * B[v(e with in-digits := s)][xs]
//   (incoming cut wires: prepared-state coefficients)
struct MixArgs {
  const float* B;
  float* A;          // [rows][2^n]
  int64_t rows;      // 4^k
  int n;
  int kin;
  int inshift[16];   // bit shift of each incoming edge's digit in e / v
};
cudaError_t launch_mix(const MixArgs& a, cudaStream_t s);

// fused fold + mix, shared-memory tiled (subcircuits with kin <= 7)
constexpr int kMaxFusedIn = 7;
constexpr int kAttrSmemMax = 64 * 1024;
constexpr int kAttrRing = 2;               // tile buffers of the ring-buffered attribution form
constexpr int kRingL1 = 4, kRingL2 = 5;     // its tiles: 2^kRingL1 low x 2^kRingL2 top data states
constexpr int kAttrPerLaunch = 16;
struct AttrDesc {
  const void* p;
  float* A;
  int in_f64;
  int n, kin, kout;
  int L1, L2;                 // x tile: 2^L1 low values x 2^L2 top-bit values
  int vec;                    // 32 x 8 tile, FP32 input, 16-byte aligned: 4 states per thread
  int async2;                 // vec, no outgoing edges, 4^kin <= 32: loads ring-buffered by cp.async
  int inshift[kMaxFusedIn];
  int outshift[16];
  int64_t block_begin;
  int64_t block_end;           // first block of the next descriptor
};
struct AttrLaunch {
  AttrDesc d[kAttrPerLaunch];
  int n;
};
cudaError_t launch_attr_fused(const AttrLaunch& L, int64_t blocks, int smem_bytes, cudaStream_t s);
cudaError_t attr_configure();

// Attribution fused into the merge (one recursion step on fresh outputs,
// states merging of Section 4 applied while attributing, Eq. 1): for a
// subcircuit whose roles follow the recursion's pattern -- the z lowest data
// bits zoomed, the next a active, the m = n - z - a highest merged -- only
// the 2^(a+m) kept states are attributed, in shared-memory tiles of 2^L1
// consecutive active values x all 2^L2 = 2^m merged values, and every tile
// writes the merged entries T[e][b] (b = the bit-reversed active bits,
// merged bits summed) through the merge's layout maps.  The resident A_i is
// not written.
struct AttrMergeDesc {
  const void* p;
  int in_f64;
  int n, kin, kout;
  int z, a;                  // zoomed (lowest data bits) and active (next) bit counts
  uint32_t zval;             // values of the zoomed bits (data-index order)
  int L1, L2;                // tile: 2^L1 active values x 2^L2 merged values (L2 = m <= 8)
  int inshift[kMaxFusedIn];
  int outshift[16];
  const uint64_t* rowmap;    // T's layout: the merge descriptor's maps
  const uint64_t* colmap;
  void* dst;                 // T_i, or the bins of a one-subcircuit query
  int kind;
  int64_t plane_stride;
  float alpha;
  int64_t block_begin;
  int64_t block_end;
};
struct AttrMergeLaunch {
  AttrMergeDesc d[kAttrPerLaunch];
  int n;
};
cudaError_t launch_attr_merge(const AttrMergeLaunch& L, int64_t blocks, int smem_bytes, cudaStream_t s);
// CTAs of the attribution-merge kernel resident on the device at once with
// smem_bytes of dynamic shared memory each (one wave).
int attr_merge_wave(bool f64, int smem_bytes);

// Staging of host inputs by the SMs: every buffer's 16-byte words copied
// from memory the device can read (mapped pinned host memory) to device
// memory, one launch for up to kAttrPerLaunch buffers (each 16-byte
// aligned, sizes multiples of 16 bytes).  Many loads in flight over the
// host link instead of one copy-engine transfer per buffer.
struct StageCopy {
  const void* src[kAttrPerLaunch];
  void* dst[kAttrPerLaunch];
  uint64_t words[kAttrPerLaunch];   // 16-byte words
  int n;
};
cudaError_t launch_stage_copy(const StageCopy& c, cudaStream_t s);

// ---- merge / zoom (Section 4, Algorithm 2) ----------------------------------
// T[e][b] = sum over data states with the zoom bits fixed and active bits
// spelling b of A[e][state]; written to dst + rowmap[e] + colmap[b].
struct MergeDesc {
  const float* A;
  int64_t rows;
  int n;
  uint32_t act_mask, mer_mask, zoom_val;  // storage-order bit masks
  int a, m;                               // active / merged bit counts
  int fast;                               // mer_mask == low m bits, act_mask == next a bits
  int lanes;                              // threads cooperating on one output (1..32, pow2)
  const uint64_t* rowmap;                 // [rows]
  const uint64_t* colmap;                 // [2^a]
  void* dst;
  int kind;                               // OutKind
  int64_t plane_stride;                   // OUT_BF16X3: elements between planes
  double alpha;
  int64_t block_begin;                    // first CTA of this descriptor
  // first-level slicing: the merge reads row rowsel[e] + row_add of A (the
  // sliced edges' digits fixed); rowsel == nullptr: row e
  const uint64_t* rowsel;
  int64_t row_add;
};
constexpr int kMaxMerge = 64;
// descs: device array of n descriptors; total_blocks = CTAs over all of them
cudaError_t launch_merge_blocks(const MergeDesc* descs, int n, int64_t total_blocks, cudaStream_t s);
// Merge pyramid of one subcircuit (A: [V][2^n]): level m = 1..n at
// pyr + V (2^n - 2^(n-m+1)), [V][2^(n-m)], level m = pairwise sums of level
// m-1 (level 0 = A).  One launch per kPyramidLevelsPerPass levels.
constexpr int kPyramidLevelsPerPass = 10;
cudaError_t launch_pyramid(const float* A, float* pyr, int64_t V, int n, cudaStream_t s);

// ---- contraction step, FP32 SIMT (Section 6.1: C = A B over the shared index)
struct GemmArgs {
  const float* A;           // [M][K]
  const float* B;           // [N][K]
  int64_t M, N, K;
  const uint64_t* rowmap;   // [M]
  const uint64_t* colmap;   // [N]
  void* C;
  int kind;                 // OutKind
  int64_t plane_stride;
  double alpha;
  int64_t chunk;            // FP32 terms per chunk before the FP64 add (0 = plain FP32)
  int vec4;                 // colmap[4j..4j+3] contiguous and 4-aligned for all j
  int accumulate;           // add into C instead of overwriting (later slices, FP32/FP64 outputs)
  double* partials;         // per-CTA sums of the written values (nullable)
  unsigned* counter;        // zero-initialised; last CTA writes *total and resets it
  double* total;
};
cudaError_t launch_gemm_simt(const GemmArgs& a, cudaStream_t s);

// ---- contraction step, split-BF16 on tcgen05 ---------------------------------
struct GemmTcArgs {
  const void* A;            // bf16 planes [3][Mp][Kp] (hi, mid, lo), K-contiguous
  const void* B;            // bf16 planes [3][Np][Kp]
  int64_t M, N, K;          // logical sizes
  int64_t Mp, Np, Kp;       // padded (Mp, Np multiples of 128; Kp multiple of 64)
  const uint64_t* rowmap;
  const uint64_t* colmap;
  void* C;
  int kind;
  int64_t plane_stride;
  double alpha;
  int64_t chunk;            // FP32 terms per pass before the FP64 add (0 = one pass; FP64 output only)
  int accumulate;           // add into C instead of overwriting (later slices, FP32/FP64 outputs)
  double* partials;
  unsigned* counter;
  double* total;
  int* err;                 // device error flag (bounded waits)
  int contig16;             // colmap: runs of 16 consecutive 4-aligned offsets, rowmap 4-aligned
  int pairs;                // allow 2-SM units (tcgen05.mma.cta_group::2) where they fill the SMs
  uint64_t wait_ns;         // limit of each barrier wait (0: 2 s)
};
cudaError_t launch_gemm_tc(const GemmTcArgs& a, cudaStream_t s);
bool gemm_tc_available();          // the driver's tensor-map encoder is reachable
int gemm_tc_min_rows();            // M and N of a tensor-core step must be >= this
int gemm_tc_k_align();             // the shared index is padded to a multiple of this
cudaError_t gemm_tc_configure();   // one-time kernel attributes (dynamic shared memory)

// ---- batched recursion level: one persistent launch over many queries -------
enum : int { kItemMerge = 0, kItemGemm = 1 };
struct BatchItem {
  int type;          // kItemMerge / kItemGemm
  int idx;           // merge descriptor or step index in the batch arrays
  int64_t tile;      // merge block (relative to the descriptor) or output tile
  int dep0, dep1;    // tensor slots that must be complete first (-1: none)
  int out;           // tensor slot this item writes (-1: none)
};
struct BatchStep {
  GemmArgs a;        // a.partials != null: the query's last step (probability sum)
  int cfg;           // tile configuration id (batch_tile_cfg)
  int from_launch;   // the output and the probability sum are BatchLaunch::out / total
  int64_t ntiles;
  double* partials;  // per-tile partial sums of the query's bins
  unsigned* counter;
  double* total;
};
struct BatchLaunch {
  const BatchItem* items;
  int64_t n_items;
  const MergeDesc* mdescs;
  const BatchStep* steps;
  unsigned* counts;          // [n_slots] completion counters (zero between launches)
  const unsigned* expected;  // [n_slots]
  int64_t n_slots;
  unsigned long long* head;
  unsigned* done;
  int* abort;
  int* err;
  uint64_t wait_ns;          // limit of each dependency wait
  void* out;                 // output of the steps marked from_launch (a single-query launch)
  double* total;             // their probability sum (nullable)
};
cudaError_t launch_batch(const BatchLaunch& L, int grid, cudaStream_t s);
cudaError_t batch_configure();
int batch_smem_bytes();
// tile configuration for a step of the batch kernel; *bm, *bn its tile
int batch_tile_cfg(int64_t M, int64_t N, int64_t K, bool chunked, int64_t chunk, int64_t* bm, int64_t* bn,
                   int policy);
constexpr int kBatchPolicies = 3;

// ---- probability check: FP64 sum of n values ---------------------------------
cudaError_t launch_sum(const void* x, int is_f64, uint64_t n, double* partials, unsigned* counter,
                       double* total, cudaStream_t s);

// ---- bin selection (Algorithm 1: keep the largest bins) ----------------------
struct SelectWork {
  unsigned* hist;          // [kPasses][kRadix]
  unsigned* state;         // small control block, see select.cu
  unsigned long long* cand_key;  // [cap]
  unsigned long long* cand_idx;  // [cap]
  unsigned* tie_count;     // [max_blocks]
  int cap;
  int max_blocks;
};
size_t select_work_bytes(int cap, int max_blocks);
void select_work_carve(void* base, int cap, int max_blocks, SelectWork* w);
cudaError_t launch_select(const SelectWork& w, const void* x, int is_f64, uint64_t n, int k,
                          double threshold, unsigned long long* bins_out, double* probs_out,
                          int* n_found, cudaStream_t s);
// Selection with scratch in a static device array instead of a workspace
// (the caller has made `device` current); select_static_bytes() is its size.
cudaError_t launch_select_static(int device, const void* x, int is_f64, uint64_t n, int k, double threshold,
                                 unsigned long long* bins_out, double* probs_out, int* n_found, cudaStream_t s);
size_t select_static_bytes();
// The same selection as ONE cooperative launch (grid barriers between the
// phases); `work` holds select_coop_bytes(grid) zero-initialised bytes,
// grid = select_coop_grid() (co-resident CTAs); err: device flag set when a
// bounded barrier wait gave up.
size_t select_coop_bytes(int grid);
int select_coop_grid();
cudaError_t launch_select_coop(void* work, int grid, const void* x, int is_f64, uint64_t n, int k, double threshold,
                               unsigned long long* bins_out, double* probs_out, int* n_found, int* err,
                               cudaStream_t s);
// The same selection with every CTA's slice of the input held in shared
// memory (one 1024-thread CTA per SM): one read of the input, 12-bit digits.
// Uses the same workspace as launch_select_coop.  select_resident_smem()
// returns 0 when n values do not fit; grid = select_resident_grid().
int select_resident_grid();
size_t select_resident_smem(uint64_t n, int is_f64, int grid, uint64_t* per);
cudaError_t launch_select_resident(void* work, int grid, const void* x, int is_f64, uint64_t n, int k,
                                   double threshold, unsigned long long* bins_out, double* probs_out, int* n_found,
                                   int* err, cudaStream_t s);
// one-time per-device kernel attributes (large shared memory for the sort)
cudaError_t select_configure();
constexpr int kSelectMaxK = 4096;

// ---- the last contraction steps fused into the resident selection ----------
// Index extraction by runs of consecutive bits: bit run t of the source
// index (len[t] bits from position pos[t]) lands at position out[t] of the
// result.  rows/cols of the last step are the parts of the bin index each
// operand owns (the bin is rowmap[i] + colmap[j], both bit deposits).
constexpr int kTailMaxRuns = 8;
struct TailPext {
  int n;
  unsigned char pos[kTailMaxRuns], len[kTailMaxRuns], out[kTailMaxRuns];
};
// One contraction step before the last, run in the same launch: its tiles
// are split over the CTAs, one tile per CTA at a time, 1024 threads each.
struct TailStep {
  GemmArgs a;
  int cfg;                  // tile shape: 0 = 32 x 32, 1 = 64 x 64, 2 = 128 x 128
  int tn_shift;             // log2 of the tiles across N
  int64_t ntiles;
};
constexpr int kTailMaxLevels = 8;
constexpr int kTailMaxPre = 16;
struct TailArgs {
  TailStep pre[kTailMaxPre];  // steps ordered by dependency level (kernel parameters: no load from memory)
  int n_pre;
  int n_levels;
  int level_end[kTailMaxLevels];   // steps [level_end[l-1], level_end[l]) form level l
  // the last step: P[b] = alpha sum_k X[i(b)][k] Y[j(b)][k] for every bin b,
  // i(b) by the runs `rows`, j(b) by `cols` (X and Y: the step's operands,
  // the one with fewer rows as Y)
  const float* X;           // [M][Kd]: read from L2, or (x_range) the rows a slice needs staged
  const float* Y;           // [N][Kd], staged whole in shared memory
  int64_t M, N;
  int Kd;
  int ystride;              // floats per staged Y row (and staged X row)
  int x_range;              // i(b) is monotone in b (X's bits above Y's): a slice's rows are a range
  int x_rows;               // rows of X staged per CTA (0: X read from L2; set at launch)
  float alpha;
  TailPext rows, cols;
  float* P;                 // the bins (FP32), written in bin order
  double* partials;         // [grid]
  double* total;            // nullable: FP64 sum of all bins
};
// Shared memory of the fused launch for n bins (0: does not fit).
size_t select_tail_smem(uint64_t n, const TailArgs& t, int grid, uint64_t* per);
cudaError_t launch_select_tail(void* work, int grid, const TailArgs& t, uint64_t n, int k, double threshold,
                               unsigned long long* bins_out, double* probs_out, int* n_found, int* err,
                               cudaStream_t s);

}  // namespace sqc

// ---- serving-loop hooks into the context (defined with the C ABI) ----------
struct sqc_ctx;
namespace sqc {
void ctx_set_alloc_stream(sqc_ctx* ctx, cudaStream_t s);   // nullptr: synchronous allocation again
int ctx_device(const sqc_ctx* ctx);
void ctx_set_fused(sqc_ctx* ctx, bool on);                  // cfg.fused_query
int32_t ctx_alloc(sqc_ctx* ctx, void** p, size_t bytes);    // budget-checked (SQC_EBUSY when over)
void ctx_free(sqc_ctx* ctx, void* p, size_t bytes);
int32_t ctx_fail(sqc_ctx* ctx, int32_t st, const char* msg);
// sqc_set_qubit_roles in two parts.  query_draft is the host part (roles,
// slicing, contraction order, layouts, maps); it reads only the context's
// configuration and the circuit, so several drafts may run at once on other
// threads while the circuit stays loaded.  query_commit is the device part
// (workspace, uploads) and registers the query; it runs on the thread that
// owns the context and consumes the draft either way.
struct QueryDraft;
const void* ctx_circuit(sqc_ctx* ctx, int64_t circuit);     // nullptr: unknown
int32_t query_draft(const sqc_ctx* ctx, int64_t circuit_id, const void* circuit, const int8_t* roles,
                    QueryDraft** out, std::string* err);
int32_t query_commit(sqc_ctx* ctx, QueryDraft* d, int64_t* query, int32_t* n_active);
void query_draft_free(QueryDraft* d);
}  // namespace sqc
