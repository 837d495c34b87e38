/*
 * sqc.h -- C ABI of the GB300 states-merging reconstruction library.
 *
 * The library reconstructs the output of a cut quantum circuit from its
 * subcircuits' outputs (ScaleQC, arXiv 2207.00933):
 *
 *   P[b] = 2^-K  sum_{e in {I,X,Y,Z}^K}  prod_i  T_i[e|_i, b|_i]      (Eq. 1)
 *
 * where T_i is subcircuit i's output attributed to the I/X/Y/Z labels of its
 * cut edges and merged into bins (Section 4, Algorithm 2), and the sum is
 * evaluated as a sequence of pairwise tensor contractions over the compute
 * graph (Section 6, Fig. 4-5).  All device work is hand-written CUDA for
 * sm_103a; there is no CPU fallback: calls fail with SQC_ECUDA when no
 * usable GPU is present.
 *
 * Conventions for every call:
 *   - Every function returns an sqc_status and never aborts the process.
 *     sqc_last_error() returns a description of the last failure on the
 *     context (or of a failed sqc_create when passed NULL).
 *   - A context is used from one host thread at a time.
 *   - Device work is enqueued on the caller's `stream` (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream) and is
 *     asynchronous unless stated otherwise.
 *   - "device pointer" arguments point to memory on the context's GPU that
 *     the caller owns and keeps alive until the work on `stream` completes.
 *
 * Index conventions (the input layout a QPU runner produces):
 *   - Edges are numbered 0..K-1.  Subcircuit i's incident edges are taken
 *     in ascending edge id.
 *   - Variant index of subcircuit i: one base-4 digit per incident edge, the
 *     lowest edge id most significant.  For an edge leaving i (i measures
 *     the wire) the digit is the measurement basis 0=I, 1=X, 2=Y, 3=Z; for an
 *     edge entering i (i initialises the wire) it is the prepared state
 *     0=|0>, 1=|1>, 2=|+>, 3=|+i>.  X is measured after H, Y after S^dagger
 *     then H; outcome 0 counts +1.
 *   - Output index of subcircuit i: y = x | c << n_i, x little-endian over
 *     i's data qubits in the order given by data_qubit[], c little-endian
 *     over i's outgoing edges in ascending edge id.
 *   - Reconstructed bin index: little-endian over the ACTIVE original
 *     qubits in ascending original index.
 */
#ifndef SQC_H
#define SQC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SQC_API __attribute__((visibility("default")))

typedef int32_t sqc_status;
enum {
  SQC_OK = 0,
  SQC_EINVAL = 1,    /* malformed argument or graph                    */
  SQC_ENOMEM = 2,    /* a device allocation failed                     */
  SQC_ESHAPE = 3,    /* buffer too small / sizes beyond the limits     */
  SQC_ECUDA = 4,     /* a CUDA call failed (includes "no GPU")         */
  SQC_ETIMEOUT = 5,  /* a bounded device wait ran out                  */
  SQC_EBUSY = 6,     /* admission refused: over the HBM budget         */
  SQC_ENOTFOUND = 7  /* unknown circuit or query handle                */
};

typedef enum { SQC_F32 = 0, SQC_F64 = 1 } sqc_dtype;

/* Arithmetic of the contraction steps.  FP32: SIMT FP32 FMA.  SPLIT_BF16:
 * every operand split into three BF16 terms (hi + mid + lo) and multiplied
 * on the tcgen05 tensor cores with FP32 accumulation, keeping the six
 * products of order <= 2 (about FP32 accuracy). */
typedef enum { SQC_PREC_FP32 = 0, SQC_PREC_SPLIT_BF16 = 1 } sqc_precision;

/* Qubit roles (Section 4): ACTIVE qubits index the output bins, MERGED
 * qubits are summed inside each bin, ZOOM0/ZOOM1 qubits are fixed to 0/1
 * (the bin chosen by an earlier recursion). */
enum { SQC_ROLE_ACTIVE = 0, SQC_ROLE_MERGED = 1, SQC_ROLE_ZOOM0 = 2, SQC_ROLE_ZOOM1 = 3 };

typedef struct sqc_ctx sqc_ctx;
typedef int64_t sqc_circuit_id;
typedef int64_t sqc_query_id;

typedef struct {
  /* Device memory the context may hold for resident subcircuit tensors and
   * query plans; 0 = no limit.  Exceeding it makes loads and role settings
   * fail with SQC_EBUSY (admission by HBM footprint). */
  uint64_t hbm_budget_bytes;
  /* Largest number of active qubits a query may ask for (2^this bins). */
  int32_t max_active_qubits;
  /* Number of cut edges K from which the last contraction step sums its
   * shared index in FP32 chunks added up in FP64 (the cross-chunk sum). */
  int32_t fp64_chunk_min_edges;
  /* FP32 terms summed per chunk before the FP64 addition (>= 16, power of 2). */
  int32_t chunk_terms;
  /* First-level index slicing (Section 6.3): number of cut edges to write
   * out explicitly, chosen greedily as the edge whose slicing shrinks the
   * total size of the subcircuit tensors most (ties: lowest edge id).  Each
   * query then runs 4^slice_edges smaller contractions whose results are
   * added into the output (in FP64 for FP64 outputs).  0 = no slicing. */
  int32_t slice_edges;
  /* Selection (sqc_top_bins): 1 = hold one 32-bit key word per value in
   * shared memory, one slice per SM, when they fit (up to ~7 million FP32
   * or FP64 values on 152 SMs; one read of the input); 0 = always the
   * streaming kernel. */
  int32_t select_resident;
  /* Merge pyramid (1 = on, default 0): after every attribution, also keep
   * the partial marginals of each A_i over its 1, 2, ..., n_i lowest
   * storage bits (pairwise sums; about as much memory again as A_i, counted
   * in the HBM budget).  A query whose merged qubits of a subcircuit are
   * exactly its highest data qubits (the recursion's roles) then reads
   * 4^{k_i} 2^{a_i} values instead of 4^{k_i} 2^{a_i + m_i}.  Worth it when
   * many queries share one load; it adds a pass over A_i to every load and
   * update. */
  int32_t merge_pyramid;
  /* Budget-driven index slicing (Section 6.3), applied after slice_edges:
   * first level -- keep writing out the cut edge that shrinks
   * sum_i 4^{k_i} 2^{a_i} (the merged subcircuit tensors, in floats) most
   * until that sum is <= 2^slice_input_log2; second level -- then keep
   * writing out the edge that shrinks the largest intermediate tensor of
   * the contraction most (ties: smaller input sum, then lower edge id)
   * until every intermediate is <= 2^slice_intermediate_log2 floats.
   * 0 = off.  At most 8 edges are sliced in all; a query whose budgets
   * would need more fails with SQC_ESHAPE. */
  int32_t slice_input_log2;
  int32_t slice_intermediate_log2;
  /* Split-BF16 steps large enough to fill every SM with 256 x 256 output
   * units (1 = on): run them on 2-SM pairs (tcgen05.mma.cta_group::2,
   * M = 256; each SM of a pair loads its own half of both operands, so a
   * pair reads every operand tile from L2 once).  0 = one SM per unit. */
  int32_t tc_pairs;
  /* Limit, in milliseconds, of every bounded device wait (the batched
   * launch's dependency waits, the tensor-core pipeline's barrier waits);
   * a wait that runs out records SQC_ETIMEOUT and the kernel drains and
   * returns.  0 = the default, 2000 ms. */
  int32_t wait_limit_ms;
  /* FP32 reconstructions (1 = on, default 0): the merge and every
   * contraction step of a query run as ONE persistent launch whose merge
   * blocks and step tiles wait (bounded) only for the tensors they read,
   * instead of one launch per stage; the bins are the same bit for bit.
   * The first FP32 reconstruct of a query into each output format builds
   * that launch's work list (allocates).  Sliced queries and split-BF16
   * keep one launch per stage. */
  int32_t fused_query;
  /* Programmatic dependent launch (1 = on, default 1): each kernel of a
   * call is launched while the previous kernel on the stream finishes; it
   * sets up what depends only on its parameters and shared memory, then
   * waits on the device (griddepcontrol.wait) before its first access to
   * memory the previous kernel may write.  Results do not change.  On the
   * 2^20-bin one-call step it saves 1-2 us of the 42 (the fused selection
   * launch's prologue overlaps the attribution-merge); on the per-stage
   * chains it measured within noise. */
  int32_t pdl;
  /* Pairwise contraction order of new query plans (Section 6.2 cost, the
   * multiplications of each step): SQC_ORDER_GREEDY (default) pairs the
   * connected tensors of fewest multiplications one step at a time;
   * SQC_ORDER_MIN_MULT takes the order with the fewest multiplications over
   * all pairwise trees (exact search over subsets, queries of up to 14
   * subcircuits; larger ones fall back to greedy).  Fewer multiplications
   * do not always mean less time for small, latency-bound steps:
   * sqc_query_autotune and sqc_batch_autotune choose by measurement. */
  int32_t contraction_order;
  /* sqc_reconstruct_select (1 = on, default 1): when a query's FP32 plan
   * allows it (sqc_query_fused_select), the contraction steps, the bins and
   * their selection run in ONE cooperative launch -- the steps before the
   * last level by level between grid barriers, then every CTA computes its
   * slice of the last step's bins into shared memory, writes them, and the
   * resident selection runs on them without reading them back.  Results
   * are those of the per-stage launches (the bins and the selected bins bit
   * for bit; the FP64 sum within rounding).  0 = per-stage launches. */
  int32_t fused_select;
} sqc_config;

enum { SQC_ORDER_GREEDY = 0, SQC_ORDER_MIN_MULT = 1 };

/* Compute graph (Section 5, Fig. 3d).  Vertices are subcircuits 0..n_C-1;
 * edge k runs from subcircuit edge_up[k] (which measures the wire) to
 * edge_down[k] (which initialises it).  Subcircuit i owns n_data[i] data
 * qubits; data_qubit[] lists them, subcircuit-major, as original qubit
 * indices; every original qubit 0..n_qubits-1 appears exactly once.
 * Limits: n_C <= 64, K <= 60, 4^{k_i} * 2^{w_i} < 2^40 per subcircuit. */
typedef struct {
  int32_t n_qubits;
  int32_t n_subcircuits;
  int32_t n_edges;
  const int32_t* edge_up;     /* [n_edges]       */
  const int32_t* edge_down;   /* [n_edges]       */
  const int32_t* n_data;      /* [n_subcircuits] */
  const int32_t* data_qubit;  /* [n_qubits]      */
} sqc_graph;

/* Fill `cfg` with the defaults (no budget, 32 active qubits, FP64 chunking
 * from 12 edges, 256 terms per chunk, resident selection; everything else
 * off). */
SQC_API void sqc_default_config(sqc_config* cfg);

/* Create a context on CUDA device `device`.  cfg may be NULL (defaults).
 * Fails with SQC_ECUDA when the device cannot be used.  *out is NULL on
 * failure; sqc_last_error(NULL) then says why. */
SQC_API sqc_status sqc_create(sqc_ctx** out, int device, const sqc_config* cfg);

/* Destroy a context and free every device buffer it holds (synchronises
 * the device first).  NULL is ignored. */
SQC_API void sqc_destroy(sqc_ctx* ctx);

/* Description of the last failure on ctx (NULL: of the last sqc_create). */
SQC_API const char* sqc_last_error(const sqc_ctx* ctx);

/* Load one circuit: validate the graph, copy it, and attribute every
 * subcircuit's variant outputs to its cut-edge labels (Eq. 1; the weights
 * of Section 2.1 with the I/X/Y/Z expansion of Peng et al.), producing the
 * resident tensors A_i[4^{k_i}][2^{n_i}] (FP32) that later queries merge.
 *   probs[i]: subcircuit i's outputs, [4^{k_i}][2^{w_i}] row-major,
 *             w_i = n_data[i] + #outgoing edges of i, in `dtype`;
 *             host pointers if probs_on_device == 0 (copied, then
 *             synchronised; while `stream` is being captured into a CUDA
 *             graph there is no synchronisation, and the buffers must be
 *             pinned and stay valid for every replay), else device
 *             pointers (read on `stream`).  Host inputs that are all
 *             mapped pinned memory (16-byte aligned, sizes multiples of
 *             16 bytes) are copied by one launch of an SM copy kernel;
 *             other host memory by one copy per buffer.
 * On success *out_id names the circuit until sqc_unload. */
SQC_API sqc_status sqc_load_subcircuit_outputs(sqc_ctx* ctx, const sqc_graph* graph,
                                               const void* const* probs, sqc_dtype dtype,
                                               int probs_on_device, sqc_circuit_id* out_id,
                                               void* stream);

/* Replace a loaded circuit's subcircuit outputs with new ones of the same
 * shapes (the next recursion's QPU results, Algorithm 1) and re-run the
 * attribution; allocates nothing.  Same argument meaning as above. */
SQC_API sqc_status sqc_update_subcircuit_outputs(sqc_ctx* ctx, sqc_circuit_id id,
                                                 const void* const* probs, sqc_dtype dtype,
                                                 int probs_on_device, void* stream);

/* Free a circuit and every query made on it. */
SQC_API sqc_status sqc_unload(sqc_ctx* ctx, sqc_circuit_id id);

/* Fix the qubit roles of one reconstruction (one recursion of Algorithm 1,
 * bins assigned as in Algorithm 2) and plan it: per-subcircuit merge,
 * contraction order (greedy on the Section 6.2 cost), layouts, workspace.
 *   roles: [n_qubits] of SQC_ROLE_*.
 * Outputs: *out_q (query handle), *n_active (log2 of the bin count).
 * Fails with SQC_ESHAPE when n_active > cfg.max_active_qubits and with
 * SQC_EBUSY when the plan's workspace would exceed the HBM budget. */
SQC_API sqc_status sqc_set_qubit_roles(sqc_ctx* ctx, sqc_circuit_id id, const int8_t* roles,
                                       sqc_query_id* out_q, int32_t* n_active);

/* Release a query and its workspace. */
SQC_API sqc_status sqc_release_query(sqc_ctx* ctx, sqc_query_id q);

/* Reconstruct the bin probabilities of query q (Eq. 1 by compute-graph
 * contraction, Section 6):
 *   out_bins: device pointer, 2^{n_active} values of out_dtype, bin index
 *             as in the header comment; out_bytes its size (checked).
 *   total_prob: nullable device pointer to one double; receives the FP64
 *             sum of all bins (the per-level probability check).
 * Merges every subcircuit (Algorithm 2), runs the planned contraction
 * steps, scales by 2^-K, writes the bins.  With out_dtype = SQC_F64 and
 * K >= cfg.fp64_chunk_min_edges the last step's shared index is summed in
 * FP32 chunks accumulated in FP64.  Asynchronous on `stream`. */
SQC_API sqc_status sqc_reconstruct(sqc_ctx* ctx, sqc_query_id q, sqc_precision precision,
                                   void* out_bins, sqc_dtype out_dtype, uint64_t out_bytes,
                                   double* total_prob, void* stream);

/* One recursion step on fresh subcircuit outputs (Algorithm 1 runs the
 * subcircuits again for every recursion; states merging, Section 4, applied
 * while attributing, Eq. 1): the bins of query q for the outputs `probs`
 * (layout, dtype and probs_on_device as in sqc_load_subcircuit_outputs),
 * with the attribution fused into the merge -- per subcircuit only the
 * states the query keeps (zoomed qubits at their fixed values) are
 * attributed, in shared-memory tiles that sum the merged qubits and write
 * the merged tensors T_i directly; no A_i is written or read.  Then the
 * contraction steps and outputs as sqc_reconstruct.  The circuit's
 * resident tensors are NOT changed: other queries keep using the outputs
 * of the last load or update.
 * probs_on_device == 2 (this call and sqc_reconstruct_select only): host
 * memory mapped for the device (pinned by cudaHostAlloc / cudaHostRegister
 * with unified addressing, as a framework's pinned tensors are): the
 * attribution reads the kept states in place over the host link, with no
 * staging copy and no synchronisation -- keep the buffers unchanged until
 * the stream has passed the call.  Other host memory fails with
 * SQC_EINVAL.  (On the 2^20-bin step this measured slower than staging,
 * 0.16 against 0.09 ms end to end: the attribution's latency-bound loads
 * each cross the host link.)
 * Applies when every subcircuit's roles follow the recursion's pattern
 * (data qubits in data_qubit order: the zoomed ones first, then the active
 * ones, then at most 8 merged ones -- what sqc_recursion_roles assigns),
 * no subcircuit has more than 7 incoming cut edges, and the query is not
 * sliced; otherwise it fails with SQC_EINVAL (then use
 * sqc_update_subcircuit_outputs + sqc_reconstruct).  Host inputs are
 * staged in the circuit's staging buffer and synchronised as in an update.
 * Asynchronous on `stream` for device inputs. */
SQC_API sqc_status sqc_reconstruct_outputs(sqc_ctx* ctx, sqc_query_id q, const void* const* probs, sqc_dtype dtype,
                                           int probs_on_device, sqc_precision precision, void* out_bins,
                                           sqc_dtype out_dtype, uint64_t out_bytes, double* total_prob,
                                           void* stream);

/* One recursion step of Algorithm 1 in one call: the bins of query q (as
 * sqc_reconstruct when probs is NULL, as sqc_reconstruct_outputs on the
 * fresh outputs `probs` otherwise; same arguments) followed by the
 * selection of their largest bins (as sqc_top_bins on out_bins with
 * n = 2^{n_active} values of out_dtype; same k, threshold and outputs).
 * With cfg.fused_select and an FP32 plan that allows it
 * (sqc_query_fused_select > 0), precision SQC_PREC_FP32 and out_dtype
 * SQC_F32, the contraction steps, the bins and the selection run in one
 * cooperative launch after the merges: the bins are computed into shared
 * memory slice by slice, written once and selected without being read
 * back.  Every output equals that of the separate calls bit for bit,
 * except total_prob (the same FP64 sum in another order: within
 * rounding).  Errors as the separate calls.  Asynchronous on `stream`
 * (host inputs: as sqc_reconstruct_outputs). */
SQC_API sqc_status sqc_reconstruct_select(sqc_ctx* ctx, sqc_query_id q, const void* const* probs, sqc_dtype dtype,
                                          int probs_on_device, sqc_precision precision, void* out_bins,
                                          sqc_dtype out_dtype, uint64_t out_bytes, double* total_prob, int32_t k,
                                          double threshold, uint64_t* bins_out, double* probs_out,
                                          int32_t* n_found, void* stream);

/* How many contraction steps of query q's FP32 plan sqc_reconstruct_select
 * runs inside its fused selection launch (all of them), or 0 when it runs
 * per-stage launches for this query: the plan is sliced, the last step's
 * shared index exceeds 64 values or its bin maps are not plain bit
 * deposits, the steps span more than 8 dependency levels, the bins plus the
 * last step's second operand do not fit the shared memory of one CTA per
 * SM, or cfg.fused_select / cfg.select_resident is off.  Host values. */
SQC_API sqc_status sqc_query_fused_select(sqc_ctx* ctx, sqc_query_id q, int32_t* n_steps);

/* Select bins (Algorithm 1: keep the largest bins): among the n values at
 * device pointer `probs` (dtype), those >= threshold, ordered by value
 * descending then bin index ascending, at most k (1 <= k <= 4096).
 * Outputs are device pointers: bins_out[k] (uint64), probs_out[k] (double),
 * n_found[1] (int32).  Uses query q's workspace; calls on the same query
 * must not overlap on the GPU.  Asynchronous on `stream`. */
SQC_API sqc_status sqc_top_bins(sqc_ctx* ctx, sqc_query_id q, const void* probs, sqc_dtype dtype,
                                uint64_t n, int32_t k, double threshold, uint64_t* bins_out,
                                double* probs_out, int32_t* n_found, void* stream);

/* Batched recursion level (one persistent launch per phase).
 *
 * A batch groups queries -- bins of possibly different loaded circuits,
 * with uneven active-qubit counts -- whose reconstructions run in
 * persistent kernel launches: every query's merge blocks and contraction
 * tiles form one dependency-ordered work list taken by persistent CTAs,
 * each item waiting (bounded) only for the tensors it reads.  The result of
 * query qs[j] goes to outs[j] (device, 2^{n_active} values of out_dtype) and
 * its FP64 probability sum to totals[j] (device array of n doubles, may be
 * NULL), exactly as sqc_reconstruct(..., precision, ...) would write them.
 * With SQC_PREC_SPLIT_BF16 the steps that each query's split-BF16 plan puts
 * on the tensor cores (sqc_query_tc_steps) run as tcgen05 launches between
 * phases -- phase j is one persistent launch of the merges and SIMT steps
 * whose inputs are complete by then, followed by the tensor-core steps
 * whose inputs it completes; the other steps run FP32 in the persistent
 * launches (mixed precision per step).  With SQC_PREC_FP32 there is one
 * phase and one launch.  Every query needs at least two subcircuits.
 *   sqc_batch_create: plans the work lists and allocates their device
 *     state (the output pointers are fixed here, so sqc_batch_run does no
 *     host work and can be replayed from a CUDA graph);
 *   sqc_batch_run: the launches on `stream`;
 *   sqc_batch_release: frees the batch (not the queries).
 * A query's workspace is shared by its batch and its single-query calls:
 * do not run both at once.  sqc_batch_status synchronises the device and
 * returns SQC_ETIMEOUT if a bounded wait of the batch ever gave up. */
typedef int64_t sqc_batch_id;
SQC_API sqc_status sqc_batch_create(sqc_ctx* ctx, int32_t n, const sqc_query_id* qs, void* const* outs,
                                    sqc_dtype out_dtype, double* totals, sqc_precision precision,
                                    sqc_batch_id* out_b);
SQC_API sqc_status sqc_batch_run(sqc_ctx* ctx, sqc_batch_id b, void* stream);
SQC_API sqc_status sqc_batch_status(sqc_ctx* ctx, sqc_batch_id b);
SQC_API sqc_status sqc_batch_release(sqc_ctx* ctx, sqc_batch_id b);
/* Failure-detection hook (the paper has no counterpart), host side only:
 * with on = 1, raises by one the completion count that the batch's last
 * intermediate tensor must reach, so that the items reading it can never
 * start; the next sqc_batch_run then ends by the bounded wait running out
 * (after cfg.wait_limit_ms), every CTA drains and returns, and
 * sqc_batch_status reports SQC_ETIMEOUT.  on = 0 restores the batch.
 * Synchronous (uploads the counts); the batch must not be running.  Fails
 * with SQC_EINVAL for a batch without intermediate tensors. */
SQC_API sqc_status sqc_batch_inject_stall(sqc_ctx* ctx, sqc_batch_id b, int32_t on);
/* Project-written autotuner of the batched launch (the paper has no
 * counterpart): for each contraction order (SQC_ORDER_GREEDY, then
 * SQC_ORDER_MIN_MULT) it plans the n queries again under that order and
 * builds the batch of sqc_batch_create(n, qs, outs, out_dtype, totals)
 * under each tile policy -- 0 by occupancy, 1 small 32 x 32 tiles, 2 large
 * 64 x 64 / 128 x 64 tiles -- times `reps` launches of each on the default
 * stream (CUDA events, after one warm-up launch) and releases it.  The
 * fastest (order, policy) wins: the queries keep plans under that order
 * and the policy becomes the context's choice for later batches (also the
 * serving loop's).  ms[6] (may be NULL) receives the mean time per launch,
 * order-major (ms[3 * order + policy]).  Under one order the bins do not
 * depend on the policy (each bin is summed in the same order); another
 * contraction order rounds differently.  The outputs and totals end as the
 * chosen order and policy write them (one more launch after the timing).
 * Synchronises the device. */
SQC_API sqc_status sqc_batch_autotune(sqc_ctx* ctx, int32_t n, const sqc_query_id* qs, void* const* outs,
                                      sqc_dtype out_dtype, double* totals, int32_t reps, int32_t* best_policy,
                                      int32_t* best_order, float* ms);

/* Contraction-order autotuner of one query (the paper has no counterpart;
 * Section 6.2 counts multiplications, which does not rank orders of
 * latency-bound steps): plans query q under SQC_ORDER_GREEDY and under
 * SQC_ORDER_MIN_MULT, times `reps` reconstructions of each into out_bins
 * (arguments as in sqc_reconstruct, on the default stream, after a
 * warm-up) and keeps the plan of the faster order (*best_order).  ms[2]
 * (may be NULL): mean ms per reconstruction under each order (equal when
 * both orders give the same plan).  Synchronises the device; allocates. */
SQC_API sqc_status sqc_query_autotune(sqc_ctx* ctx, sqc_query_id q, sqc_precision precision, void* out_bins,
                                      sqc_dtype out_dtype, uint64_t out_bytes, int32_t reps, int32_t* best_order,
                                      float* ms);

/* Serving loop: continuous batching of zoom queries (one recursion level
 * each) against circuits already loaded on the context.
 *
 * sqc_server_create starts one server thread that owns `ctx` from then on
 * (do not call other functions on ctx until sqc_server_destroy returns).
 * Clients call sqc_server_submit from any thread; the server admits waiting
 * requests in arrival order while their plans and outputs fit the context's
 * HBM budget (sqc_config.hbm_budget_bytes; a request that does not fit waits
 * until launches retire), and launches each group of admitted requests as
 * one persistent batch (plain = 1: one FP32 reconstruction per request,
 * one launch per stage -- the server turns cfg.fused_query off) on
 * one of n_streams non-blocking streams, so launches overlap; requests that
 * arrive meanwhile go into the next free stream.  A request larger than the
 * whole budget fails with SQC_EBUSY; requests still waiting when the server
 * is destroyed are cancelled (state failed, SQC_EBUSY).  All allocations, uploads
 * and frees are stream-ordered: the loop never synchronises the device.
 * The host part of the waiting requests' plans (contraction order, layouts,
 * maps) runs on up to 8 short-lived planner threads (half the host's
 * hardware threads) per admission round; the rest stays on the server
 * thread. 
 * Results are FP32 bins, identical to sqc_reconstruct(SQC_PREC_FP32) of the
 * same query run alone. */
typedef struct sqc_server sqc_server;
typedef struct {
  int32_t max_batch;   /* most requests per launch (default 64)           */
  int32_t n_streams;   /* launches in flight at once, 1..32 (default 4)   */
  int32_t plain;       /* 1: one reconstruction per request (no batching) */
  int32_t reserved[5];
} sqc_server_config;

SQC_API void sqc_server_default_config(sqc_server_config* cfg);
SQC_API sqc_status sqc_server_create(sqc_ctx* ctx, const sqc_server_config* cfg, sqc_server** out);
/* roles: [n_qubits] as in sqc_set_qubit_roles; *ticket identifies the request. */
SQC_API sqc_status sqc_server_submit(sqc_server* srv, sqc_circuit_id circuit, const int8_t* roles, int32_t n_qubits,
                                     int64_t* ticket);
/* *state: 0 waiting, 1 running, 2 done, 3 failed (the call then returns the
 * failure), 4 collected; *latency_us: submit-to-completion time once done. */
SQC_API sqc_status sqc_server_poll(sqc_server* srv, int64_t ticket, int32_t* state, double* latency_us,
                                   int32_t* n_active);
/* Copy a done request's 2^{n_active} FP32 bins to host_out (capacity in
 * values); the server moved them to host memory when the launch retired.
 * SQC_EBUSY if not done yet. */
SQC_API sqc_status sqc_server_result(sqc_server* srv, int64_t ticket, float* host_out, uint64_t capacity);
/* Block until no request is waiting or running (SQC_ETIMEOUT after timeout_s). */
SQC_API sqc_status sqc_server_drain(sqc_server* srv, double timeout_s);
SQC_API sqc_status sqc_server_stats(sqc_server* srv, int64_t* launches, int64_t* admitted, int64_t* busy_refusals);
/* Finish the requests in flight, free everything the server holds, stop the thread. */
SQC_API void sqc_server_destroy(sqc_server* srv);

/* Allocation-free bin selection.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code
 * embedded in a host application that owns every device allocation, or a
 * latency-critical loop in which a cudaMalloc (which can synchronise the
 * device) is not acceptable.  It returns exactly what sqc_top_bins returns
 * for the same arguments, needs no context and no query, and allocates
 * nothing: its scratch is one static device array of about 140 KiB in the
 * library (held on every GPU that loads the library until the process
 * exits).
 *   device: the GPU that holds `probs` and the outputs (made current for
 *           the call).  The first call on a device only looks up the
 *           array's device address (cudaGetSymbolAddress) and keeps it for
 *           later calls; make that first call before any stream capture.
 *           The kept address belongs to the device's primary context: after
 *           a cudaDeviceReset the library must be reloaded before this entry
 *           point is used again on that device.
 *   k must be in [1, 4096] (the scratch's capacity); larger k fails with
 *   SQC_ESHAPE.  Other arguments as in sqc_top_bins.
 * Every call shares the one array: calls whose GPU work may overlap (other
 * streams, other host threads) race and must be serialised by the caller.
 * Errors are reported through sqc_last_error(NULL). */
SQC_API sqc_status sqc_top_bins_noalloc(int device, const void* probs, sqc_dtype dtype, uint64_t n, int32_t k,
                                        double threshold, uint64_t* bins_out, double* probs_out,
                                        int32_t* n_found, void* stream);

/* Device memory the context holds now (resident circuits, plans, batches,
 * workspaces) and its budget (0 = none); host values. */
SQC_API sqc_status sqc_memory_info(const sqc_ctx* ctx, uint64_t* held_bytes, uint64_t* budget_bytes);

/* The cut edges query q slices (Section 6.3), in the order the greedy rule
 * chose them: *n_sliced values written to edges (capacity cap). */
SQC_API sqc_status sqc_query_slices(const sqc_ctx* ctx, sqc_query_id q, int32_t* n_sliced, int32_t* edges,
                                    int32_t cap);

/* Introspection of a planned query (host values, no device work):
 * n_steps contraction steps; flops = sum of 2*M*N*K over the steps;
 * merge_bytes = bytes the merge reads and writes; work_bytes = device
 * workspace held. */
SQC_API sqc_status sqc_query_info(const sqc_ctx* ctx, sqc_query_id q, int32_t* n_steps, double* flops,
                                  double* merge_bytes, uint64_t* work_bytes);

/* Split-BF16 plan of query q (built by its first SPLIT_BF16 reconstruct;
 * 0 and 0 before that): *n_tc of its *n_steps contraction steps run on the
 * tcgen05 tensor cores, the others (M or N below 128) in FP32 on the SIMT
 * cores.  Host values, no device work.  n_steps may be NULL. */
SQC_API sqc_status sqc_query_tc_steps(const sqc_ctx* ctx, sqc_query_id q, int32_t* n_tc, int32_t* n_steps);

/* Shape of contraction step `step` (0-based, in launch order) of query q:
 * the step computes C[M][N] = sum over Kd of A[M][Kd] * B[N][Kd]
 * (Section 6.1, Fig. 4a).  Host values, no device work. */
SQC_API sqc_status sqc_query_step(const sqc_ctx* ctx, sqc_query_id q, int32_t step, int64_t* M, int64_t* N,
                                  int64_t* Kd);

/* States assignment (Section 4, Algorithm 2, target-bin loop): while the
 * product of the bin counts l'_i exceeds M, halve (rounding up) the largest,
 * ties to the lowest subcircuit index.  l[n_subcircuits] in, l_out out.
 * Host only: needs no context and no GPU. */
SQC_API sqc_status sqc_assign_states(int32_t n_subcircuits, const uint64_t* l, uint64_t M, uint64_t* l_out);

/* Qubit roles of one recursion (Algorithm 1 with Algorithm 2's
 * assignment): zoom[n_qubits] marks the qubits earlier recursions fixed
 * (SQC_ROLE_ZOOM0/ZOOM1; any other value = free).  Per subcircuit the free
 * data qubits, in the graph's data_qubit order, enumerate its states j; with
 * l'_i = 2^{a_i} bins, j % l'_i makes the first a_i of them active, the rest
 * merged.  roles[n_qubits] out.  Host only. */
SQC_API sqc_status sqc_recursion_roles(const sqc_graph* graph, const int8_t* zoom, uint64_t M, int8_t* roles);

/* Host-only preview of the FP32 plan that sqc_set_qubit_roles builds for
 * `roles` on a circuit of this graph under configuration `cfg` (NULL:
 * defaults): first-level slicing (Section 6.3; by `slice_edges` or by the
 * budgets `slice_input_log2` / `slice_intermediate_log2`) and the greedy
 * pairwise contraction order on the Section 6.2 cost (connected pairs
 * first, then fewest multiplications, then the smaller result).  Needs no
 * GPU and allocates no device memory.
 *   n_steps (out): contraction steps (n_subcircuits - 1);
 *   steps: nullable host array [cap_steps][3] of (M, N, K) per step in
 *          execution order -- C[M x N] = A[M x K] B[N x K]^T, K = 4^{shared
 *          cut edges}; the last step's M x N is 2^{n_active};
 *   n_sliced (out), sliced: nullable [cap_sliced] sliced edge ids in the
 *          order they were chosen;
 *   flops: nullable, 2 M N K summed over the steps of one slice;
 *   work_bytes: nullable, the device workspace sqc_set_qubit_roles would
 *          allocate for the query's FP32 plan;
 *   err: nullable buffer of err_len bytes receiving the reason of a
 *          failure (NUL-terminated, truncated).
 * Errors as sqc_set_qubit_roles (SQC_EINVAL for a bad graph, role or
 * configuration, SQC_ESHAPE for an unreachable slicing budget or too many
 * active qubits). */
SQC_API sqc_status sqc_plan_preview(const sqc_graph* graph, const int8_t* roles, const sqc_config* cfg,
                                    int32_t* n_steps, int64_t* steps, int32_t cap_steps, int32_t* n_sliced,
                                    int32_t* sliced, int32_t cap_sliced, double* flops, uint64_t* work_bytes,
                                    char* err, int32_t err_len);

/* Stage timing (tracing).  When enabled, the library records a pair of CUDA
 * events on the caller's stream around each stage it launches and counts
 * its kernel launches.  Stages: */
enum {
  SQC_STAGE_ATTRIBUTE = 0,  /* attribution of variant outputs (load/update) */
  SQC_STAGE_MERGE = 1,      /* merge/zoom of all subcircuits                */
  SQC_STAGE_CONTRACT = 2,   /* contraction steps except the last            */
  SQC_STAGE_FINAL = 3,      /* last contraction step (scaled bins, K7 sum)  */
  SQC_STAGE_SELECT = 4,     /* bin selection                                 */
  SQC_STAGE_COUNT = 5
};

/* Turn stage timing on (1) or off (0); turning it on clears the record.
 * Mode 2 is for work captured into a CUDA graph: the event pairs recorded
 * during capture become graph nodes and are kept; every sqc_profile_read
 * then reports the times of the most recent replay, and *launches the
 * kernels recorded during capture (one replay's worth). */
SQC_API sqc_status sqc_profile_enable(sqc_ctx* ctx, int on);

/* Read (and, outside mode 2, clear) the record: ms[SQC_STAGE_COUNT] total milliseconds per
 * stage, calls[SQC_STAGE_COUNT] how many times each stage ran, *launches the
 * number of kernels launched.  Synchronises with the recorded events.  Any
 * output may be NULL. */
SQC_API sqc_status sqc_profile_read(sqc_ctx* ctx, double* ms, int64_t* calls, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* SQC_H */
