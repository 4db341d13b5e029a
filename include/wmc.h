/*
 * wmc.h -- C ABI of the B300 execution stage for tensor-network weighted
 * model counting (Dudek & Vardi, "Parallel Weighted Model Counting with
 * Tensor Networks").
 *
 * The library reduces a weighted CNF to a tensor network (Thm 3.2), plans a
 * contraction tree with a portfolio of elimination orders (Sec. 3.3), and
 * executes the tree on one GPU as a post-order walk of pairwise
 * contractions (Algorithm 2), each a hand-written sm_103a CUDA kernel.
 *
 * Conventions for every entry point
 *   - Every call returns an int status (WMC_OK = 0 or a negative WMC_E*
 *     code, or WMC_PENDING = 1 from wmc_poll).  Nothing throws across the
 *     ABI.  wmc_last_error() returns a thread-local message for the last
 *     failing call on the calling thread.
 *   - The library owns every handle it returns and copies every input
 *     array it is given; callers may free their arrays after the call.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device.  Streams are cudaStream_t passed
 *     as void* (NULL = the legacy default stream).
 *   - Weights are float64.  w_pos[v] = W(x_{v+1}, 1) and w_neg[v] =
 *     W(x_{v+1}, 0) (Def. 2.1).  Evidence is expressed as a zero weight.
 *   - Query batches are query-major: element [q * n_vars + v].
 *   - Results are wmc_result records: value = mant * 2^exp2, so counts far
 *     outside the float64 range (grid formulas reach 1e-956) are exact in
 *     range.
 */
#ifndef WMC_B300_H
#define WMC_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define WMC_OK 0
#define WMC_PENDING 1           /* wmc_poll: the query has not finished      */
#define WMC_EINVAL (-1)         /* malformed argument (bad literal, size ...) */
#define WMC_ENOMEM (-2)         /* host or device allocation failed          */
#define WMC_EPLAN_TOO_BIG (-3)  /* plan exceeds max_rank_cap / memory budget */
#define WMC_ECUDA (-4)          /* a CUDA runtime call failed                */
#define WMC_ETIMEOUT (-5)       /* a bounded wait gave up                    */
#define WMC_EUNKNOWN_TICKET (-6)/* wmc_poll: ticket never issued or consumed */
#define WMC_ESHUTDOWN (-7)      /* server is shutting down                   */

/* Precision of the contraction path. */
#define WMC_FP64 0          /* float64 mantissas, per-tensor pow2 exponents  */
#define WMC_SCALED_FP32 1   /* float32 mantissas with float32 accumulation,
                               per-(tensor, query) pow2 exponents; the root
                               contraction accumulates in float64          */

/* Elimination-order heuristics for wmc_plan. */
#define WMC_ORDER_BEST 0       /* portfolio below, keep the lowest max-rank */
#define WMC_ORDER_MINFILL 1    /* min-fill, ties: degree then lowest id     */
#define WMC_ORDER_MINDEGREE 2  /* min-degree, ties: lowest id               */
#define WMC_ORDER_SWEEP 3      /* level sweep of a multi-source BFS         */
#define WMC_ORDER_GIVEN 4      /* caller-supplied order (wmc_plan_opts.order) */

/* wmc_result.flags */
#define WMC_FLAG_EXACT_INT 0x1u      /* every weight was 1 and the count is
                                        below 2^53: mant*2^exp2 is exact     */
#define WMC_FLAG_FP32_FLUSH 0x2u     /* a float32 product of nonzero entries
                                        may have underflowed (conservative:
                                        set whenever the smallest nonzero
                                        scaled operands' product is below the
                                        smallest normal float)                */
#define WMC_FLAG_NO_BOUND 0x4u       /* a weight was negative: rel_err_bound
                                        does not apply                        */
#define WMC_FLAG_DEVICE_TIMEOUT 0x8u /* a bounded wait inside a kernel gave up;
                                        the value is invalid (wmc_execute and
                                        the server report WMC_ETIMEOUT)       */
#define WMC_FLAG_FELL_BACK_FP64 0x10u /* the query's scaled-FP32 walk may have
                                        flushed (WMC_FLAG_FP32_FLUSH), so
                                        wmc_execute / wmc_execute_slices ran
                                        it again on the same tree in FP64;
                                        the value and bound are FP64's        */

typedef struct wmc_network wmc_network_t;
typedef struct wmc_plan wmc_plan_t;
typedef struct wmc_server wmc_server_t;
typedef struct wmc_batch wmc_batch_t;

typedef struct {
  double mant;          /* value = mant * 2^exp2, |mant| in [0.5, 1) or 0   */
  int64_t exp2;
  double log10;         /* log10(|value|), -inf for 0                        */
  uint32_t flags;       /* WMC_FLAG_*                                        */
  uint32_t reserved;
  double rel_err_bound; /* a-priori relative error bound for nonnegative
                           weights: gamma_d = d*u/(1-d*u), u the unit
                           roundoff, d the most roundings on any path from
                           a leaf to the root                               */
} wmc_result;

/* Reduction: Thm 3.2.  Builds the network {A_x} u {B_C} of a CNF with n_vars
 * variables and n_clauses clauses.  lits holds DIMACS literals (+v / -v,
 * 1 <= v <= n_vars) and clause i is lits[clause_off[i] .. clause_off[i+1]).
 * Repeated literals are merged and tautological clauses dropped (neither
 * changes W); an empty clause makes W = 0.  w_pos / w_neg (host, n_vars
 * each) are the default weights used by wmc_execute when it is given no
 * weights; they may be NULL (all weights 1).  The COPY tensors A_x are kept
 * in hyperedge form: each variable is one index shared by every tensor that
 * mentions it, and A_x becomes the weight vector [W(x,0), W(x,1)].
 * A clause may have any number of literals; one over more than 62
 * variables is planned only with clause factoring
 * (wmc_plan_opts.factor_clauses_above).
 * Errors: WMC_EINVAL for a literal 0 or |lit| > n_vars, negative sizes or a
 * non-monotone clause_off; WMC_ENOMEM. */
int wmc_network_create(int32_t n_vars, int64_t n_clauses, const int32_t *lits,
                       const int64_t *clause_off, const double *w_pos,
                       const double *w_neg, wmc_network_t **out);
void wmc_network_destroy(wmc_network_t *net);

typedef struct {
  int64_t n_vars;
  int64_t n_clauses_kept;   /* after dropping tautologies                   */
  int64_t n_tensors_strict; /* |N| of Thm 3.2: n_vars + clauses kept        */
  int64_t n_indices_strict; /* |I| of Thm 3.2: sum of distinct vars/clause  */
  int64_t max_clause_rank;
  int32_t has_empty_clause;
  int32_t reserved;
} wmc_network_info_t;
int wmc_network_info(const wmc_network_t *net, wmc_network_info_t *out);

typedef struct {
  int32_t precision;        /* WMC_FP64 or WMC_SCALED_FP32                  */
  int32_t ordering;         /* WMC_ORDER_*                                  */
  int32_t max_rank_cap;     /* reject plans whose largest tensor (in index
                               count, before the query index) exceeds this;
                               0 = 30                                       */
  int32_t slice_to_rank;    /* index slicing (Alg. 3): if > 0, fix variables
                               one at a time until the largest tensor has at
                               most this many indices (at most 24 variables,
                               2^24 slices); every execution then runs the
                               walk once per slice assignment and sums the
                               results (Thm 4.2).  0 = no slicing           */
  int64_t mem_budget_bytes; /* reject plans whose workspace at Q = 1
                               exceeds this; 0 = no limit                   */
  const int32_t *order;     /* WMC_ORDER_GIVEN: n_vars 1-based ids (host,
                               copied)                                      */
  int32_t factor_clauses_above; /* clause factoring (FactorTree, Def. 3.4 and
                               Thm 3.3): if > 0 (at least 3), every clause
                               with more literals than this becomes a chain
                               of OR gates y_1 = l_1 | l_2, y_k = y_{k-1} |
                               l_{k+1}, closed by (y_{r-2} | l_r), each gate
                               the three clause tensors (~a | y), (~b | y),
                               (a | b | ~y); the gate outputs are auxiliary
                               indices with weight 1 for both values (no
                               weight leaf, labels n_vars, n_vars + 1, ...),
                               so W is unchanged.  Not combinable with
                               WMC_ORDER_GIVEN.  0 = off                   */
  int32_t block_fp;         /* block-floating-point float32 (scaled-FP32
                               plans): if > 0, every tensor keeps one int32
                               exponent per query lane for each block of
                               2^(block_fp - 1) consecutive assignments of
                               its non-query indices (weight vectors: one per
                               entry), so entries of different blocks may
                               differ by any factor and only entries of one
                               block share float32's range; nodes add their
                               float32 products in float64 and normalise
                               each output block.  Every node runs on the
                               block-floating-point kernel (no chains, no
                               small-node phase).  At most 9; blocks of at
                               most 2^11 outputs with the query bits (Q *
                               2^(block_fp - 1) <= 2048); not combinable
                               with index slicing.  0 = off                 */
} wmc_plan_opts;

/* Planning: Sec. 3.3.  Builds a contraction tree by bucket elimination
 * along an elimination order of the primal graph (each bucket contracted
 * smallest-first, an index summed at its last appearance), then assigns
 * every intermediate tensor's index order so the dominant contractions read
 * and write contiguously.  Host only.  opts may be NULL (defaults).
 * Errors: WMC_EINVAL, WMC_EPLAN_TOO_BIG, WMC_ENOMEM. */
int wmc_plan(const wmc_network_t *net, const wmc_plan_opts *opts,
             wmc_plan_t **out);
void wmc_plan_destroy(wmc_plan_t *plan);

typedef struct {
  int32_t max_rank;         /* largest tensor rank (index count)            */
  int32_t max_node_rank;    /* largest |I(A) u I(B)| over contractions      */
  int64_t n_leaves;
  int64_t n_nodes;          /* pairwise contractions                        */
  int64_t workspace_bytes;  /* device workspace wmc_execute_device needs
                               for this Q                                  */
  int64_t peak_tensor_bytes;/* the arena part of workspace_bytes           */
  double algorithmic_bytes; /* sum over nodes of |A|+|B|+|C| element bytes */
  double flops;             /* sum over nodes of 2 * |iteration space|      */
  int32_t precision;
  int32_t ordering_used;
  int32_t max_path_roundings; /* d of wmc_result.rel_err_bound            */
  int32_t launches_per_walk;  /* kernel launches one walk enqueues        */
  int32_t n_slice_vars;       /* index slicing: s sliced variables, 2^s
                                 walks per execution (0: none)           */
  int32_t slice_vars[24];     /* their 0-based ids; slice bit k = var k  */
  int32_t n_aux_vars;         /* clause factoring: auxiliary indices      */
  int32_t reserved;
} wmc_plan_info_t;
/* Q >= 1 is the number of queries batched along the extra query index. */
int wmc_plan_info(const wmc_plan_t *plan, int32_t Q, wmc_plan_info_t *out);

/* Node list of the contraction tree, for inspection and host-side tests.
 * Tensor ids: leaves first (0 .. n_leaves-1), then node outputs in
 * post-order.  For node i: children ids and the index labels (0-based
 * variable ids) of the output in bit order (bit j of the linear offset is
 * labels[j]).  For leaf ids: kind 0 = clause tensor (fals = the falsifying
 * assignment bits, the tensor is 1 elsewhere), 1 = weight vector of
 * labels[0], 2 = the scalar 1.  `labels` must hold 64 entries. */
int wmc_plan_node(const wmc_plan_t *plan, int64_t node, int64_t *left,
                  int64_t *right, int32_t *n_labels, int32_t *labels);
int wmc_plan_leaf(const wmc_plan_t *plan, int64_t leaf, int32_t *kind,
                  int32_t *n_labels, int32_t *labels, uint64_t *fals);

/* Execution: Algorithm 2 on the GPU for Q queries at once.  Host buffers:
 * w_pos_q / w_neg_q are [Q][n_vars] float64 (NULL = the network's default
 * weights for every query); out is [Q] wmc_result.  Copies the weights to
 * the device, runs the captured CUDA graph of the plan on `stream`, copies
 * the Q results back and synchronises the stream.  Device memory is a
 * workspace cached inside the plan (allocated on first use for each Q).
 * Errors: WMC_EINVAL (Q < 1 or Q > 4096), WMC_ENOMEM, WMC_ECUDA. */
int wmc_execute(wmc_plan_t *plan, int32_t Q, const double *w_pos_q,
                const double *w_neg_q, void *stream, wmc_result *out);

/* Index slicing across processes: as wmc_execute, but only the slice
 * assignments eta in [slice_lo, slice_hi) of a sliced plan (0 <= slice_lo
 * <= slice_hi <= 2^n_slice_vars); out[q] is their partial sum.  Partial
 * sums of disjoint ranges covering every slice add up (exponent-aligned)
 * to the full result.  An unsliced plan has the single slice 0. */
int wmc_execute_slices(wmc_plan_t *plan, int32_t Q, const double *w_pos_q,
                       const double *w_neg_q, int64_t slice_lo, int64_t slice_hi,
                       void *stream, wmc_result *out);

/* Sum of partial results (Thm 4.2: the count is the sum over the slice
 * assignments eta of the counts conditioned on eta), e.g. the shares that
 * several processes computed with wmc_execute_slices over disjoint slice
 * ranges (Alg. 3, one share per process).  parts: host, n records (n >= 0;
 * may be NULL when n = 0); out: host, one record.  The parts are brought to
 * the largest part's binary exponent and added in order in float64, so
 * counts far outside the float64 range combine without overflow.  flags:
 * the OR of the parts' flags, except WMC_FLAG_EXACT_INT, which is kept only
 * if every part carries it and the sum is below 2^53.  rel_err_bound: the
 * largest part bound plus (n - 1) * 2^-53 (nonnegative parts).  Host only,
 * allocates nothing.  Errors: WMC_EINVAL (NULL out, negative n, a part
 * that is not finite). */
int wmc_combine_results(const wmc_result *parts, int64_t n, wmc_result *out);

/* Execution with device-resident inputs and outputs, asynchronous on
 * `stream`.  d_w_pos / d_w_neg: device [Q][n_vars] float64.  d_workspace:
 * device memory of at least wmc_plan_info(Q).workspace_bytes, 256-byte
 * aligned, owned by the caller and not used by anything else until the
 * stream passes this call.  Results: d_mant[Q] (float64) and d_exp2[Q]
 * (int64) with value = d_mant[q] * 2^d_exp2[q] (d_mant not normalised),
 * d_flags[Q] (uint32, WMC_FLAG_FP32_FLUSH).  Allocates nothing.
 * Errors: WMC_EINVAL (workspace too small or misaligned), WMC_ECUDA. */
int wmc_execute_device(wmc_plan_t *plan, int32_t Q, const double *d_w_pos,
                       const double *d_w_neg, void *d_workspace,
                       size_t workspace_bytes, double *d_mant,
                       int64_t *d_exp2, uint32_t *d_flags, void *stream);

/* Allocation-free variant of wmc_execute_device.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory when
 * they run a count -- a library embedded in a host process whose device
 * memory is entirely owned by another allocator (a framework's caching
 * allocator, a pool reserved up front), or code that must not call
 * cudaMalloc/cudaFree once it is running, since both can synchronise the
 * device.  Same walk, kernels and results (bit for bit) as
 * wmc_execute_device, but the leaf tables and the workspace live in a
 * fixed 32 MiB scratch array that is part of the library's device image
 * (every GPU that loads the library holds it until exit).  Calls no
 * cudaMalloc, cudaFree or other allocating routine.  Plans whose tables
 * plus workspace at this Q exceed 32 MiB are rejected with WMC_EINVAL
 * (wmc_last_error gives the size).  The first call on each device looks up
 * the scratch's device address, with that device current, and keeps it
 * for the life of the process (a cudaDeviceReset of that device
 * invalidates it, as it invalidates every plan's device state).  The leaf
 * tables are copied from host memory only when the scratch holds another
 * plan's (or another Q's); the call descriptor travels as a kernel
 * argument.  Every call shares the one scratch array, which keeps the last
 * call's contents; the walk clears what it accumulates into, but calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads without ordering between their streams) race on it: serialise
 * them.  Inputs and outputs as for wmc_execute_device (asynchronous on
 * `stream`).  Errors: WMC_EINVAL (bad argument, plan too large), WMC_ECUDA. */
int wmc_execute_device_noalloc(wmc_plan_t *plan, int32_t Q,
                               const double *d_w_pos, const double *d_w_neg,
                               double *d_mant, int64_t *d_exp2,
                               uint32_t *d_flags, void *stream);

/* One pairwise contraction C = A . B (Eq. (1) on the network {A, B}; the
 * matrix-multiplication view of Sec. 4.2), on device memory, asynchronous on
 * `stream`.  Kernel choice: the streaming kernel when one operand is small,
 * a dense kernel when the node is a batched matrix product with at least
 * 2^6 values on each free side (float32 with at least 2^7 per free side and
 * 2^4 summed values: the tensor-core kernel, see wmc_set_tensor_cores; at
 * most 4 summed values, one operand's first 10 free indices at C's lowest
 * 10 bits and at least 2^24 outputs: a streaming outer-product kernel, see
 * wmc_set_outer_products; otherwise a tiled scalar kernel whose summed
 * range is split across blocks when there are few output tiles), the
 * generic kernel otherwise.  The tensor-core kernel's packed operands (8 bytes per
 * operand entry) and the split partial sums live in stream-ordered scratch
 * from a memory pool of the library's own, which keeps up to 8 GiB cached.  Bit j of a tensor's linear offset is index labels_x[j];
 * every index has extent 2.  Indices of C must appear in A or B; indices of
 * A or B absent from C are summed; an index in A, B and C is a batch index.
 * precision WMC_FP64: a, b, c are float64.  WMC_SCALED_FP32: a, b, c are
 * float32 mantissas; the true tensors are a * 2^exp_a[0] etc.: exp_a and
 * exp_b (device int64[1]) are read, exp_c (device int64[1]) is written,
 * and c is normalised so that max|c| lies in [1, 2).  For WMC_FP64 the
 * exp pointers may be NULL.  Ranks <= 31, at most 24 summed indices.
 * Errors: WMC_EINVAL, WMC_ECUDA. */
int wmc_contract_pair(int32_t precision, int32_t rank_a,
                      const int32_t *labels_a, const void *a, int32_t rank_b,
                      const int32_t *labels_b, const void *b, int32_t rank_c,
                      const int32_t *labels_c, void *c, const int64_t *exp_a,
                      const int64_t *exp_b, int64_t *exp_c, void *stream);

/* Autotuning of wmc_contract_pair (default off): when on, the first call
 * of each node shape (precision, the three label lists, whether c is
 * 16-byte aligned) times every legal kernel variant that adds the summed
 * terms in the canonical order -- the generic kernel, the streaming kernel
 * at several block counts, the TMA-staged streaming kernel at one to three
 * blocks per SM, the tiled and the outer-product dense kernels -- on the
 * call's own buffers (one warm-up and three timed runs each, synchronising
 * `stream`), and later calls of that shape use the fastest.  All these
 * variants give the same bits, so tuning changes times only.  Shapes whose
 * fixed rule picks a variant with another summation order (the tensor-core
 * product, the split summed range) are not tuned.  The choices are kept
 * for the life of the process (the matrix-multiplication view of Sec. 4.2:
 * kernel and launch shape against the batch / summed / free split). */
void wmc_set_autotune(int32_t on);
/* The variants of a node shape (labels as for wmc_contract_pair; c_aligned16
 * nonzero when C will be 16-byte aligned): *n receives their number, the
 * first min(*n, max_n) are written to kinds / blocks (kind 0 generic, 1
 * streaming, 2 TMA-staged streaming, 3 tiled dense, 4 outer-product dense,
 * 5 tensor-core dense, 6 tiled dense with a split summed range, 7
 * streaming with four units per thread; blocks 0 = the kernel's own
 * count, else the block count (kinds 1, 7) or blocks per SM (kind 2)); the
 * fixed rule's variant is listed first; *chosen is the index
 * of the one wmc_contract_pair uses now (the tuned one once measured).
 * Host only.  Errors: WMC_EINVAL. */
int wmc_pair_variants(int32_t precision, int32_t rank_a, const int32_t *labels_a,
                      int32_t rank_b, const int32_t *labels_b, int32_t rank_c,
                      const int32_t *labels_c, int32_t c_aligned16, int32_t max_n,
                      int32_t *kinds, int64_t *blocks, int32_t *n, int32_t *chosen);

/* Converts a float64 device tensor of n elements to a scaled float32 one:
 * out = x * 2^-E rounded to float32 and exp_out[0] = E, with E chosen so
 * that max|out| lies in [1, 2).  Asynchronous on `stream`. */
int wmc_to_scaled_fp32(const double *x, int64_t n, float *out,
                       int64_t *exp_out, void *stream);

/* ------------------------------------------------------- uneven batches */
/* Many formulas of different shapes in one persistent launch (Alg. 2 for
 * each).  wmc_batch_create admits plans in order while the sum of their
 * single-query workspaces fits mem_budget_bytes (0 = no limit); *n_admitted
 * receives how many.  All plans must share a precision.  Each formula is
 * evaluated with its network's default weights.  Execution: one graph of
 * four kernels -- clear, leaves, a persistent task-queue contraction kernel
 * (tasks = chunks of 2^14 outputs of one node -- for the frontier-times-
 * bucket nodes that carry almost all bytes, 2^14 assignments of the
 * frontier's indices, each thread reading the frontier's entries once and
 * writing every output that differs only in the bucket tensor's own
 * indices; runs of up to four consecutive frontier eliminations of a
 * formula in one pass over the frontier, each thread holding the 2^D
 * values over the chain's indices in registers, as wmc_set_fusion does
 * for one plan; within a formula the nodes
 * run in post-order, across formulas and within a node concurrently; the
 * task list is built by list scheduling, the formulas with the longest
 * remaining chains first; every dependency wait is bounded at one second),
 * and the results.
 * Errors: WMC_EINVAL, WMC_EPLAN_TOO_BIG (nothing fits), WMC_ENOMEM,
 * WMC_ECUDA, WMC_ETIMEOUT. */
int wmc_batch_create(wmc_plan_t *const *plans, int32_t n_plans,
                     int64_t mem_budget_bytes, wmc_batch_t **out,
                     int32_t *n_admitted);
/* Task size and order of batches created after the call: chunk_log2 = log2
 * of the outputs per task, or of the assignments u per task for nodes in
 * stream mode (8..16; 0 = the default 14; chains take a quarter of that
 * many units, at least 2^8), order 0 = list
 * scheduling by the formulas' remaining chains (default), 1 = round-robin
 * over the formulas in post-order.  Results are the same bits either way
 * (a node's outputs do not depend on how they are split into tasks). */
void wmc_set_batch_schedule(int32_t chunk_log2, int32_t order);
/* Longest run of frontier eliminations (Alg. 2: each step sums one index
 * of the frontier and adds at most one) that batches created after the call
 * execute as one pass: 2..4, or 0 (or 1) for one pass per contraction.
 * Default 4.  A chain's inner tensors are never stored and are not
 * rescaled between its steps (the scales are powers of two): results are
 * the same bits either way; workspace and algorithmic bytes shrink. */
void wmc_set_batch_fusion(int32_t max_steps);
/* Small subtrees in batches created after the call: every node of output
 * rank <= max_rank (1..14) with at most 2^8 summed terms whose children are
 * leaves or such nodes (the root excepted) runs inside the task of its
 * maximal such subtree -- one block, its nodes one after another with no
 * dependency waits, all of a formula's subtrees before its other nodes --
 * so that a formula's strictly ordered steps are its large nodes alone.
 * 0 = every node is a task of its own.  Default 12.  Results are the same
 * bits either way. */
void wmc_set_batch_subtrees(int32_t max_rank);
typedef struct {
  int64_t n_formulas;
  int64_t n_nodes;          /* scheduled units: a node, a chain, or the set of a
                               formula's small subtrees */
  int64_t n_tasks;
  int64_t workspace_bytes;
  double algorithmic_bytes;
  int32_t max_rank;
  int32_t grid;             /* persistent blocks (set after first execute) */
} wmc_batch_info_t;
int wmc_batch_info(const wmc_batch_t *batch, wmc_batch_info_t *out);
/* Synchronous on `stream`; out[i] is the result of admitted formula i. */
int wmc_batch_execute(wmc_batch_t *batch, void *stream, wmc_result *out);
/* Layout of admitted formula i (0 <= i < n_formulas), for inspection: the
 * byte offset of its workspace inside the batch workspace, its largest
 * tensor rank and its number of pairwise contractions.  Any output pointer
 * may be NULL.  Errors: WMC_EINVAL (bad handle or index). */
int wmc_batch_formula_info(const wmc_batch_t *batch, int32_t i,
                           int64_t *ws_offset, int32_t *max_rank,
                           int64_t *n_nodes);
void wmc_batch_destroy(wmc_batch_t *batch);

/* ------------------------------------------------------------- serving */
typedef struct {
  int32_t precision;        /* WMC_FP64 or WMC_SCALED_FP32 (of the plan)   */
  int32_t max_batch;        /* largest Q of one wave (power of 2, <= 1024) */
  int32_t max_waves;        /* waves in flight at once (each its own stream
                               and workspace)                               */
  int32_t partial_overlap;  /* 0 (default): a wave of fewer than max_batch
                               queries starts only when no wave is running,
                               so under load the next wave grows while the
                               current one runs; full waves start in any
                               free slot.  1: any free slot starts a wave
                               from whatever is queued                     */
  int64_t arena_bytes;      /* device memory for all wave workspaces; a wave
                               of Q queries is admitted only while its
                               workspace fits; 0 = max_waves * ws(max_batch) */
  int64_t max_wave_wait_us; /* how long the batcher waits for more queries
                               before launching a partial wave              */
} wmc_server_opts;

/* Continuous-batching server over one plan.  Queries submitted while waves
 * are running are gathered into the next wave as soon as a wave slot and
 * its workspace are free; waves run on separate streams and overlap on the
 * device.  Every query's result is independent of the wave it lands in. */
int wmc_server_create(wmc_plan_t *plan, const wmc_server_opts *opts,
                      wmc_server_t **out);
/* Copies n_vars weights each (host); returns a ticket (never reused). */
int wmc_submit(wmc_server_t *srv, const double *w_pos, const double *w_neg,
               uint64_t *ticket);
/* n queries at once: w_pos / w_neg are [n][n_vars] (host, row-major);
 * tickets[n] receives consecutive tickets.  One lock for the whole batch,
 * so a client with many queries in hand does not pay a call per query. */
int wmc_submit_many(wmc_server_t *srv, int64_t n, const double *w_pos,
                    const double *w_neg, uint64_t *tickets);
/* WMC_OK (result written, ticket retired), WMC_PENDING, or an error. */
int wmc_poll(wmc_server_t *srv, uint64_t ticket, wmc_result *out);
/* As wmc_poll; *done_ns (may be NULL) receives the CLOCK_MONOTONIC time in
 * nanoseconds at which the server published the result. */
int wmc_poll_ex(wmc_server_t *srv, uint64_t ticket, wmc_result *out,
                int64_t *done_ns);
/* Blocks until the ticket completes or timeout_us elapses (WMC_ETIMEOUT). */
int wmc_wait(wmc_server_t *srv, uint64_t ticket, int64_t timeout_us,
             wmc_result *out);
typedef struct {
  int64_t submitted, completed, waves, failed_waves;
  double mean_wave_q;
  int64_t max_in_flight;    /* most waves that were on the device at once */
} wmc_server_stats_t;
int wmc_server_stats(wmc_server_t *srv, wmc_server_stats_t *out);
void wmc_server_destroy(wmc_server_t *srv);

/* Measurement: runs the walk of wmc_execute_device once WITHOUT the graph,
 * with a CUDA event after every launch, and synchronises `stream`.  For
 * launch i (i < min(n_max, launch count)): node_ms[i] = its device time,
 * kind[i] = 0 generic contraction, 1 streaming contraction, 4 streaming
 * contraction with TMA-staged operand, 5 dense tiled contraction, 6 fused
 * pair of eliminations, 7 small-node phase (one persistent launch), 8 run
 * of frontier eliminations in one pass, 9 runs of such chains in one
 * launch, 10 one-block walk, 11 batched small contraction (two large
 * operands, few free and summed indices), 2 leaf or bookkeeping kernel,
 * 3 memset; alg_bytes[i] = the bytes a contraction
 * must move (|A| + |B| + |C| in its element type).  Returns the launch
 * count through *n_launches.  Same arguments and errors as
 * wmc_execute_device; creates and destroys its own events. */
int wmc_profile_walk(wmc_plan_t *plan, int32_t Q, const double *d_w_pos,
                     const double *d_w_neg, void *d_workspace,
                     size_t workspace_bytes, double *d_mant, int64_t *d_exp2,
                     uint32_t *d_flags, void *stream, int64_t n_max,
                     float *node_ms, int32_t *kind, double *alg_bytes,
                     int64_t *n_launches);

/* Autotuning of a plan's walk (the tuner of kernel shape against the
 * index split, at the level of the whole walk): for batch size Q, times
 * the walk under up to eight layouts -- chains of up to 6, 4, 3 or 2
 * consecutive frontier eliminations per pass or none, the small-node phase
 * on or off, runs of chains in one launch (float32) -- on the network's
 * default weights (median of five walks after two warm-up walks, on
 * `stream`, synchronously), checks that every layout returns the first
 * one's values bit for bit (a layout that does not is rejected, ms = -1),
 * and installs the fastest as the plan's layout for Q: later calls with
 * this Q (wmc_execute, wmc_execute_device, servers created afterwards) use
 * it, and wmc_plan_info(Q) reports its workspace and launch count.
 * Allocates its own device buffers while it runs.  Call it before sharing
 * the plan with other threads.  Errors: WMC_EINVAL, WMC_ENOMEM, WMC_ECUDA. */
typedef struct {
  int32_t n_candidates;    /* layouts timed (<= 8)                          */
  int32_t chosen;          /* index of the installed one                    */
  int32_t fuse[8];         /* longest chain per pass (0: one pass per node) */
  int32_t small_phase[8];  /* small-node phase on (1) or off (0)            */
  int32_t chain_runs[8];   /* runs of chains in one launch: max tiles (0: off) */
  int32_t launches[8];     /* kernel launches per walk                      */
  float ms[8];             /* median walk time; -1: rejected                */
} wmc_tune_report;
int wmc_autotune_plan(wmc_plan_t *plan, int32_t Q, void *stream, wmc_tune_report *out);

/* Execution option: the longest run of consecutive frontier eliminations
 * contracted in one pass over the frontier tensor (the intermediates never
 * reach memory), 2..6; 0 or 1 turns fusion off; negative (the default):
 * up to 6 for walks of at most 16 query lanes, up to 4 for wider ones.
 * Runs of up to four (k2_chain) take vector lanes and growth steps and
 * stage the frontier through shared memory; runs of five or six
 * (k2_chain_direct, float32) hold 64 values of one lane per thread, load
 * them directly and take no growth step -- fewer launches for small walks,
 * slower than four-step runs where the walk is bound by HBM.  Affects
 * plans laid out after the call (a plan caches its layout per Q). */
void wmc_set_fusion(int32_t on);
/* Execution option (default on): every node whose whole subtree is small
 * (at most 2^16 outputs including the query bits, at most 2^8 summed
 * terms) runs inside one persistent launch at the start of the walk
 * instead of a launch per node.  Affects plans laid out after the call. */
void wmc_set_small_phase(int32_t on);
/* Execution option (default off): a formula whose every node has at most
 * 2^16 outputs (with the query bits) and 2^8 summed terms, with at most 4
 * query lanes, and whose live tensors fit in 200 KB, runs its whole walk in
 * one thread block: leaves and intermediates in shared memory, the nodes
 * level by level (each node at the latest level below its parent; a level's
 * nodes are independent, so each level is one phase between block
 * barriers), with no launch per node and no dependency waits through
 * global memory.  Results are the same bits as the small-node phase.
 * Measured level with the small-node phase on the random 3-CNF n = 20
 * walks (in FP64 one SM's FP64 rate bounds it), so it is off by default.
 * Affects plans laid out after the call. */
void wmc_set_cta_walk(int32_t on);
/* Execution option (default on): chain kernels are launched as programmatic
 * dependent launches, so that each one's set-up overlaps the tail of the
 * launch before it.  Affects graphs captured after the call. */
void wmc_set_dependent_launch(int32_t on);
/* Execution option (default on): wmc_contract_pair runs float32 dense
 * products with at least 2^7 rows, 2^7 columns and 2^4 summed terms on the
 * tensor cores (tcgen05, 3xTF32 with float32 accumulation: each operand is
 * packed once, scaled and split into TF32 hi and lo parts, then a
 * persistent kernel multiplies 128 x 256 (or 128 x 128) output tiles);
 * off, on the scalar tiled kernel.  The two agree within float32 rounding,
 * not bit for bit. */
void wmc_set_tensor_cores(int32_t on);
/* Execution option (default on): walk nodes that join two large operands
 * with at most 2 summed indices run on the batched small-contraction
 * kernel (a thread per batch assignment, the few free indices in
 * registers) instead of the generic one; the same bits either way.
 * Affects plans laid out after the call. */
void wmc_set_batched_pairs(int32_t on);
/* Execution option (default on): wmc_contract_pair runs dense products
 * with at most 4 summed values whose C has one operand's first 10 free
 * indices as its lowest 10 bits, at least 2^24 outputs and a 16-byte
 * aligned c, on a streaming outer-product kernel (each thread keeps 4
 * consecutive entries of that operand in registers and writes 4
 * consecutive outputs per value of the other side); off, on the tiled
 * scalar kernel.  Both add the summed terms in the same order, so the
 * results are the same bits.  Read at each call; walks keep the tiled
 * kernel. */
void wmc_set_outer_products(int32_t on);
/* Execution option (default on): wmc_execute and wmc_execute_slices run the
 * queries of a scaled-FP32 plan whose results carry WMC_FLAG_FP32_FLUSH
 * again in FP64 on the same contraction tree (one extra walk over those
 * queries) and return the FP64 values with WMC_FLAG_FELL_BACK_FP64.  The
 * device entries and the server report the flush flag and leave the choice
 * to the caller. */
void wmc_set_fp64_fallback(int32_t on);
/* Execution option (default 0 = off): consecutive four-step float32
 * chains of the walk whose every chain has at most max_tiles tiles run as
 * one launch (k2_chain_seq: tiles handed out in chain order from per-chain
 * counters, each block waiting, bounded, for the previous chain's
 * completion count), which replaces a launch and a grid completion per
 * chain by counter waits.  Results are bit-identical either way.  Affects
 * plans laid out after the call. */
void wmc_set_chain_runs(int32_t max_tiles);

/* Host-side bounds check of the walk for batch size Q: replays the index
 * arithmetic of every contraction launch (all bulk copies of every tile,
 * the extreme and sampled per-thread offsets) on the CPU and verifies each
 * access lies inside its tensor.  *n_checked (may be NULL) receives the
 * number of work units checked.  WMC_EINVAL names the first violation. */
int wmc_debug_check_bounds(wmc_plan_t *plan, int32_t Q, int64_t *n_checked);

/* ------------------------------------------------------------- misc */
const char *wmc_last_error(void);
/* Number of kernels this library launched since load (for accounting). */
int64_t wmc_kernel_launch_count(void);
/* Test hook: wmc_contract_pair runs the variant (kind, blocks) of
 * wmc_pair_variants (WMC_EINVAL if the node has no such variant); kind < 0
 * turns the hook off. */
void wmc_debug_force_pair_variant(int32_t kind, int64_t blocks);
/* Test hook: make the next n device allocations fail with WMC_ENOMEM. */
void wmc_debug_fail_next_allocs(int32_t n);
/* Test hook: while on == 1, the walk's first launch that stages tiles with
 * bulk copies never issues its first tile's copy; while on == 2, the first
 * run of chains (k2_chain_seq) never issues the copies of its first chain's
 * tile 0.  The bounded mbarrier wait runs out (about a second), the other
 * blocks' bounded waits see the error word, and the call reports
 * WMC_ETIMEOUT; no fault, trap or hang.  Affects graphs captured while it
 * is set. */
void wmc_debug_stall_copies(int32_t on);

#ifdef __cplusplus
}
#endif
#endif /* WMC_B300_H */
