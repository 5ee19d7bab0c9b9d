/*
 * neat.h -- C ABI of the B300 (sm_103a) NEAT population-evaluation library.
 *
 * Evaluates a whole population of NEAT genomes held in the padded tensor
 * encoding of TensorNEAT (arXiv 2504.08339):
 *   Sec. 3.1 (Tensorized Encodings): one row per node / connection, rows past
 *     a genome's size (and holes left by removal) are NaN padding; the
 *     population tensors are P_N[P, N, .] and P_C[P, C, .].
 *   Sec. 3.3 (Tensorized Network Inference): a transformation stage computes
 *     the topological order N_order (and here also layer indices and a packed
 *     per-genome program that replaces the dense C_exp tensor); a calculation
 *     stage sets v[inputs] = I and, in N_order, v[k] = f_n(f_c(v | in-edges of
 *     k) | attributes of k) with f_c = w * x and f_n = act(b + r * agg(.));
 *     O = v[outputs].
 *   App. B (genome interface): input_idx = arange(I), output_idx =
 *     arange(I, I + O), i.e. node ROWS 0..I-1 are the inputs and rows
 *     I..I+O-1 the outputs.
 *
 * Memory conventions (all entry points):
 *   - Every array argument is a DEVICE pointer owned by the caller, row-major,
 *     float32 or int32/uint32 as declared, aligned to its element size (conns
 *     to 16 bytes).  The library never frees it and keeps no reference after
 *     the call returns.  A misaligned or NULL required pointer gives
 *     NEAT_ERR_ARG and launches nothing.
 *   - The plan's workspace is caller-owned device memory of at least
 *     neat_workspace_bytes() bytes (256-byte aligned); it holds the
 *     transformed programs between calls.  The plan object itself is a small
 *     host allocation.
 *   - Calls are asynchronous on `stream`; the return code reports only host
 *     side argument checks and launch errors.  Problems of individual genomes
 *     are reported through the per-genome status words (NEAT_G_* bits).
 *   - A plan must not be used on two streams at once.
 *
 * Node rows:       nodes[P, N, 5] = (key, bias, response, activation id, aggregation id)
 * Connection rows: conns[P, C, 4] = (in key, out key, weight, enabled)
 * A row is padding iff one of its key columns is NaN; a connection is enabled
 * iff `enabled` is neither NaN nor 0.  Keys are integers in [0, 2^24), unique
 * per genome, resolved by lookup (they need not equal row indices).
 */
#ifndef NEAT_H
#define NEAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same declaration as the CUDA runtime's stream handle. */
typedef struct CUstream_st *cudaStream_t;

typedef enum {
  NEAT_OK = 0,
  NEAT_ERR_ARG = -1,          /* bad size, NULL or misaligned pointer          */
  NEAT_ERR_CUDA = -2,         /* a CUDA launch or runtime call failed           */
  NEAT_ERR_WORKSPACE = -3,    /* workspace smaller than neat_workspace_bytes() */
  NEAT_ERR_UNSUPPORTED = -4,  /* sizes beyond the library limits below          */
  NEAT_ERR_STATE = -5,        /* e.g. forward before any transform              */
  NEAT_ERR_TIMEOUT = -6       /* a kernel's bounded wait gave up (neat_plan_check) */
} neat_status;

/* Device-side failure bits of a plan (neat_plan_device_errors): set by a
 * kernel that could not finish some genomes; those genomes' outputs are NaN.
 *   NEAT_DEV_TIMEOUT    a bounded wait for a bulk copy of a batch program gave
 *                       up (after neat_tuning.wait_polls polls)
 *   NEAT_DEV_NO_SCRATCH a genome found no workspace value slot (not reachable
 *                       with the launch shapes the library picks) */
#define NEAT_DEV_TIMEOUT 1u
#define NEAT_DEV_NO_SCRATCH 2u

/* Limits of this build. */
#define NEAT_MAX_NODES 1024
#define NEAT_MAX_CONNS 8192

/* Activation ids (node column 3): textbook, unscaled forms. */
#define NEAT_ACT_IDENTITY 0 /* z                 */
#define NEAT_ACT_SIGMOID 1  /* 1 / (1 + e^-z)    */
#define NEAT_ACT_TANH 2     /* tanh z            */
#define NEAT_ACT_RELU 3     /* max(0, z)         */
#define NEAT_ACT_SIN 4      /* sin z             */
#define NEAT_ACT_GAUSSIAN 5 /* e^(-z^2)          */
#define NEAT_ACT_ABS 6      /* |z|               */
/* Aggregation ids (node column 4); an empty aggregation is 0 for all four. */
#define NEAT_AGG_SUM 0
#define NEAT_AGG_PRODUCT 1
#define NEAT_AGG_MAX 2 /* fmax fold (NaN-ignoring) */
#define NEAT_AGG_MEAN 3

/* Per-genome status bits written by neat_transform.  A genome with any bit
 * set gets NaN outputs from the forward calls and zero gradients; with any
 * bit other than CYCLE it also gets no order (order/layer all -1). */
#define NEAT_G_CYCLE 1u            /* enabled connections form a cycle (or a self-loop) */
#define NEAT_G_DANGLING_KEY 2u     /* an enabled connection names a key no node has      */
#define NEAT_G_DUP_KEY 4u          /* two valid node rows share a key                    */
#define NEAT_G_DUP_EDGE 8u         /* two enabled rows with the same (in, out)           */
#define NEAT_G_EDGE_INTO_INPUT 16u /* an enabled connection ends at an input node        */
#define NEAT_G_BAD_ATTR 32u        /* key not an integer in [0,2^24); act/agg id out of
                                      range or not integral; NaN bias/response on a
                                      non-input node; NaN weight on an enabled row   */
#define NEAT_G_IO_ROW_INVALID 64u  /* one of rows 0..I+O-1 is padding                    */

typedef struct neat_plan neat_plan;

/* Library version (major * 10000 + minor * 100 + patch). */
int neat_version(void);

/* Human-readable name of a status code (static string). */
const char *neat_status_string(neat_status s);

/* The cudaError_t value behind the calling thread's most recent
 * NEAT_ERR_CUDA (0 if none occurred). */
int neat_last_cuda_error(void);

/* Bytes of device workspace a plan for these sizes needs (0 on bad sizes).
 * Sizes: P >= 0 genomes, N in [I+O, NEAT_MAX_NODES] node rows, C in
 * [1, NEAT_MAX_CONNS] connection rows, I >= 1 inputs, O >= 1 outputs. */
size_t neat_workspace_bytes(int P, int N, int C, int I, int O);

/* Create a plan.  `workspace` is caller-owned device memory (256-byte
 * aligned, >= neat_workspace_bytes(P,N,C,I,O) bytes) that must outlive the
 * plan.  The plan binds to the current CUDA device.  *out is set on success. */
neat_status neat_plan_create(neat_plan **out, int P, int N, int C, int I, int O,
                             void *workspace, size_t workspace_bytes);

/* Destroy a plan (host memory only; the workspace stays the caller's). */
neat_status neat_plan_destroy(neat_plan *plan);

/* Tuning knobs picked by the autotuner (0 = library default).
 *   warps_per_cta    warps of a sample-parallel or HyperNEAT-query CTA (1..16)
 *   samples_per_lane samples one lane evaluates in the sample-parallel forward,
 *                    queries one lane evaluates in the HyperNEAT query (1, 2, 4);
 *                    0 (default, reported as 0): two for S >= 64 in calls
 *                    without saved aggregates, else one;
 *                    the HyperNEAT query four; the recurrent forward one (it
 *                    takes 1 or 2, larger values as 2)
 *   lvl_threads      threads of a level-synchronous (small-sample) CTA: 32..256,
 *                    a multiple of 32; each warp of it evaluates its own batches
 *                    (default: the CTA size that keeps the most warps resident)
 *   small_s_max      largest S that uses the level-synchronous forward (1..64,
 *                    -1 = never; default 8); larger S, calls that ask for the
 *                    saved aggregates, and batches that do not fit in shared
 *                    memory use the sample-parallel forward
 *   lvl_budget_kb    program bytes (KiB, 8..160) of a level-synchronous batch
 *                    (raised to what the largest possible genome of the plan
 *                    needs); applied by the next neat_transform.  0 (default,
 *                    reported as 0): each transform picks the smallest budget,
 *                    in 128-byte steps, whose batches do not outnumber the
 *                    warps a one-sample forward keeps resident
 *   prune_dead       0 (default): every valid node is evaluated, as the
 *                    paper's calculation does; 1: forwards that return only the
 *                    outputs, the HyperNEAT query and the backward skip the
 *                    nodes no output depends on (the same outputs; their
 *                    parameters' gradients are 0); applied by the next
 *                    neat_transform
 *   wait_polls       polls of a level-synchronous warp's wait for its staged
 *                    batch program before it gives up on the batch (0: the
 *                    default 2^22; -1: no poll, every batch gives up at once,
 *                    which exercises the failure path).  A batch given up on
 *                    gets NaN outputs and sets NEAT_DEV_TIMEOUT; the warp
 *                    still waits (bounded) for its copies before it reuses
 *                    its buffer.
 *   bwd_global       0 (default): the backward keeps each warp's value,
 *                    aggregate and adjoint arrays in shared memory when a
 *                    genome of the plan's N, C fits there, else in workspace
 *                    slots (global memory, L2-resident); 1: always in
 *                    workspace slots. */
typedef struct {
  int warps_per_cta;
  int samples_per_lane;
  int lvl_threads;
  int small_s_max;
  int lvl_budget_kb;
  int prune_dead;
  int wait_polls;
  int bwd_global;
} neat_tuning;
neat_status neat_plan_set_tuning(neat_plan *plan, const neat_tuning *t);
neat_status neat_plan_get_tuning(const neat_plan *plan, neat_tuning *t);

/* The plan's device failure word (NEAT_DEV_* bits, OR-ed by the kernels since
 * it was last cleared; neat_transform clears it): copied to *errors (device
 * u32, caller-owned) on `stream` and, if `clear` != 0, reset to 0 after the
 * copy.  Asynchronous and stream-ordered (capturable in a CUDA graph). */
neat_status neat_plan_device_errors(neat_plan *plan, uint32_t *errors, int clear,
                                    cudaStream_t stream);

/* Synchronising check: waits for `stream`, reads and clears the failure word;
 * NEAT_ERR_TIMEOUT if NEAT_DEV_TIMEOUT was set, NEAT_ERR_WORKSPACE if
 * NEAT_DEV_NO_SCRATCH was, NEAT_OK otherwise.  Not during a stream capture. */
neat_status neat_plan_check(neat_plan *plan, cudaStream_t stream);

/* Structure check of the plan's transformed population (no counterpart in
 * the paper; the range checks a debugging build would make, run as kernels
 * over the structures instead of inside the evaluation kernels).  Checks
 * every index the forward, backward and HyperNEAT kernels read from the
 * structures the last transform wrote -- queue entries, genome headers,
 * packed position programs (records, edge ranges, sources earlier than their
 * node in a feed-forward transform), input / output positions, compiled
 * programs (pair ranges, value rows, layer starts, output rows) and level
 * batch programs (arena place, staged head size, header offsets, genome
 * table, round table, task and edge slots) -- against the arrays they
 * address, reading only inside the workspace whatever its contents.
 *   bits   device u32, caller-owned, 4-byte aligned: set to the OR of
 *          NEAT_BAD_* bits (0: every structure in range), asynchronously on
 *          `stream`
 * NEAT_ERR_STATE before any transform, NEAT_ERR_ARG for a NULL or misaligned
 * `bits`. */
#define NEAT_BAD_QUEUE 1u    /* a queue entry is not a genome id */
#define NEAT_BAD_PACKED 2u   /* a header or packed position program out of range */
#define NEAT_BAD_COMPILED 4u /* a compiled program out of range */
#define NEAT_BAD_BATCHES 8u  /* a level batch program out of range */
neat_status neat_plan_validate(const neat_plan *plan, uint32_t *bits, cudaStream_t stream);

/* Transformation stage (Sec. 3.3) for all P genomes.
 *   nodes   [P, N, 5] f32, conns [P, C, 4] f32 (read only)
 *   order   [P, N] i32 out: node ROWS in topological order -- Kahn by frontier,
 *           each frontier in ascending key -- padded with -1
 *   layer   [P, N] i32 out: frontier index of each row (-1 for padding rows
 *           and rows not emitted)
 *   n_layers[P] i32 out, gstatus [P] u32 out (NEAT_G_* bits)
 * Also (re)builds the plan's packed programs; later forward/backward calls
 * evaluate the genomes of the most recent transform. */
neat_status neat_transform(neat_plan *plan, const float *nodes, const float *conns, int32_t *order,
                           int32_t *layer, int32_t *n_layers, uint32_t *gstatus,
                           cudaStream_t stream);

/* Calculation stage (Sec. 3.3), batched form: one persistent launch pulls
 * size-sorted genomes from a device work queue over ragged-packed programs.
 *   inputs  genome g, sample s, input i at inputs[g * in_pop_stride + s * I + i]
 *           (in_pop_stride 0 = one input set shared by all genomes; otherwise
 *           >= S * I)
 *   S       input vectors per genome (S >= 0)
 *   outputs [P, S, O] f32 out; NaN for genomes with a nonzero status
 *   saved   optional [P, N, S] f32 out (NULL to skip): saved[g][p][s] is the
 *           aggregated input a of the node at canonical position p for sample
 *           s (positions of input nodes and p >= V are not written), kept for
 *           neat_backward; sample-contiguous so that both kernels move it in
 *           whole 128-byte lines. */
neat_status neat_forward(neat_plan *plan, const float *inputs, int64_t in_pop_stride, int S,
                         float *outputs, float *saved, cudaStream_t stream);

/* Transformation for RECURRENT ("concurrent") networks (Sec. 3.3 names
 * feed-forward and concurrent networks; only the former gets a topological
 * order).  Same validation and status bits as neat_transform except that
 * cycles and self-loops are legal (NEAT_G_CYCLE is never set); every valid
 * node is placed in ascending key order.  gstatus [P] u32 out.  Afterwards
 * only neat_forward_recurrent applies (the other calculation entry points
 * return NEAT_ERR_STATE until the next neat_transform). */
neat_status neat_transform_recurrent(neat_plan *plan, const float *nodes, const float *conns,
                                     uint32_t *gstatus, cudaStream_t stream);

/* Recurrent calculation over T synchronous iterations (0 <= T <= 65536):
 * v^0 = the inputs on input nodes and 0 on every other node; in iteration t
 * every non-input node k takes act(b_k + r_k * agg_e(w_e * v^{t-1}[src_e]))
 * while the inputs stay clamped; outputs [P, S, O] = v^T at the output
 * nodes (NaN for genomes with a nonzero status).  Inputs, strides and S as in
 * neat_forward.  Valid after neat_transform_recurrent or neat_transform (a
 * genome with NEAT_G_CYCLE then has NaN outputs).  With T at least the depth
 * of an acyclic genome the outputs equal the feed-forward ones. */
neat_status neat_forward_recurrent(neat_plan *plan, const float *inputs, int64_t in_pop_stride,
                                   int S, int T, float *outputs, cudaStream_t stream);

/* Calculation stage, plain padded form (the comparison baseline): every
 * genome walks all N padded positions of its padded program; no queue, no
 * packing, no compiled programs.  Up to 8 samples per genome a one-warp CTA
 * per (genome, sample) puts its lanes over each node's incoming edges; above
 * that a one-warp CTA per (genome, 32 samples) puts them over samples.
 * Same arguments and results as neat_forward (no saved buffer). */
neat_status neat_forward_plain(neat_plan *plan, const float *inputs, int64_t in_pop_stride, int S,
                               float *outputs, cudaStream_t stream);

/* Reverse mode of the calculation stage (no counterpart in the paper; the
 * gradient of L with respect to weights, biases, responses and inputs given
 * grad_outputs = dL/dO).
 *   inputs, in_pop_stride, S as in neat_forward
 *   grad_outputs [P, S, O] f32
 *   saved        the buffer filled by neat_forward with the same inputs, or
 *                NULL to recompute the forward values inside the kernel
 *   grad_weight  [P, C] f32 out, by connection row (0 on padding/disabled rows)
 *   grad_bias, grad_response [P, N] f32 out, by node row (0 on inputs/padding)
 *   grad_inputs  optional [P, S, I] f32 out (NULL to skip); with a shared input
 *                set (in_pop_stride 0) it is still written per genome, and
 *                neat_sum_genomes gives the shared set's gradient [S, I].
 * Sums over samples are deterministic (no floating-point atomics). */
neat_status neat_backward(neat_plan *plan, const float *inputs, int64_t in_pop_stride, int S,
                          const float *grad_outputs, const float *saved, float *grad_weight,
                          float *grad_bias, float *grad_response, float *grad_inputs,
                          cudaStream_t stream);

/* Sum over genomes: out[j] = sum_{g = 0 .. P-1} x[g * n + j] for 0 <= j < n,
 * accumulated in double precision in ascending genome order and rounded to
 * f32 once (deterministic).  Turns neat_backward's per-genome grad_inputs of
 * an input set that every genome shares (in_pop_stride 0) into that set's
 * gradient: the chain rule through the one tensor all genomes read.
 *   x [P, n] f32 device, out [n] f32 device out (the ranges may not overlap).
 * P = 0 writes zeros.  NEAT_ERR_ARG for negative sizes, NULL or unaligned
 * pointers, or overlapping ranges (nothing launched). */
neat_status neat_sum_genomes(const float *x, int P, int64_t n, float *out, cudaStream_t stream);

/* HyperNEAT substrate query (the CPPN use of NEAT networks).  Requires I = 5,
 * O = 1.  For every genome and every (source, target) pair of a grid x grid
 * substrate, cell c = j * grid + i at (x, y) = (-1 + 2i/(grid-1),
 * -1 + 2j/(grid-1)), the CPPN is evaluated on (x_s, y_s, x_t, y_t, 1) and
 *   weights[g, s, t] = o if |o| > thresh else 0        ([P, grid^2, grid^2] f32)
 * Coordinates are generated in the kernel.  2 <= grid <= 128. */
neat_status neat_hyperneat_query(neat_plan *plan, int grid, float thresh, float *weights,
                                 cudaStream_t stream);

/* Size of the fixed device array used by neat_forward_noalloc. */
#define NEAT_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Transformation + batched forward in one call that allocates nothing (the
 * paper has no counterpart: this serves callers that cannot allocate device
 * memory when they evaluate, e.g. code inside an allocator-free real-time
 * loop or a plugin that is handed only its input and output buffers).
 *   nodes [P, N, 5], conns [P, C, 4], inputs / in_pop_stride / S as in
 *   neat_forward; outputs [P, S, O] f32 out; gstatus [P] u32 out.
 * The plan workspace and the transform's order/layer tensors live in one
 * static device array of NEAT_NOALLOC_SCRATCH_BYTES compiled into the library
 * (held by every GPU that loads it until the process exits).  The call uses
 * 16 regions of it, each rounded up to 256 bytes: at most
 * P (48 N + 24 C + 4 (I + O) + 60) + 4352 bytes.  A population whose regions
 * do not fit returns NEAT_ERR_WORKSPACE before any launch (the limit is
 * exactly 1,800 genomes of N = 128, C = 512, I = 27, O = 8 and 227 of N = 1024,
 * C = 4096, I = 17, O = 6).  Every shape check (sizes, alignment, shared
 * memory, the 2^31 work-item limit of P * ceil(S / 32)) also comes before the
 * first launch.  Uses the sample-parallel forward with each genome's values in
 * shared memory, for every S.
 * The first call on a device (that device current) looks up the array's
 * address with cudaGetSymbolAddress and sets kernel attributes: make it before
 * any stream capture.  All calls share the array and each call overwrites it:
 * calls that overlap on the GPU race and must be serialised by the caller.
 * No cudaMalloc, cudaFree or other allocating call is made. */
neat_status neat_forward_noalloc(const float *nodes, const float *conns, int P, int N, int C,
                                 int I, int O, const float *inputs, int64_t in_pop_stride, int S,
                                 float *outputs, uint32_t *gstatus, cudaStream_t stream);

/* HyperNEAT substrate evaluation (the paper names HyperNEAT but describes no
 * substrate; this is the two-sheet substrate of the query grid): an input
 * sheet and an output sheet of K = G^2 cells; weights[g][s][t] (the query's
 * layout: source cell s, target cell t) connects input cell s to output cell
 * t; for every input pattern, y_t = act(sum_s w[s][t] x_s), no bias.
 *   weights [P, K, K] f32; inputs: pattern p of genome g, cell c at
 *           inputs[g * in_pop_stride + p * K + c] (stride 0: one pattern set
 *           shared by every genome, otherwise >= S * K)
 *   act     activation id (NEAT_ACT_*); outputs [P, S, K] f32 out
 * Sums run over s in ascending order in fp32 (deterministic).  Plan-free. */
neat_status neat_substrate_forward(const float *weights, int P, int K, const float *inputs,
                                   int64_t in_pop_stride, int S, int act, float *outputs,
                                   cudaStream_t stream);

/* neat_hyperneat_query into `weights` [P, grid^2, grid^2] followed by
 * neat_substrate_forward of those weights on the same stream: every CPPN's
 * substrate network evaluated on S input patterns without a host round trip. */
neat_status neat_hyperneat_substrate(neat_plan *plan, int grid, float thresh, const float *inputs,
                                     int64_t in_pop_stride, int S, int act, float *weights,
                                     float *outputs, cudaStream_t stream);

/* Tensorized operations of Sec. 3.2 on the population tensors, in place (no
 * counterpart needs a host round trip: the list is data).  ops [P, K, 8] f32:
 * operation k of genome g is (kind, row, v0..v5), applied in order k = 0..K-1:
 *   1 add node:        nodes[r] = (v0..v4), r = the first row whose key is NaN
 *   2 remove node:     nodes[row] = NaN
 *   3 add connection:  conns[r] = (v0..v3), r = the first row with a NaN key
 *   4 remove connection: conns[row] = NaN
 *   5 set node attribute: nodes[row][v0] = v1 (column v0 in 1..4)
 *   6 set connection attribute: conns[row][v0] = v1 (column v0 in 2..3)
 *   any other kind: nothing
 * An operation with no free row, a row outside the table or a column outside
 * its range changes nothing and sets bit k (k < 32) of op_status[g]
 * (optional [P] u32 out).  Removing a node leaves its connections (remove
 * them with their own operations).  One warp per genome, asynchronous. */
neat_status neat_apply_ops(float *nodes, float *conns, int P, int N, int C, const float *ops,
                           int K, uint32_t *op_status, cudaStream_t stream);

/* neat_apply_ops on the plan's population sizes followed by neat_transform
 * (same arguments), on one stream: one generation's structural edits and the
 * new programs without a round trip to the host. */
neat_status neat_mutate_transform(neat_plan *plan, float *nodes, float *conns, const float *ops,
                                  int K, uint32_t *op_status, int32_t *order, int32_t *layer,
                                  int32_t *n_layers, uint32_t *gstatus, cudaStream_t stream);

/* Compatibility distance of every pair of P genomes (Alg. 1 speciates the
 * population by distances between networks; App. A names the disjoint and
 * homologous coefficients, 1.0 and 0.5 by default there).  For genomes A, B:
 *   delta = (c_d D_n + c_h H_n) / max(n_A, n_B) + (c_d D_c + c_h H_c) / max(m_A, m_B)
 * (a term is 0 when both counts are 0).  Node genes (n of them): the valid node
 * rows, keyed by node key.  Connection genes (m): the valid connection rows,
 * enabled or not, keyed by (in key, out key); the lowest row of a repeated
 * key counts once.  D = keys present in exactly one genome; H = sum over shared
 * keys of |b_A - b_B| + |r_A - r_B| + [act differs] + [agg differs] (0 for input
 * rows) for nodes, |w_A - w_B| + [enabled differs] for connections.
 *   nodes [P, N, 5], conns [P, C, 4] f32 as for neat_transform
 *   gstatus optional [P] u32 (from neat_transform or neat_transform_recurrent):
 *           a genome with a bit other than NEAT_G_CYCLE gets NaN distances;
 *           NULL: every genome is taken as valid
 *   dist    [P, P] f32 out, row-major; symmetric bit for bit, 0 on the diagonal
 *   scratch caller-owned device memory, 256-byte aligned, at least
 *           neat_distance_scratch_bytes(P, N, C) bytes
 * Plan-free; asynchronous on `stream`.  NEAT_ERR_WORKSPACE if the scratch is
 * too small, NEAT_ERR_UNSUPPORTED for sizes beyond the limits. */
size_t neat_distance_scratch_bytes(int P, int N, int C);
neat_status neat_distance(const float *nodes, const float *conns, const uint32_t *gstatus, int P,
                          int N, int C, int I, int O, float c_disjoint, float c_homologous,
                          float *dist, void *scratch, size_t scratch_bytes, cudaStream_t stream);

/* Measurement helper (the paper has no counterpart): shared-memory read
 * bandwidth, the peak of the on-chip term of the roofline.  Launches `blocks`
 * CTAs of 512 threads on `stream`; each CTA fills a 64 KiB shared array
 * (32-bit word w = w * 0x9E3779B1 mod 2^32) and each thread then reads
 * 8 * iters 16-byte words, consecutive threads on consecutive words (no bank
 * conflicts): words (t + 512 u + it) mod 4096 for u < 8, it < iters.  The XOR
 * of all words thread t read goes to sink[block * 512 + t] (device u32
 * [blocks * 512], caller-owned), so no read is optimised away.  Bytes read =
 * blocks * 512 * 128 * iters; time the launch with events on `stream`.
 * NEAT_ERR_ARG for blocks < 1, iters < 0 or a NULL/misaligned sink. */
neat_status neat_probe_smem_read(int blocks, int iters, uint32_t *sink, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* NEAT_H */
