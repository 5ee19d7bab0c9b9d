// Internal definitions shared by the library's kernels and host code.
//
// The transformed program (what Sec. 3.3's transformation stage produces: the
// topological order and the expanded connections C_exp) is stored per genome
// as a list of node records in canonical position order plus, for each node,
// its enabled incoming connections as (source position, weight) records.  This
// is C_exp without its O(N^2) dense storage: the column C_exp[:, k] of the
// paper becomes the contiguous edge range of node k.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/neat.h"
#include "act_math.cuh"

namespace neat {

// -- node record (16 B) -------------------------------------------------------
// meta bits: [0,14) in-degree, [16,20) activation id, [20,24) aggregation id,
// bit 24 = input node, bit 25 = valid position, bit 26 = a non-input node no
// output depends on (feed-forward transform only): a forward that returns
// only the outputs need not evaluate it.
constexpr uint32_t META_CNT_MASK = 0x3fffu;
constexpr uint32_t META_INPUT = 1u << 24;
constexpr uint32_t META_VALID = 1u << 25;
constexpr uint32_t META_DEAD = 1u << 26;
struct __align__(16) NodeRec {
  float bias;
  float resp;
  uint32_t in_begin;  // first incoming edge, relative to the genome's edge base
  uint32_t meta;
};
__host__ __device__ inline int meta_cnt(uint32_t m) { return int(m & META_CNT_MASK); }
__host__ __device__ inline int meta_act(uint32_t m) { return int((m >> 16) & 15u); }
__host__ __device__ inline int meta_agg(uint32_t m) { return int((m >> 20) & 15u); }

// -- edge record (8 B): source canonical position and weight -------------------
struct __align__(8) EdgeRec {
  uint32_t src;
  float w;
};

// -- per-genome header (48 B) ---------------------------------------------------
struct __align__(16) GenomeHdr {
  int V;         // valid nodes (0 for a rejected genome)
  int E;         // enabled connections
  int L;         // layers (frontiers)
  uint32_t status;
  int node_off;  // ragged-packed offsets (queue order)
  int edge_off;
  int nlive;     // non-input nodes some output depends on (the others: META_DEAD)
  int nch;       // 4-edge chunks of the level-synchronous form over those nodes:
                 // sum of ceil(indeg/4)
  int elive;     // enabled connections into those nodes
  int crows;     // value rows of the compiled program (0: none)
  int clayers;   // layers holding compiled nodes (their first nodes: Ws::clay)
  int cpairs;    // edge pairs of the compiled program
};

// -- compiled program (outputs-only walks) -----------------------------------------
// Built by the feed-forward transform for every valid genome: the nodes some
// output depends on, in canonical order, with their incoming edges in pairs,
// and a VALUE ROW per value instead of a position: rows 0..I-1 hold the
// inputs, rows I and I+1 the constants 0 and 1, and the node values take rows
// from I+2 on, a row being reused once the layer of the last node that reads
// it is done (a linear scan in canonical order, releases deferred to the end
// of each layer, so that the nodes of one layer may run concurrently).  The
// outputs keep their rows.
// Each node's edge list is padded to an even length with an edge that leaves
// the aggregate unchanged: weight 0 on the zero row for sum and mean, weight 1
// on the one row for product, a repeat of the last edge for max.
//   CNode.pairs = first pair (within the genome) | pair count << CN_PAIR_BITS
//   CNode.meta  = value row | activation << 20 | aggregation << 23 |
//                 (in-degree odd) << 25
//   pair (uint4) = (source row 0, w0, source row 1, w1)
// clay[g][k] = the first compiled node of the k-th layer that holds any
// (k < clayers), clay[g][clayers] = the compiled node count.
struct __align__(16) CNode {
  float bias, resp;
  uint32_t pairs;
  uint32_t meta;
};
constexpr uint32_t CN_PAIR_BITS = 17, CN_ROW_BITS = 20;
// pair capacity per genome: sum over nodes of ceil(in-degree / 2) <= (C + N) / 2
__host__ __device__ inline int cpair_cap(int N, int C) { return (C + N) / 2 + 1; }

// -- level-synchronous batches (small-S form) --------------------------------------
// Consecutive genomes of a layer-sorted queue are packed into small batches,
// one per warp at a time.  A batch program lives in the level arena as one
// contiguous, 16-byte aligned block:
//   BatchHead (48 B)
//   gio       int32[n_genomes*(1+I+O)] genome id, input slots, output slots
//   --- off_round: the head part above is staged into the warp's shared
//       memory (a bulk copy); the rest is read from global memory (L2), each
//       round's records one round ahead
//   rounds    uint32[n_rounds + 1]     first task | first chunk << 16
//   tasks     TaskRec[n_tasks]         non-input nodes, by (layer, activation
//                                      class, act, -cnt)
//   eslot     uint16[4 * n_chunks]     source value slot of each edge; the first
//                                      entry of a chunk carries the task's
//                                      aggregation in bits 12-13
//   ew        float[4 * n_chunks]      weight of each edge
struct __align__(16) BatchHead {
  int n_genomes, n_slots, n_rounds, n_tasks;
  int n_chunks, off_round, off_task, off_eslot;
  int off_gio, prog_bytes, off_ew;
  uint32_t act_mask;  // bit a set: some task has activation a
};
// where a batch program sits in the arena
struct __align__(16) BatchLoc {
  int off;    // byte offset in the arena
  int bytes;  // program bytes (multiple of 16)
  int head;   // bytes of the head part (= off_round, multiple of 16)
  int pad;
};

// Task record (16 B).  meta: [0,14) in-degree, [14,17) activation,
// [17,19) aggregation, [19,31) destination slot.
struct __align__(16) TaskRec {
  float bias;
  float resp;
  uint32_t chunk;  // first 4-edge chunk, batch-relative
  uint32_t meta;
};
constexpr int LVL_SLOT_BITS = 12;
constexpr int LVL_MAX_SLOTS = 1 << LVL_SLOT_BITS;  // 4096 value slots per batch
constexpr int LVL_MAX_GENOMES = 64;                // genomes per batch (hard cap)
// the plain form puts lanes over a node's incoming edges (one warp per
// sample) up to this many samples per genome, over samples above it
constexpr int PLAIN_EDGE_S_MAX = 8;
constexpr int LVL_CONST_SLOTS = 2;                 // slots 0 and 1: the constants 0 and 1
__host__ __device__ inline uint32_t task_meta(int cnt, int act, int agg, int slot) {
  return uint32_t(cnt) | (uint32_t(act) << 14) | (uint32_t(agg) << 17) | (uint32_t(slot) << 19);
}
__host__ __device__ inline int task_cnt(uint32_t m) { return int(m & 0x3fffu); }
__host__ __device__ inline int task_act(uint32_t m) { return int((m >> 14) & 7u); }
__host__ __device__ inline int task_agg(uint32_t m) { return int((m >> 17) & 3u); }
__host__ __device__ inline int task_slot(uint32_t m) { return int(m >> 19); }

// Bytes a genome contributes to a batch program (upper bound): 16 B per task,
// 24 B per 4-edge chunk, 4 B per genome id and I/O slot, and round-table
// entries (4 B each: one per layer, plus one per task for the rounds split at
// the chunk cap).  A batch program takes at most LVL_BATCH_FIXED (header and
// alignment of its five arrays) plus the sum of its genomes' bytes.
constexpr int LVL_BATCH_FIXED = 112;
__host__ __device__ inline int lvl_genome_bytes(int tasks, int nch, int L, int I, int O, bool ok) {
  const int b = 4 * (1 + I + O) + (ok ? 20 * tasks + 24 * nch + 4 * L + 4 : 4);
  return (b + 15) & ~15;
}
// largest genome bytes for N node rows and C connection rows: at most N - I
// tasks, sum over tasks of ceil(indeg / 4) <= (C + 3 (N - I)) / 4 chunks, N layers
inline int lvl_pb_max(int N, int C, int I, int O) {
  return lvl_genome_bytes(N - I, (C + 3 * (N - I)) / 4, N, I, O, true);
}
// per-warp program buffer: any single genome fits (the budget knob may ask
// for more, never for less)
inline int lvl_min_budget(int N, int C, int I, int O) {
  return (LVL_BATCH_FIXED + lvl_pb_max(N, C, I, O) + 127) & ~127;
}
constexpr int LVL_MIN_BUDGET = 8 * 1024;    // smallest budget knob (KiB granularity)
constexpr int LVL_MAX_BUDGET = 160 * 1024;  // largest budget knob
inline int lvl_budget(int N, int C, int I, int O, int knob_bytes = 0) {
  // the budget of an explicit knob; without one the transform searches for
  // the budget that fills the resident warps (k_lvl_plan), and this 16 KiB
  // (about five locomotion-sized genomes per warp batch, rounds of about 21
  // tasks and 35 chunks) is only the fallback value kept in the workspace
  const int want = knob_bytes > 0 ? knob_bytes : 16 * 1024;
  const int m = lvl_min_budget(N, C, I, O);
  return want > m ? ((want + 127) & ~127) : m;
}
// bytes of a warp's staged head part (header and I/O slots): room for at
// least one genome; the batch cut keeps every head within it
__host__ __device__ inline int lvl_head_cap(int I, int O) {
  const int one = (int(sizeof(BatchHead)) + 4 * (1 + I + O) + 15 + 127) & ~127;
  return one > 2048 ? one : 2048;
}
// value slots of a batch (>= N + the two constants: any single genome fits)
inline int lvl_slots(int N) { return N + LVL_CONST_SLOTS > 1024 ? N + LVL_CONST_SLOTS : 1024; }
// chunks of a round (>= the chunks of any one task: in-degree <= min(N - 1, C))
inline int lvl_pcap(int N, int C) {
  const int t = ((N - 1 < C ? N - 1 : C) + 3) / 4;
  return t > 128 ? t : 128;
}

// -- workspace layout ------------------------------------------------------------
struct Layout {
  size_t hdr, pnode, pedge, perow, prow, player, pio, qorder, qlvl, knode, kedge, kerow, counters;
  size_t base;                                 // bytes of the regions above
  size_t lvl_goff, lvl_first, lvl_loc, lvl_arena;  // small-S schedule
  size_t lvl_arena_bytes;
  int lvl_max_batches;
  size_t core;                       // bytes of everything above
  size_t cnode, cpair, cout, clay;      // compiled program (after core)
  size_t sp_scratch, sp_scratch_bytes;  // per-warp node value slots
  size_t total;
};

// Sample-parallel value arrays: SP_SCRATCH_WARP_SAMPLES / 32 warp slots of
// [N][32] floats in the workspace (fewer slots when a lane evaluates several
// samples); a warp keeps the node values of the genome it evaluates in its
// slot, where they stay L1/L2-resident while in use.  10,240 one-sample
// slots: enough for every resident warp of the recurrent forward (32 a SM,
// two value buffers each; with 8,192 its grid stopped at 24 a SM: 2.12 vs
// 1.95 ms on 10,000 cyclic genomes) and of the HyperNEAT query.
constexpr size_t SP_SCRATCH_WARP_SAMPLES = 10240 * 32;
inline size_t sp_scratch_bytes(int N) { return SP_SCRATCH_WARP_SAMPLES * size_t(N) * sizeof(float); }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline Layout make_layout(int P, int N, int C, int I, int O) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t p = size_t(P);
  L.hdr = take(sizeof(GenomeHdr) * p);
  L.pnode = take(sizeof(NodeRec) * p * N);
  L.pedge = take(sizeof(EdgeRec) * p * C);
  L.perow = take(sizeof(int32_t) * p * C);
  L.prow = take(sizeof(int32_t) * p * N);
  L.player = take(sizeof(int32_t) * p * N);
  L.pio = take(sizeof(int32_t) * p * (I + O));
  L.qorder = take(sizeof(int32_t) * (p + 1));
  L.qlvl = take(sizeof(int32_t) * (p + 1));
  L.knode = take(sizeof(NodeRec) * p * N);
  L.kedge = take(sizeof(EdgeRec) * p * C);
  L.kerow = take(sizeof(int32_t) * p * C);
  L.counters = take(sizeof(uint32_t) * 64);
  L.base = off;
  // small-S schedule: at most one batch per genome; a batch program is at
  // most LVL_BATCH_FIXED + the bytes of its genomes
  L.lvl_max_batches = int(p) + 1;
  L.lvl_goff = take(sizeof(int32_t) * (p + 1));
  L.lvl_first = take(sizeof(int32_t) * (size_t(L.lvl_max_batches) + 2));
  L.lvl_loc = take(sizeof(BatchLoc) * (size_t(L.lvl_max_batches) + 1));
  L.lvl_arena_bytes = p * size_t(lvl_pb_max(N, C, I, O) + LVL_BATCH_FIXED) + 256;
  L.lvl_arena = take(L.lvl_arena_bytes);
  L.core = off;
  L.cnode = take(sizeof(CNode) * p * N);
  L.cpair = take(sizeof(uint4) * p * size_t(cpair_cap(N, C)));
  L.cout = take(sizeof(int32_t) * p * O);
  L.clay = take(sizeof(int32_t) * p * (N + 1));
  L.sp_scratch_bytes = sp_scratch_bytes(N);
  L.sp_scratch = take(L.sp_scratch_bytes);
  L.total = off;
  return L;
}

// Device-side view of a plan's workspace.
struct Ws {
  GenomeHdr *hdr;
  NodeRec *pnode;
  EdgeRec *pedge;
  int32_t *perow;
  int32_t *prow;
  int32_t *pio;
  int32_t *qorder;
  NodeRec *knode;
  EdgeRec *kedge;
  int32_t *kerow;
  uint32_t *counters;
  int32_t *player;
  int32_t *qlvl;
  int32_t *lvl_goff;
  int32_t *lvl_first;
  BatchLoc *lvl_loc;
  unsigned char *lvl_arena;
  CNode *cnode;       // compiled program [P][N], pairs [P][cpair_cap], output
  uint4 *cpair;       // rows [P][O], layer starts [P][N + 1] (nullptr: none)
  int32_t *cout;
  int32_t *clay;
  float *sp_scratch;  // per-warp node value slots (nullptr: none)
  size_t sp_scratch_floats;
  int lvl_budget;  // bytes of a batch program buffer (per warp), set at transform time
  int lvl_slots;   // value slots of a batch
  int lvl_pcap;    // chunks of a round
  int lvl_max_batches;
  int prune;  // skip the nodes no output depends on (set at transform time)
  int P, N, C, I, O;
};

inline Ws make_ws(void *base, const Layout &L, int P, int N, int C, int I, int O) {
  char *b = static_cast<char *>(base);
  Ws w;
  w.hdr = reinterpret_cast<GenomeHdr *>(b + L.hdr);
  w.pnode = reinterpret_cast<NodeRec *>(b + L.pnode);
  w.pedge = reinterpret_cast<EdgeRec *>(b + L.pedge);
  w.perow = reinterpret_cast<int32_t *>(b + L.perow);
  w.prow = reinterpret_cast<int32_t *>(b + L.prow);
  w.pio = reinterpret_cast<int32_t *>(b + L.pio);
  w.qorder = reinterpret_cast<int32_t *>(b + L.qorder);
  w.knode = reinterpret_cast<NodeRec *>(b + L.knode);
  w.kedge = reinterpret_cast<EdgeRec *>(b + L.kedge);
  w.kerow = reinterpret_cast<int32_t *>(b + L.kerow);
  w.counters = reinterpret_cast<uint32_t *>(b + L.counters);
  w.player = reinterpret_cast<int32_t *>(b + L.player);
  w.qlvl = reinterpret_cast<int32_t *>(b + L.qlvl);
  w.lvl_goff = reinterpret_cast<int32_t *>(b + L.lvl_goff);
  w.lvl_first = reinterpret_cast<int32_t *>(b + L.lvl_first);
  w.lvl_loc = reinterpret_cast<BatchLoc *>(b + L.lvl_loc);
  w.lvl_arena = reinterpret_cast<unsigned char *>(b + L.lvl_arena);
  w.cnode = reinterpret_cast<CNode *>(b + L.cnode);
  w.cpair = reinterpret_cast<uint4 *>(b + L.cpair);
  w.cout = reinterpret_cast<int32_t *>(b + L.cout);
  w.clay = reinterpret_cast<int32_t *>(b + L.clay);
  w.sp_scratch = L.sp_scratch_bytes ? reinterpret_cast<float *>(b + L.sp_scratch) : nullptr;
  w.sp_scratch_floats = L.sp_scratch_bytes / sizeof(float);
  w.lvl_budget = lvl_budget(N, C, I, O);
  w.lvl_slots = lvl_slots(N);
  w.lvl_pcap = lvl_pcap(N, C);
  w.prune = 0;
  w.lvl_max_batches = L.lvl_max_batches;
  w.P = P; w.N = N; w.C = C; w.I = I; w.O = O;
  return w;
}

// counters[] slots (CTR_LVL_ITEM and CTR_LVL_DONE together: the level
// forward's 64-bit claim counter)
constexpr int CTR_FWD_ITEM = 0, CTR_FWD_DONE = 1, CTR_HN_ITEM = 2, CTR_HN_DONE = 3,
              CTR_LVL_ITEM = 4, CTR_LVL_DONE = 5, CTR_FWD_BIG = 6, CTR_SP_NBIG = 7,
              CTR_NBATCH = 8, CTR_ERR = 9, CTR_REC_ITEM = 10, CTR_REC_DONE = 11;
// genomes of at least this cost (sp_cost) are evaluated by a whole CTA in the
// sample-parallel forward (counters[CTR_SP_NBIG] of them, a queue prefix);
// measured best on the uneven workload: 2048 evaluating every node, 512 with
// the nodes no output depends on skipped (the CTA-wide walk then covers the
// long per-warp items that otherwise end the launch)
constexpr int SP_COOP_COST = 2048, SP_COOP_COST_PRUNED = 512;
__host__ __device__ inline int sp_coop_cost(bool prune) {
  return prune ? SP_COOP_COST_PRUNED : SP_COOP_COST;
}
// cost of a genome in the sample-parallel forward: edges + 2 * nodes of the
// part some output depends on, plus a quarter per skipped position
__host__ __device__ inline int sp_cost(const GenomeHdr &h) {
  return h.elive + 2 * h.nlive + (h.V - h.nlive) / 4;
}
// error bits in counters[CTR_ERR] (the NEAT_DEV_* bits of neat.h)
constexpr uint32_t ERR_TMA_TIMEOUT = NEAT_DEV_TIMEOUT, ERR_SP_NO_SCRATCH = NEAT_DEV_NO_SCRATCH;

// -- selects on small ids ------------------------------------------------------------
// `id == K ? x : y` as one predicated select written in PTX.  A chain of plain
// selects on the same id (activation or aggregation) is merged by the
// compiler into a multiway switch, i.e. an indirect jump, which costs a warp
// ~270 cycles on this GPU even when all lanes agree; these stay selects.
template <int K>
__device__ __forceinline__ float sel_eq(int id, float x, float y) {
  float r;
  asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %1, %2;\n\tselp.f32 %0, %3, %4, p;\n\t}"
      : "=f"(r)
      : "r"(id), "n"(K), "f"(x), "f"(y));
  return r;
}
// c ? x : y for a condition the compiler must not turn into a branch
__device__ __forceinline__ float sel_if(bool c, float x, float y) {
  float r;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %1, 0;\n\tselp.f32 %0, %2, %3, p;\n\t}"
      : "=f"(r)
      : "r"(int(c)), "f"(x), "f"(y));
  return r;
}
// id == k as an opaque test (an if-chain of these stays a chain of two-way
// branches instead of becoming a multiway switch)
__device__ __forceinline__ bool is_id(int id, int k) {
  int r;
  asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %1, %2;\n\tselp.s32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(id), "r"(k));
  return r != 0;
}
// bit `id` of `mask` (an opaque test: branches on it stay two-way)
__device__ __forceinline__ bool bit_of(uint32_t mask, int id) {
  uint32_t r;
  asm("{\n\t.reg .u32 t;\n\tshr.b32 t, %1, %2;\n\tand.b32 %0, t, 1;\n\t}"
      : "=r"(r)
      : "r"(mask), "r"(id));
  return r != 0u;
}

// -- activations (textbook forms, evaluated by the methods of act_math.cuh) --------
constexpr uint32_t ACT_BIT_EXP = (1u << NEAT_ACT_SIGMOID) | (1u << NEAT_ACT_TANH) |
                                 (1u << NEAT_ACT_GAUSSIAN);  // the functions built on e^x
constexpr uint32_t ACT_BIT_SIN = 1u << NEAT_ACT_SIN;

// argument of the one exponential an activation needs: e^{-z} (sigmoid),
// e^{-2|z|} (tanh), e^{-z^2} (gaussian); 0 for the others
__device__ __forceinline__ float act_exp_arg(int a, float z) {
  float x = sel_eq<NEAT_ACT_SIGMOID>(a, -z, 0.0f);
  x = sel_eq<NEAT_ACT_TANH>(a, -2.0f * fabsf(z), x);
  return sel_eq<NEAT_ACT_GAUSSIAN>(a, -(z * z), x);
}


// act_a(z) for an activation id a in [0, 6] (the transform rejects others)
// where every lane of the warp evaluates the same activation (the
// sample-parallel, HyperNEAT, recurrent, backward and substrate kernels):
// only its own function runs, with the CUDA math library's functions.  The
// dispatch is one multiway branch: in these kernels many warps are resident,
// so its latency is hidden, and it costs fewer instructions than a chain of
// tests (the level kernel, whose lanes mix activations, uses act_lanes).
__device__ __forceinline__ float act_apply(int a, float z) {
  switch (a) {
    case NEAT_ACT_IDENTITY: return z;
    case NEAT_ACT_SIGMOID: return 1.0f / (1.0f + expf(-z));
    case NEAT_ACT_TANH: return tanhf(z);
    case NEAT_ACT_RELU: return fmaxf(z, 0.0f);
    case NEAT_ACT_SIN: return sinf(z);
    case NEAT_ACT_GAUSSIAN: return expf(-(z * z));
    case NEAT_ACT_ABS: return fabsf(z);
  }
  return __int_as_float(0x7fc00000);
}

// act applied to n values with one dispatch (the same functions as act_apply)
template <int n>
__device__ __forceinline__ void act_apply_n(int a, float (&z)[n]) {
  switch (a) {
    case NEAT_ACT_IDENTITY: return;
    case NEAT_ACT_SIGMOID:
#pragma unroll
      for (int j = 0; j < n; ++j) z[j] = 1.0f / (1.0f + expf(-z[j]));
      return;
    case NEAT_ACT_TANH:
#pragma unroll
      for (int j = 0; j < n; ++j) z[j] = tanhf(z[j]);
      return;
    case NEAT_ACT_RELU:
#pragma unroll
      for (int j = 0; j < n; ++j) z[j] = fmaxf(z[j], 0.0f);
      return;
    case NEAT_ACT_SIN:
#pragma unroll
      for (int j = 0; j < n; ++j) z[j] = sinf(z[j]);
      return;
    case NEAT_ACT_GAUSSIAN:
#pragma unroll
      for (int j = 0; j < n; ++j) z[j] = expf(-(z[j] * z[j]));
      return;
    case NEAT_ACT_ABS:
#pragma unroll
      for (int j = 0; j < n; ++j) z[j] = fabsf(z[j]);
      return;
  }
#pragma unroll
  for (int j = 0; j < n; ++j) z[j] = __int_as_float(0x7fc00000);
}

// d act / dz given z and v = act(z) (one activation for the whole warp)
__device__ __forceinline__ float act_deriv(int a, float z, float v) {
  switch (a) {
    case NEAT_ACT_IDENTITY: return 1.0f;
    case NEAT_ACT_SIGMOID: return v * (1.0f - v);
    case NEAT_ACT_TANH: return 1.0f - v * v;
    case NEAT_ACT_RELU: return z > 0.0f ? 1.0f : 0.0f;
    case NEAT_ACT_SIN: return cosf(z);
    case NEAT_ACT_GAUSSIAN: return -2.0f * z * v;
    case NEAT_ACT_ABS: return z > 0.0f ? 1.0f : (z < 0.0f ? -1.0f : 0.0f);
  }
  return __int_as_float(0x7fc00000);
}

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// NEAT_OK for cudaSuccess; otherwise records e for neat_last_cuda_error() (per
// host thread) and returns NEAT_ERR_CUDA
neat_status cuda_error_status(cudaError_t e);

// -- launch wrappers (defined in the .cu files) ------------------------------------
// recurrent != 0: no topological order (cycles legal); every valid node in
// ascending key forms one frontier; order / layer / n_layers may be null
cudaError_t launch_transform(const Ws &w, const float *nodes, const float *conns, int32_t *order,
                             int32_t *layer, int32_t *n_layers, uint32_t *gstatus,
                             cudaStream_t st, int recurrent = 0);
cudaError_t launch_queue_build(const Ws &w, int mode, cudaStream_t st);
// Sample-parallel launch shape: `spl` samples per lane (1, 2, 4); genomes
// with V <= vcap keep their values in shared memory, the others in the
// warp's workspace slot (vcap 0: every genome in the workspace, N: none).
struct SpShape {
  int warps, spl, vcap, grid;
  int coop;  // CTA-wide evaluation of the most expensive genomes (needs value slots)
};
cudaError_t launch_forward_sp(const Ws &w, const float *inputs, int64_t stride, int S,
                              float *outputs, float *saved, const SpShape &sh, cudaStream_t st);
size_t forward_sp_smem(int vcap, int warps, int spl);
// warp slots of the workspace value array for `spl` samples per lane
inline int sp_scratch_slots(const Ws &w, int spl) {  // slots of N + 2 rows
  return w.sp_scratch ? int(w.sp_scratch_floats / (size_t(w.N + 2) * 32 * spl)) : 0;
}
cudaError_t launch_forward_plain(const Ws &w, const float *inputs, int64_t stride, int S,
                                 float *outputs, cudaStream_t st);
// structure check (neat_plan_validate): NEAT_BAD_* bits OR-ed into *bits
// (zeroed first); feedforward = 1 after neat_transform, 0 after the
// recurrent transform (no compiled programs or batches)
cudaError_t launch_validate(const Ws &w, const Layout &L, int feedforward, uint32_t *bits,
                            int sm_count, cudaStream_t st);
// recurrent calculation: T synchronous iterations, spl (1 or 2) samples per
// lane, `warps` per CTA, `grid` CTAs (grid * warps <= sp_scratch_slots(w,
// 2 * spl): two value buffers per warp)
cudaError_t launch_forward_recurrent(const Ws &w, const float *inputs, int64_t stride, int S,
                                     int T, float *outputs, int spl, int warps, int grid,
                                     cudaStream_t st);
int forward_rec_occupancy(int warps, int spl);
// HyperNEAT two-sheet substrate: y = act(x W) per genome
cudaError_t launch_substrate(const float *w, int P, int K, const float *x, int64_t stride, int S,
                             int act, float *y, cudaStream_t st);
// tensorized operations (Sec. 3.2) in place, one warp per genome
cudaError_t launch_apply_ops(float *nodes, float *conns, int P, int N, int C, const float *ops,
                             int K, uint32_t *op_status, cudaStream_t st);
// out [n] = sum over the P genomes of x [P, n] (ascending genome order,
// double-precision accumulation, one rounding)
cudaError_t launch_sum_genomes(const float *x, int P, int64_t n, float *out, int sm_count,
                               cudaStream_t st);
// Backward: `warps` per CTA.  global_values = false: one CTA per genome with
// smem_bytes of dynamic shared memory (at least backward_smem(N, C, 1)); a
// genome runs on as many warps as blocks of its size fit in smem_bytes.
// global_values = true: grid_ctas CTAs with backward_fixed_smem(N, C) bytes of
// shared memory (the records and pull lists) walk the queue, each warp's
// arrays in a workspace slot of backward_slot_floats(N, C) floats (grid_ctas *
// warps slots must fit in sp_scratch).
cudaError_t launch_backward(const Ws &w, const float *inputs, int64_t stride, int S,
                            const float *grad_out, const float *saved, float *gw, float *gb,
                            float *gr, float *gi, int warps, int smem_bytes, bool global_values,
                            int grid_ctas, cudaStream_t st);
size_t backward_smem(int N, int C, int warps);
size_t backward_fixed_smem(int N, int C);
size_t backward_slot_floats(int N, int C);
int backward_occupancy(bool global_values, int warps, int smem_bytes);
// HyperNEAT query: spl queries per lane (1, 2 or 4), `ctas` CTAs of `warps`
// warps with smem_bytes of dynamic shared memory (>= hn_prog_bytes(N, C): a
// compiled program's records and pairs).  A genome whose value array does not
// fit next to its program uses the warp's workspace slot instead (unless every
// genome fits, ctas * warps <= sp_scratch_slots(w, spl)).
__host__ __device__ inline int hn_prog_bytes(int N, int C) {
  return N * 16 + cpair_cap(N, C) * 16;
}

cudaError_t launch_hyperneat(const Ws &w, int grid, float thresh, float *weights, int spl,
                             int warps, int ctas, int smem_bytes, cudaStream_t st);
// one-time kernel attributes and occupancy queries (host side)
cudaError_t transform_set_smem_limit(int bytes);
size_t transform_smem(int N, int C);
cudaError_t forward_set_smem_limit(int bytes);
cudaError_t backward_set_smem_limit(int bytes);
int forward_sp_occupancy(int warps, size_t smem, int spl);
int hyperneat_occupancy(int spl, int warps, size_t smem);
// level-synchronous small-S form
// level batches: target > 0 picks the smallest budget (from budget_lo up)
// whose cut gives at most `target` batches; target 0 uses w.lvl_budget
cudaError_t launch_lvl_build(const Ws &w, int target, int budget_lo, cudaStream_t st);
// shared memory of one warp of the level-synchronous forward: its staged head
// part, value slots and chunk partials for st_samples per tile
size_t lvl_warp_bytes(const Ws &w, int st_samples);
size_t lvl_vals_bytes(const Ws &w, int st_samples);
// `warps` per CTA, each owning lvl_warp_bytes; a staging wait gives up after
// `polls` polls (0: at once)
cudaError_t launch_forward_lvl(const Ws &w, const float *inputs, int64_t stride, int S,
                               float *outputs, int warps, int grid, int polls, int pdl,
                               cudaStream_t st);
cudaError_t lvl_set_smem_limit(int bytes);
int forward_lvl_occupancy(int warps, size_t smem, int st_samples);
int lvl_tile(int S);

}  // namespace neat

namespace neat {
// Raise a kernel's dynamic shared-memory limit to what the device allows
// next to the kernel's own static shared memory.
template <class K>
inline cudaError_t set_dyn_smem_limit(K kernel, int optin_bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin_bytes - int(a.sharedSizeBytes));
}
}  // namespace neat
