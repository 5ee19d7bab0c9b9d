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

namespace neat {

// -- node record (16 B) -------------------------------------------------------
// meta bits: [0,14) in-degree, [16,20) activation id, [20,24) aggregation id,
// bit 24 = input node, bit 25 = valid position.
constexpr uint32_t META_CNT_MASK = 0x3fffu;
constexpr uint32_t META_INPUT = 1u << 24;
constexpr uint32_t META_VALID = 1u << 25;
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

// -- per-genome header (32 B) ---------------------------------------------------
struct __align__(16) GenomeHdr {
  int V;         // valid nodes (0 for a rejected genome)
  int E;         // enabled connections
  int L;         // layers (frontiers)
  uint32_t status;
  int node_off;  // ragged-packed offsets (queue order)
  int edge_off;
  int lvl_off;   // level-synchronous schedule (small-S form): batch of this genome
  int pad;
};

// -- level-synchronous batch header (small-S form) -------------------------------
struct __align__(16) BatchHdr {
  int n_genomes;   // genomes in the batch
  int n_slots;     // node-value slots used by the batch
  int n_rounds;    // level rounds
  int n_tasks;     // node tasks over all rounds
  int n_edges;     // edge records over all tasks
  int prog_off;    // byte offset of the batch program in the schedule arena
  int prog_bytes;  // bytes of the batch program (multiple of 16)
  int first_q;     // queue index of the batch's first genome
};

// Task record of the level-synchronous form (16 B).
struct __align__(16) TaskRec {
  float bias;
  float resp;
  uint32_t ebeg;   // first edge (batch-relative)
  uint32_t meta;   // cnt | act << 16 | agg << 20 | dst slot << ... (see below)
};
// TaskRec.meta: [0,12) count, [12,16) act, [16,20) agg ... slot stored apart.

// -- workspace layout ------------------------------------------------------------
struct Layout {
  size_t hdr, pnode, pedge, perow, prow, pio, qorder, knode, kedge, kerow, counters;
  size_t lvl_bhdr, lvl_arena, lvl_io;   // small-S schedule
  size_t lvl_arena_bytes;
  size_t total;
};

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
  L.pio = take(sizeof(int32_t) * p * (I + O));
  L.qorder = take(sizeof(int32_t) * (p + 1));
  L.knode = take(sizeof(NodeRec) * p * N);
  L.kedge = take(sizeof(EdgeRec) * p * C);
  L.kerow = take(sizeof(int32_t) * p * C);
  L.counters = take(sizeof(uint32_t) * 64);
  // small-S schedule: one batch per genome at most; per task 16 B + slot 2 B,
  // per edge 6 B, per round 4 B, plus alignment slack per batch.
  L.lvl_bhdr = take(sizeof(BatchHdr) * (p + 1));
  L.lvl_arena_bytes = p * (size_t(N) * 20 + size_t(C) * 8 + size_t(N) * 8 + 256);
  L.lvl_arena = take(L.lvl_arena_bytes);
  L.lvl_io = take(sizeof(int32_t) * p * (I + O));
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
  BatchHdr *lvl_bhdr;
  unsigned char *lvl_arena;
  int32_t *lvl_io;
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
  w.lvl_bhdr = reinterpret_cast<BatchHdr *>(b + L.lvl_bhdr);
  w.lvl_arena = reinterpret_cast<unsigned char *>(b + L.lvl_arena);
  w.lvl_io = reinterpret_cast<int32_t *>(b + L.lvl_io);
  w.P = P; w.N = N; w.C = C; w.I = I; w.O = O;
  return w;
}

// counters[] slots
constexpr int CTR_FWD_ITEM = 0, CTR_FWD_DONE = 1, CTR_HN_ITEM = 2, CTR_HN_DONE = 3,
              CTR_LVL_ITEM = 4, CTR_LVL_DONE = 5, CTR_NBATCH = 8;

// -- activations (textbook forms; accurate libm-style device functions) -----------
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

// d act / dz given z and v = act(z)
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

// -- launch wrappers (defined in the .cu files) ------------------------------------
cudaError_t launch_transform(const Ws &w, const float *nodes, const float *conns, int32_t *order,
                             int32_t *layer, int32_t *n_layers, uint32_t *gstatus,
                             cudaStream_t st);
cudaError_t launch_queue_build(const Ws &w, int mode, cudaStream_t st);
cudaError_t launch_forward_sp(const Ws &w, const float *inputs, int64_t stride, int S,
                              float *outputs, float *saved, int warps, int grid,
                              cudaStream_t st);
size_t forward_sp_smem(int N, int warps);
cudaError_t launch_forward_plain(const Ws &w, const float *inputs, int64_t stride, int S,
                                 float *outputs, cudaStream_t st);
cudaError_t launch_backward(const Ws &w, const float *inputs, int64_t stride, int S,
                            const float *grad_out, const float *saved, float *gw, float *gb,
                            float *gr, float *gi, int warps, cudaStream_t st);
size_t backward_smem(int N, int C, int warps);
cudaError_t launch_hyperneat(const Ws &w, int grid, float thresh, float *weights, int warps,
                             int ctas, cudaStream_t st);
// one-time kernel attributes and occupancy queries (host side)
cudaError_t transform_set_smem_limit(int bytes);
size_t transform_smem(int N, int C);
cudaError_t forward_set_smem_limit(int bytes);
cudaError_t backward_set_smem_limit(int bytes);
int forward_sp_occupancy(int warps, size_t smem);
int hyperneat_occupancy(int warps, size_t smem);

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
