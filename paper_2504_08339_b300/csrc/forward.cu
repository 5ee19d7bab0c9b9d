// Calculation stage (TensorNEAT Sec. 3.3): v[inputs] = I, then in canonical
// order v[k] = act(b + r * agg_e(w_e * v[src_e])); O = v[outputs].
//
// Sample-parallel forms: a warp owns one genome and 32 samples; lane l walks
// the genome's program for sample l with node values laid out
// [position][lane] (one 128-byte line per position), program records read
// with warp-uniform (broadcast) loads.  No lane ever reads another lane's
// values, so the walk needs no synchronisation at all.
//
//  k_forward_sp     persistent grid, warps claim (genome, 32 * SPL-sample
//                   tile) items from a device work queue in size-sorted order
//                   over the ragged-packed programs (the batched form); node
//                   values in the warp's workspace slot, cached by L1.
//  k_forward_plain  one CTA per (genome, tile) over the padded programs,
//                   visiting all N padded positions (the plain form).
//  k_forward_plain_edges  the plain form for S <= PLAIN_EDGE_S_MAX: one warp
//                   per (genome, sample), lanes over a node's incoming edges
//                   (a butterfly combines their partial aggregates).
//  k_hyperneat      the batched form with inputs generated in the kernel
//                   (substrate coordinates), several queries per lane and a
//                   threshold epilogue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "neat_internal.cuh"

namespace neat {
namespace {

__device__ __forceinline__ EdgeRec ld_edge(const EdgeRec *p) {
  const uint2 x = __ldg(reinterpret_cast<const uint2 *>(p));
  EdgeRec e;
  e.src = x.x;
  e.w = __uint_as_float(x.y);
  return e;
}

__device__ __forceinline__ NodeRec ld_node(const NodeRec *p) {
  const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
  NodeRec n;
  n.bias = __uint_as_float(x.x);
  n.resp = __uint_as_float(x.y);
  n.in_begin = x.z;
  n.meta = x.w;
  return n;
}

// Aggregated inputs a[j] = agg_e(w_e * v[src_e]) of one node for this lane's
// SPL samples; vl = v + lane, v the warp's [position][SPL][32] value array
// (shared or global memory).  Every sample uses the same rounding order
// whatever SPL.
template <int SPL>
__device__ __forceinline__ void node_agg(const NodeRec &n, const EdgeRec *__restrict__ er,
                                         const float *vl, float (&a)[SPL]) {
  constexpr int RS = 32 * SPL;  // floats per position
  const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
  const EdgeRec *e = er + n.in_begin;
  if (cnt == 0) {
#pragma unroll
    for (int j = 0; j < SPL; ++j) a[j] = 0.0f;
    return;
  }
  // U edges per block: their record and value loads are all issued before the
  // first use (more loads in flight); sums keep two accumulators, even edges
  // into a0 and odd edges into a1, so the rounding order does not depend on U
  constexpr int U = SPL == 1 ? 8 : (SPL == 2 ? 4 : 2);
  if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
    float a0[SPL], a1[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) a0[j] = a1[j] = 0.0f;
    int k = 0;
    for (; k + U <= cnt; k += U) {
      EdgeRec ee[U];
      float vv[U][SPL];
#pragma unroll
      for (int u = 0; u < U; ++u) ee[u] = ld_edge(e + k + u);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < SPL; ++j) vv[u][j] = vl[ee[u].src * RS + j * 32];
#pragma unroll
      for (int u = 0; u < U; u += 2)
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
          a0[j] = fmaf(ee[u].w, vv[u][j], a0[j]);
          a1[j] = fmaf(ee[u + 1].w, vv[u + 1][j], a1[j]);
        }
    }
    for (; k + 1 < cnt; k += 2) {
      const EdgeRec e0 = ld_edge(e + k), e1 = ld_edge(e + k + 1);
      const float *p0 = vl + e0.src * RS, *p1 = vl + e1.src * RS;
#pragma unroll
      for (int j = 0; j < SPL; ++j) {
        a0[j] = fmaf(e0.w, p0[j * 32], a0[j]);
        a1[j] = fmaf(e1.w, p1[j * 32], a1[j]);
      }
    }
    if (k < cnt) {
      const EdgeRec e0 = ld_edge(e + k);
      const float *p0 = vl + e0.src * RS;
#pragma unroll
      for (int j = 0; j < SPL; ++j) a0[j] = fmaf(e0.w, p0[j * 32], a0[j]);
    }
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
      const float s = a0[j] + a1[j];
      a[j] = agg == NEAT_AGG_MEAN ? s / float(cnt) : s;
    }
    return;
  }
  // product and max: folds in edge order, loads issued U edges ahead
  const bool prod = agg == NEAT_AGG_PRODUCT;
  int k = 0;
  if (prod) {
#pragma unroll
    for (int j = 0; j < SPL; ++j) a[j] = 1.0f;
  } else {
    const EdgeRec e0 = ld_edge(e);
    const float *p0 = vl + e0.src * RS;
#pragma unroll
    for (int j = 0; j < SPL; ++j) a[j] = e0.w * p0[j * 32];
    k = 1;
  }
  for (; k + U <= cnt; k += U) {
    EdgeRec ee[U];
    float vv[U][SPL];
#pragma unroll
    for (int u = 0; u < U; ++u) ee[u] = ld_edge(e + k + u);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < SPL; ++j) vv[u][j] = vl[ee[u].src * RS + j * 32];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < SPL; ++j)
        a[j] = prod ? a[j] * (ee[u].w * vv[u][j]) : fmaxf(a[j], ee[u].w * vv[u][j]);
  }
  for (; k < cnt; ++k) {
    const EdgeRec e0 = ld_edge(e + k);
    const float *p0 = vl + e0.src * RS;
#pragma unroll
    for (int j = 0; j < SPL; ++j)
      a[j] = prod ? a[j] * (e0.w * p0[j * 32]) : fmaxf(a[j], e0.w * p0[j * 32]);
  }
}

// Value (and saved aggregate) of the node at position p for this lane's SPL
// samples; inputs are left alone, and so are nodes no output depends on
// unless the aggregates are saved.
template <bool SAVE, int SPL>
__device__ __forceinline__ void eval_node(const NodeRec &n, int p, const EdgeRec *__restrict__ er,
                                          float *vl, float *const (&scol)[SPL], int S) {
  if (n.meta & (SAVE ? META_INPUT : META_INPUT | META_DEAD)) return;
  float a[SPL];
  node_agg<SPL>(n, er, vl, a);
  const int act = meta_act(n.meta);
#pragma unroll
  for (int j = 0; j < SPL; ++j) {
    vl[(p * SPL + j) * 32] = act_apply(act, fmaf(n.resp, a[j], n.bias));
    if (SAVE && scol[j] != nullptr) scol[j][size_t(p) * S] = a[j];
  }
}

// Walk positions [0, V) of a ragged program (inputs already in v); vl = v +
// lane.  SAVE: scol[j][p * S] (scol[j] nullptr for an inactive sample)
// receives the aggregate of position p for sample j.
template <bool SAVE, int SPL>
__device__ __forceinline__ void walk_program(const NodeRec *__restrict__ nr,
                                             const EdgeRec *__restrict__ er, int V, float *vl,
                                             float *const (&scol)[SPL], int S) {
  for (int p = 0; p < V; ++p) eval_node<SAVE, SPL>(ld_node(nr + p), p, er, vl, scol, S);
}

__device__ __forceinline__ void grid_done_reset(uint32_t *item_ctr, uint32_t *done_ctr,
                                                uint32_t *extra_ctr = nullptr) {
  // the last CTA to finish returns the queue counters to zero, so every launch
  // (including graph replays) starts from a clean queue
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(done_ctr, 1u);
    if (t == gridDim.x - 1) {
      atomicExch(item_ctr, 0u);
      if (extra_ctr != nullptr) atomicExch(extra_ctr, 0u);
      atomicExch(done_ctr, 0u);
    }
  }
}

// the SPL values of one lane in a staged value row (one vector load / store)
template <int SPL>
struct HnVec;
template <>
struct HnVec<1> {
  __device__ __forceinline__ static void ld(const char *p, float (&x)[1]) {
    x[0] = *reinterpret_cast<const float *>(p);
  }
  __device__ __forceinline__ static void st(char *p, const float (&x)[1]) {
    *reinterpret_cast<float *>(p) = x[0];
  }
};
template <>
struct HnVec<2> {
  __device__ __forceinline__ static void ld(const char *p, float (&x)[2]) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    x[0] = v.x;
    x[1] = v.y;
  }
  __device__ __forceinline__ static void st(char *p, const float (&x)[2]) {
    *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]);
  }
};
template <>
struct HnVec<4> {
  __device__ __forceinline__ static void ld(const char *p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  }
  __device__ __forceinline__ static void st(char *p, const float (&x)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
  }
};

// a[j] = fma(w, x[j], a[j]) for the SPL queries, two per instruction (the
// paired fp32 FMA; each component rounds as fmaf)
template <int SPL>
__device__ __forceinline__ void hn_fma(float w, const float (&x)[SPL], float (&a)[SPL]) {
  if constexpr (SPL == 1) {
    a[0] = fmaf(w, x[0], a[0]);
  } else {
#pragma unroll
    for (int j = 0; j < SPL; j += 2) {
      const float2 r = __ffma2_rn(make_float2(w, w), make_float2(x[j], x[j + 1]),
                                  make_float2(a[j], a[j + 1]));
      a[j] = r.x;
      a[j + 1] = r.y;
    }
  }
}

// Addresses of a walk's records and values: generic 64-bit pointers when they
// live in global memory (GLOBAL: records through the read-only path, values
// in the workspace slots), 32-bit shared-window addresses when both are
// staged in shared memory (explicit shared-space instructions: fewer address
// instructions than generic accesses; volatile with a memory clobber, so
// they keep their order with the walk's other shared accesses).
template <bool GLOBAL>
using waddr_t = std::conditional_t<GLOBAL, const char *, uint32_t>;
template <bool GLOBAL>
__device__ __forceinline__ waddr_t<GLOBAL> waddr(const void *p) {
  if constexpr (GLOBAL) return static_cast<const char *>(p);
  else return uint32_t(__cvta_generic_to_shared(p));
}
template <bool GLOBAL>
__device__ __forceinline__ uint4 w_ld16(waddr_t<GLOBAL> a) {
  if constexpr (GLOBAL) {
    return __ldg(reinterpret_cast<const uint4 *>(a));
  } else {
    uint4 r;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "r"(a)
                 : "memory");
    return r;
  }
}
template <int SPL, bool GLOBAL>
__device__ __forceinline__ void w_ldv(waddr_t<GLOBAL> a, float (&x)[SPL]) {
  if constexpr (GLOBAL) {
    HnVec<SPL>::ld(a, x);
  } else if constexpr (SPL == 1) {
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x[0]) : "r"(a) : "memory");
  } else if constexpr (SPL == 2) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x[0]), "=f"(x[1]) : "r"(a) : "memory");
  } else {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
                 : "r"(a)
                 : "memory");
  }
}
template <int SPL, bool GLOBAL>
__device__ __forceinline__ void w_stv(waddr_t<GLOBAL> a, const float (&x)[SPL]) {
  if constexpr (GLOBAL) {
    HnVec<SPL>::st(const_cast<char *>(a), x);
  } else if constexpr (SPL == 1) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(x[0]) : "memory");
  } else if constexpr (SPL == 2) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x[0]), "f"(x[1]) : "memory");
  } else {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x[0]), "f"(x[1]),
                 "f"(x[2]), "f"(x[3])
                 : "memory");
  }
}

// whether a walk loads its records ahead of the evaluation (see cwalk)
template <int SPL, bool GLOBAL>
constexpr bool kCnPrefetch = SPL > 1 && GLOBAL;
// the first edge pair of a compiled node (zeros when it has none)
template <int SPL, bool GLOBAL>
__device__ __forceinline__ uint4 cnode_first_pair(const uint4 nraw, const waddr_t<GLOBAL> pairs) {
  const waddr_t<GLOBAL> pp = pairs + 16u * (nraw.z & ((1u << CN_PAIR_BITS) - 1u));
  return (nraw.z >> CN_PAIR_BITS) != 0u ? w_ld16<GLOBAL>(pp) : make_uint4(0u, 0u, 0u, 0u);
}
// One compiled node (its 16-byte record nraw) for this lane's SPL samples;
// e0 its first edge pair when the walk loads records ahead (kCnPrefetch),
// else unused (the pair is loaded here).
template <int SPL, bool GLOBAL, bool PF = kCnPrefetch<SPL, GLOBAL>>
__device__ __forceinline__ void cnode_eval(const uint4 nraw, const uint4 e0, const waddr_t<GLOBAL> pairs,
                                           const waddr_t<GLOBAL> vb) {
  constexpr int SH = 7 + (SPL == 4 ? 2 : (SPL == 2 ? 1 : 0));
  const float bias = __uint_as_float(nraw.x), resp = __uint_as_float(nraw.y);
  const uint32_t meta = nraw.w;
  const int np = int(nraw.z >> CN_PAIR_BITS);
  const waddr_t<GLOBAL> pp = pairs + 16u * (nraw.z & ((1u << CN_PAIR_BITS) - 1u));
  const int agg = int(meta >> (CN_ROW_BITS + 3)) & 3;
  // PF: e0 holds the first pair (when np > 0), loaded ahead by the walk
  float a[SPL];
  if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
    float a0[SPL], a1[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) a0[j] = a1[j] = 0.0f;
#pragma unroll 2
    for (int k = 0; k < np; ++k) {
      const uint4 e = PF && k == 0 ? e0 : w_ld16<GLOBAL>(pp + 16u * uint32_t(k));
      float x0[SPL], x1[SPL];
      w_ldv<SPL, GLOBAL>(vb + (e.x << SH), x0);
      w_ldv<SPL, GLOBAL>(vb + (e.z << SH), x1);
      hn_fma<SPL>(__uint_as_float(e.y), x0, a0);
      hn_fma<SPL>(__uint_as_float(e.w), x1, a1);
    }
#pragma unroll
    for (int j = 0; j < SPL; ++j) a[j] = a0[j] + a1[j];
    if (agg == NEAT_AGG_MEAN && np > 0) {
      const float cnt = float(2 * np - int((meta >> (CN_ROW_BITS + 5)) & 1u));
#pragma unroll
      for (int j = 0; j < SPL; ++j) a[j] = a[j] / cnt;
    }
  } else if (np == 0) {
#pragma unroll
    for (int j = 0; j < SPL; ++j) a[j] = 0.0f;
  } else if (agg == NEAT_AGG_MAX) {
    const uint4 e = PF ? e0 : w_ld16<GLOBAL>(pp);
    float x0[SPL], x1[SPL];
    w_ldv<SPL, GLOBAL>(vb + (e.x << SH), x0);
    w_ldv<SPL, GLOBAL>(vb + (e.z << SH), x1);
#pragma unroll
    for (int j = 0; j < SPL; ++j)
      a[j] = fmaxf(__uint_as_float(e.y) * x0[j], __uint_as_float(e.w) * x1[j]);
    for (int k = 1; k < np; ++k) {
      const uint4 f = w_ld16<GLOBAL>(pp + 16u * uint32_t(k));
      w_ldv<SPL, GLOBAL>(vb + (f.x << SH), x0);
      w_ldv<SPL, GLOBAL>(vb + (f.z << SH), x1);
#pragma unroll
      for (int j = 0; j < SPL; ++j) {
        a[j] = fmaxf(a[j], __uint_as_float(f.y) * x0[j]);
        a[j] = fmaxf(a[j], __uint_as_float(f.w) * x1[j]);
      }
    }
  } else {  // product
#pragma unroll
    for (int j = 0; j < SPL; ++j) a[j] = 1.0f;
    for (int k = 0; k < np; ++k) {
      const uint4 f = PF && k == 0 ? e0 : w_ld16<GLOBAL>(pp + 16u * uint32_t(k));
      float x0[SPL], x1[SPL];
      w_ldv<SPL, GLOBAL>(vb + (f.x << SH), x0);
      w_ldv<SPL, GLOBAL>(vb + (f.z << SH), x1);
#pragma unroll
      for (int j = 0; j < SPL; ++j) {
        a[j] = a[j] * (__uint_as_float(f.y) * x0[j]);
        a[j] = a[j] * (__uint_as_float(f.w) * x1[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < SPL; ++j) a[j] = fmaf(resp, a[j], bias);
  act_apply_n<SPL>(int(meta >> CN_ROW_BITS) & 7, a);
  w_stv<SPL, GLOBAL>(vb + ((meta & ((1u << CN_ROW_BITS) - 1u)) << SH), a);
}

template <int SPL, bool GLOBAL, bool PF = kCnPrefetch<SPL, GLOBAL>>
__device__ __forceinline__ void cnode_eval(const uint4 nraw, const waddr_t<GLOBAL> pairs,
                                           const waddr_t<GLOBAL> vb) {
  const uint4 e0 = PF ? cnode_first_pair<SPL, GLOBAL>(nraw, pairs) : make_uint4(0u, 0u, 0u, 0u);
  cnode_eval<SPL, GLOBAL, PF>(nraw, e0, pairs, vb);
}

// Walk of a compiled program (CNode records and edge pairs; see
// neat_internal.cuh) for this lane's SPL samples.  vb = the warp's value array
// + lane * SPL floats (bytes); value row r of it at vb + r * 128 * SPL
// ([row][32 lanes][SPL]: one vector access per row and lane).  GLOBAL: records
// and values in global memory, else both in shared memory.  Per node: a
// 16-byte record; per two edges: one 16-byte pair; per edge and sample: one
// value and one FMA.  Sum and mean keep even edges in a0 and odd edges in a1,
// the rounding order of the position walk.
//
// With two or four samples a lane and the records in global memory (the
// workspace-slot walk), the records run ahead of the evaluation:
// node c + 1's first pair and node c + 2's record are loaded before node c
// is evaluated (records only: values are read when their node runs), which
// takes two dependent L2 loads off every node's chain (16,384 uneven
// genomes, two samples a lane at 64 registers: 981 -> 916 us).  One sample a
// lane keeps the plain loop (the extra records spill under its 42-register
// bound), and so does a walk of records staged in shared memory (short
// latency).
template <int SPL, bool GLOBAL, bool PF = kCnPrefetch<SPL, GLOBAL>>
__device__ __forceinline__ void cwalk(const CNode *__restrict__ nodes, int nn,
                                      const uint4 *__restrict__ pairs, char *vb) {
  const waddr_t<GLOBAL> na = waddr<GLOBAL>(nodes), pa = waddr<GLOBAL>(pairs),
                        va = waddr<GLOBAL>(vb);
  if constexpr (!PF) {
    for (int c = 0; c < nn; ++c)
      cnode_eval<SPL, GLOBAL, false>(w_ld16<GLOBAL>(na + 16u * uint32_t(c)), pa, va);
  } else {
    if (nn <= 0) return;
    uint4 r0 = w_ld16<GLOBAL>(na);
    uint4 r1 = w_ld16<GLOBAL>(na + 16u * uint32_t(min(1, nn - 1)));
    uint4 p0 = cnode_first_pair<SPL, GLOBAL>(r0, pa);
    for (int c = 0; c < nn; ++c) {
      const uint4 p1 = cnode_first_pair<SPL, GLOBAL>(r1, pa);
      const uint4 r2 = w_ld16<GLOBAL>(na + 16u * uint32_t(min(c + 2, nn - 1)));
      cnode_eval<SPL, GLOBAL, true>(r0, p0, pa, va);
      r0 = r1;
      r1 = r2;
      p0 = p1;
    }
  }
}

// Item = (genome in queue order, tile of 32 * SPL samples); lane l evaluates
// samples tile * 32 * SPL + j * 32 + l, j < SPL.  A call without saved
// aggregates walks the genome's compiled program (value rows, only the nodes
// the outputs depend on), one that saves them the position program.  Values
// needing at most vcap rows live in this warp's shared-memory array, the
// others in the warp's slot of the workspace value array (N + 2 rows;
// L1/L2-resident while in use).
//
// With `coop`, the items of the queue's first counters[CTR_SP_NBIG] genomes
// (the most expensive ones, sp_cost >= sp_coop_cost) are taken by whole CTAs:
// the CTA's warps split each frontier's positions (no position of a frontier
// reads another's value) with a barrier between frontiers, in the slot of the
// CTA's first warp.  One warp walking such a genome alone would finish long
// after the rest of the grid.  The remaining items are claimed per warp.
//
// Registers: one sample a lane fits 42 (three 512-thread CTAs an SM); two or
// four a lane take up to 80 (six 4-warp CTAs), with the records loaded ahead
// (cwalk) without spilling.  On the uneven population (16,384 genomes, S =
// 64, 4-warp CTAs, us per launch): two a lane 1,050 at a 42-register bound,
// 982 at 64, 916 at 64 with the records ahead, 897 at 72, 886 at 80; one a
// lane at 64 registers loses more warps than it gains (1,065 -> 1,250).
template <int SPL, bool COMP>
__global__ void __launch_bounds__(512, SPL == 1 ? 3 : 1) __maxnreg__(SPL == 1 ? 255 : 80)
    k_forward_sp(Ws w, const float *__restrict__ inputs, int64_t stride, int S,
                             float *__restrict__ out, float *__restrict__ saved, int tiles,
                             int vcap, int coop) {
  constexpr int RS = 32 * SPL;
  extern __shared__ __align__(16) float smv[];
  __shared__ int s_item;
  __shared__ int s_lstart[NEAT_MAX_NODES + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int N = w.N, I = w.I, O = w.O;
  float *vs = smv + size_t(wid) * vcap * RS;
  const size_t slot = size_t(blockIdx.x) * nw + wid, SLOT = size_t(N + 2) * RS;
  float *vg = (w.sp_scratch != nullptr && (slot + 1) * SLOT <= w.sp_scratch_floats)
                  ? w.sp_scratch + slot * SLOT
                  : nullptr;
  const int total = w.P * tiles;
  const int big_items = coop ? min(total, int(w.counters[CTR_SP_NBIG]) * tiles) : 0;

  // ---- CTA-wide items (vg of warp 0 is the CTA's slot: the grid is sized
  // so that every warp of it has one)
  float *vc = (w.sp_scratch != nullptr &&
               (size_t(blockIdx.x) * nw + 1) * SLOT <= w.sp_scratch_floats)
                  ? w.sp_scratch + size_t(blockIdx.x) * nw * SLOT
                  : nullptr;
  while (big_items > 0) {
    if (threadIdx.x == 0) s_item = int(atomicAdd(w.counters + CTR_FWD_BIG, 1u));
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= big_items) break;
    const int q = item / tiles, tile = item - q * tiles;
    const int g = w.qorder[q];
    const GenomeHdr h = w.hdr[g];
    int sj[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) sj[j] = tile * RS + j * 32 + lane;
    if (vc == nullptr || h.L > NEAT_MAX_NODES) {  // no slot: never with a plan's shape
      if (threadIdx.x == 0) atomicOr(w.counters + CTR_ERR, ERR_SP_NO_SCRATCH);
      if (wid == 0)
#pragma unroll
        for (int j = 0; j < SPL; ++j)
          if (sj[j] < S)
            for (int o = 0; o < O; ++o) out[(size_t(g) * S + sj[j]) * O + o] = qnan();
      continue;
    }
    if constexpr (COMP) {  // every valid genome of such a plan has its compiled program
      {
        // compiled program: the CTA's warps split each layer's compiled nodes,
        // values [row][32][SPL] in the CTA's slot
        const CNode *cn = w.cnode + size_t(g) * N;
        const uint4 *cp = w.cpair + size_t(g) * cpair_cap(N, w.C);
        const int32_t *cl = w.clay + size_t(g) * (N + 1);
        for (int i = wid; i < I + 2; i += nw)
#pragma unroll
          for (int j = 0; j < SPL; ++j) {
            const bool active = sj[j] < S;
            const float *in = inputs + size_t(g) * stride + size_t(active ? sj[j] : 0) * I;
            vc[(i * 32 + lane) * SPL + j] =
                i < I ? (active ? __ldg(in + i) : 0.0f) : (i == I ? 0.0f : 1.0f);
          }
        __syncthreads();
        char *vb = reinterpret_cast<char *>(vc + lane * SPL);
        for (int k = 0; k < h.clayers; ++k) {
          // (each warp's next node record and first pair loaded ahead, as in
          // cwalk, with two or more samples a lane)
          const int c0 = cl[k] + wid, c1 = cl[k + 1];
          if constexpr (!kCnPrefetch<SPL, true>) {
            for (int c = c0; c < c1; c += nw)
              cnode_eval<SPL, true>(__ldg(reinterpret_cast<const uint4 *>(cn + c)),
                                    waddr<true>(cp), waddr<true>(vb));
          } else if (c0 < c1) {
            uint4 r0 = __ldg(reinterpret_cast<const uint4 *>(cn + c0));
            uint4 p0 = cnode_first_pair<SPL, true>(r0, waddr<true>(cp));
            for (int c = c0; c < c1; c += nw) {
              const uint4 r1 = __ldg(reinterpret_cast<const uint4 *>(cn + min(c + nw, c1 - 1)));
              const uint4 p1 = cnode_first_pair<SPL, true>(r1, waddr<true>(cp));
              cnode_eval<SPL, true>(r0, p0, waddr<true>(cp), waddr<true>(vb));
              r0 = r1;
              p0 = p1;
            }
          }
          __syncthreads();
        }
        const int32_t *orow = w.cout + size_t(g) * O;
        for (int o = wid; o < O; o += nw)
#pragma unroll
          for (int j = 0; j < SPL; ++j)
            if (sj[j] < S) out[(size_t(g) * S + sj[j]) * O + o] = vc[(orow[o] * 32 + lane) * SPL + j];
        __syncthreads();  // the slot is reused by the next item
        continue;
      }
    } else {
      const int32_t *lay = w.player + size_t(g) * N;
      for (int p = threadIdx.x; p < h.V; p += blockDim.x)
        if (p == 0 || lay[p - 1] != lay[p]) s_lstart[lay[p]] = p;
      if (threadIdx.x == 0) s_lstart[h.L] = h.V;
      float *vl = vc + lane;
      const int32_t *io = w.pio + size_t(g) * (I + O);
      for (int i = wid; i < I; i += nw)
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
          const bool active = sj[j] < S;
          const float *in = inputs + size_t(g) * stride + size_t(active ? sj[j] : 0) * I;
          vl[(io[i] * SPL + j) * 32] = active ? __ldg(in + i) : 0.0f;
        }
      __syncthreads();
      const NodeRec *nr = w.knode + h.node_off;
      const EdgeRec *er = w.kedge + h.edge_off;
      float *scol[SPL];
#pragma unroll
      for (int j = 0; j < SPL; ++j)
        scol[j] = (saved != nullptr && sj[j] < S) ? saved + size_t(g) * N * S + sj[j] : nullptr;
      for (int l = 0; l < h.L; ++l) {
        const int p1 = s_lstart[l + 1];
        for (int p = s_lstart[l] + wid; p < p1; p += nw) {
          if (!COMP && saved != nullptr)
            eval_node<true, SPL>(ld_node(nr + p), p, er, vl, scol, S);
          else
            eval_node<false, SPL>(ld_node(nr + p), p, er, vl, scol, S);
        }
        __syncthreads();
      }
      for (int o = wid; o < O; o += nw)
#pragma unroll
        for (int j = 0; j < SPL; ++j)
          if (sj[j] < S) out[(size_t(g) * S + sj[j]) * O + o] = vl[(io[I + o] * SPL + j) * 32];
    }
    __syncthreads();  // the slot and s_lstart are reused by the next item
  }

  // ---- per-warp items
  for (;;) {
    int item = 0;
    if (lane == 0) item = int(atomicAdd(w.counters + CTR_FWD_ITEM, 1u));
    item = __shfl_sync(0xffffffffu, item, 0) + big_items;
    if (item >= total) break;
    const int q = item / tiles, tile = item - q * tiles;
    const int g = w.qorder[q];
    const GenomeHdr h = w.hdr[g];
    // COMP: a call without saved aggregates on a plan with compiled programs
    // (every valid genome of such a plan has one)
    const int need = COMP ? h.crows : h.V;  // rows of the value array
    int sj[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) sj[j] = tile * RS + j * 32 + lane;
    if (h.status != 0u || (need > vcap && vg == nullptr)) {
      if (h.status == 0u && lane == 0) atomicOr(w.counters + CTR_ERR, ERR_SP_NO_SCRATCH);
#pragma unroll
      for (int j = 0; j < SPL; ++j)
        if (sj[j] < S)
          for (int o = 0; o < O; ++o) out[(size_t(g) * S + sj[j]) * O + o] = qnan();
      continue;
    }
    if constexpr (COMP) {
      // compiled program, values [row][32][SPL]: rows 0..I-1 the inputs, I and
      // I+1 the constants 0 and 1
      const CNode *cn = w.cnode + size_t(g) * N;
      const uint4 *cp = w.cpair + size_t(g) * cpair_cap(N, w.C);
      const int32_t *orow = w.cout + size_t(g) * O;
      auto run = [&](float *v) {
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
          const bool active = sj[j] < S;
          const float *in = inputs + size_t(g) * stride + size_t(active ? sj[j] : 0) * I;
          for (int i = 0; i < I; ++i) v[(i * 32 + lane) * SPL + j] = active ? __ldg(in + i) : 0.0f;
          v[(I * 32 + lane) * SPL + j] = 0.0f;
          v[((I + 1) * 32 + lane) * SPL + j] = 1.0f;
        }
        cwalk<SPL, true>(cn, h.nlive, cp, reinterpret_cast<char *>(v + lane * SPL));
#pragma unroll
        for (int j = 0; j < SPL; ++j)
          if (sj[j] < S)
            for (int o = 0; o < O; ++o)
              out[(size_t(g) * S + sj[j]) * O + o] = v[(orow[o] * 32 + lane) * SPL + j];
      };
      if (need <= vcap)
        run(vs);  // shared memory
      else
        run(vg);
    } else {
      float *v = need <= vcap ? vs : vg;
      float *vl = v + lane;
      const int32_t *io = w.pio + size_t(g) * (I + O);
#pragma unroll
      for (int j = 0; j < SPL; ++j) {
        const bool active = sj[j] < S;
        const float *in = inputs + size_t(g) * stride + size_t(active ? sj[j] : 0) * I;
        for (int i = 0; i < I; ++i) vl[(io[i] * SPL + j) * 32] = active ? __ldg(in + i) : 0.0f;
      }
      const NodeRec *nr = w.knode + h.node_off;
      const EdgeRec *er = w.kedge + h.edge_off;
      if (!COMP && saved != nullptr) {
        float *scol[SPL];
#pragma unroll
        for (int j = 0; j < SPL; ++j)
          scol[j] = sj[j] < S ? saved + size_t(g) * N * S + sj[j] : nullptr;
        walk_program<true, SPL>(nr, er, h.V, vl, scol, S);
      } else {
        float *const scol[SPL] = {};
        walk_program<false, SPL>(nr, er, h.V, vl, scol, S);
      }
#pragma unroll
      for (int j = 0; j < SPL; ++j)
        if (sj[j] < S)
          for (int o = 0; o < O; ++o)
            out[(size_t(g) * S + sj[j]) * O + o] = vl[(io[I + o] * SPL + j) * 32];
    }
  }
  grid_done_reset(w.counters + CTR_FWD_ITEM, w.counters + CTR_FWD_DONE, w.counters + CTR_FWD_BIG);
}

// Recurrent calculation (T synchronous iterations; inputs clamped, v^0 = 0
// elsewhere, outputs v^T).  Warps claim (genome, 32 * SPL-sample tile) items
// from the size-sorted queue; lane l evaluates samples tile * 32 * SPL +
// j * 32 + l, j < SPL (every record load serves SPL samples).  The warp's
// workspace slot holds two [N][SPL][32] value buffers, v^{t-1} (read) and
// v^t (written), swapped after every iteration.
// (launch bound: 64 registers, four 8-warp CTAs an SM)
template <int SPL>
__global__ void __launch_bounds__(256, 4)
    k_forward_rec(Ws w, const float *__restrict__ inputs, int64_t stride, int S, int T,
                  float *__restrict__ out, int tiles) {
  constexpr int RS = 32 * SPL;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int N = w.N, I = w.I, O = w.O;
  const size_t slot = size_t(blockIdx.x) * (blockDim.x >> 5) + wid;
  float *buf = (w.sp_scratch != nullptr && (slot + 1) * 2 * size_t(N) * RS <= w.sp_scratch_floats)
                   ? w.sp_scratch + slot * 2 * size_t(N) * RS
                   : nullptr;
  const int total = w.P * tiles;
  for (;;) {
    int item = 0;
    if (lane == 0) item = int(atomicAdd(w.counters + CTR_REC_ITEM, 1u));
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int q = item / tiles, tile = item - q * tiles;
    const int g = w.qorder[q];
    const GenomeHdr h = w.hdr[g];
    int sj[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) sj[j] = tile * RS + j * 32 + lane;
    if (h.status != 0u || buf == nullptr) {
      if (buf == nullptr && lane == 0) atomicOr(w.counters + CTR_ERR, ERR_SP_NO_SCRATCH);
#pragma unroll
      for (int j = 0; j < SPL; ++j)
        if (sj[j] < S)
          for (int o = 0; o < O; ++o) out[(size_t(g) * S + sj[j]) * O + o] = qnan();
      continue;
    }
    float *a = buf + lane, *b = buf + size_t(N) * RS + lane;  // value (p, j) at [(p * SPL + j) * 32]
    const int V = h.V;
    for (int p = 0; p < V; ++p)
#pragma unroll
      for (int j = 0; j < SPL; ++j) {
        a[(p * SPL + j) * 32] = 0.0f;
        b[(p * SPL + j) * 32] = 0.0f;
      }
    const int32_t *io = w.pio + size_t(g) * (I + O);
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
      const bool active = sj[j] < S;
      const float *in = inputs + size_t(g) * stride + size_t(active ? sj[j] : 0) * I;
      for (int i = 0; i < I; ++i) {
        const float x = active ? __ldg(in + i) : 0.0f;
        a[(io[i] * SPL + j) * 32] = x;
        b[(io[i] * SPL + j) * 32] = x;
      }
    }
    const NodeRec *nr = w.knode + h.node_off;
    const EdgeRec *er = w.kedge + h.edge_off;
    for (int t = 0; t < T; ++t) {
      // each node's record loaded one node ahead (10,000 cyclic genomes, S =
      // 64, T = 8: 2.36 -> 2.12 ms); V >= I + O >= 2 for a valid genome
      NodeRec n = ld_node(nr);
      for (int p = 0; p < V; ++p) {
        const NodeRec nx = ld_node(nr + min(p + 1, V - 1));
        if (!(n.meta & META_INPUT)) {
          float ag[SPL];
          node_agg<SPL>(n, er, a, ag);
#pragma unroll
          for (int j = 0; j < SPL; ++j) ag[j] = fmaf(n.resp, ag[j], n.bias);
          act_apply_n<SPL>(meta_act(n.meta), ag);
#pragma unroll
          for (int j = 0; j < SPL; ++j) b[(p * SPL + j) * 32] = ag[j];
        }
        n = nx;
      }
      float *tmp = a;
      a = b;
      b = tmp;
    }
#pragma unroll
    for (int j = 0; j < SPL; ++j)
      if (sj[j] < S)
        for (int o = 0; o < O; ++o) out[(size_t(g) * S + sj[j]) * O + o] = a[(io[I + o] * SPL + j) * 32];
  }
  grid_done_reset(w.counters + CTR_REC_ITEM, w.counters + CTR_REC_DONE);
}

__global__ void __launch_bounds__(32) k_forward_plain(Ws w, const float *__restrict__ inputs,
                                                      int64_t stride, int S,
                                                      float *__restrict__ out) {
  extern __shared__ __align__(16) float smv[];
  const int lane = threadIdx.x;
  const int N = w.N, C = w.C, I = w.I, O = w.O;
  const int g = blockIdx.x, s = blockIdx.y * 32 + lane;
  const bool active = s < S;
  const GenomeHdr h = w.hdr[g];
  float *orow = out + (size_t(g) * S + (active ? s : 0)) * O;
  if (h.status != 0u) {
    if (active)
      for (int j = 0; j < O; ++j) orow[j] = qnan();
    return;
  }
  const int32_t *io = w.pio + size_t(g) * (I + O);
  const float *in = inputs + size_t(g) * stride + size_t(active ? s : 0) * I;
  for (int i = 0; i < I; ++i) smv[io[i] * 32 + lane] = active ? __ldg(in + i) : 0.0f;
  const NodeRec *nr = w.pnode + size_t(g) * N;
  const EdgeRec *er = w.pedge + size_t(g) * C;
  for (int p = 0; p < N; ++p) {  // every padded position
    const NodeRec n = ld_node(nr + p);
    if (!(n.meta & META_VALID) || (n.meta & META_INPUT)) continue;
    float a[1];
    node_agg<1>(n, er, smv + lane, a);
    smv[p * 32 + lane] = act_apply(meta_act(n.meta), fmaf(n.resp, a[0], n.bias));
  }
  if (active)
    for (int j = 0; j < O; ++j) orow[j] = smv[io[I + j] * 32 + lane];
}

// Plain form with lanes over edges: warp (genome g = blockIdx.x, sample s =
// blockIdx.y) walks all N padded positions; the node records of 32 positions
// are loaded at once (lane j holds position p0 + j) and handed out by
// shuffles; lane l folds edges l, l + 32, ... of the node, the warp combines
// the 32 partial aggregates with a butterfly and lane 0 stores the value.
// Lanes without an edge hold the aggregation's neutral element (0 for sums,
// 1 for products, NaN for max: fmaxf ignores it, and a max over edges that
// are all NaN stays NaN, as the edge-order fold gives).
__device__ __forceinline__ float bfly_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ float bfly_prod(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x *= __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ float bfly_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__global__ void __launch_bounds__(32) k_forward_plain_edges(Ws w, const float *__restrict__ inputs,
                                                            int64_t stride, int S,
                                                            float *__restrict__ out) {
  extern __shared__ __align__(16) float smv[];  // [N] this sample's node values
  const int lane = threadIdx.x;
  const int N = w.N, C = w.C, I = w.I, O = w.O;
  const int g = blockIdx.x, s = blockIdx.y;
  const GenomeHdr h = w.hdr[g];
  float *orow = out + (size_t(g) * S + s) * O;
  if (h.status != 0u) {
    for (int j = lane; j < O; j += 32) orow[j] = qnan();
    return;
  }
  const int32_t *io = w.pio + size_t(g) * (I + O);
  const float *in = inputs + size_t(g) * stride + size_t(s) * I;
  for (int i = lane; i < I; i += 32) smv[io[i]] = __ldg(in + i);
  __syncwarp();
  const NodeRec *nr = w.pnode + size_t(g) * N;
  const EdgeRec *er = w.pedge + size_t(g) * C;
  for (int p0 = 0; p0 < N; p0 += 32) {
    NodeRec mine{};
    if (p0 + lane < N) mine = ld_node(nr + p0 + lane);
    const int nq = min(32, N - p0);
    for (int q = 0; q < nq; ++q) {
      const uint32_t meta = __shfl_sync(0xffffffffu, mine.meta, q);
      if (!(meta & META_VALID) || (meta & META_INPUT)) continue;  // warp-uniform
      const float bias = __shfl_sync(0xffffffffu, mine.bias, q);
      const float resp = __shfl_sync(0xffffffffu, mine.resp, q);
      const int beg = __shfl_sync(0xffffffffu, mine.in_begin, q);
      const int cnt = meta_cnt(meta), agg = meta_agg(meta);
      float a = 0.0f;
      if (cnt > 0) {
        if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
          float part = 0.0f;
          for (int k = lane; k < cnt; k += 32) {
            const EdgeRec e = ld_edge(er + beg + k);
            part = fmaf(e.w, smv[e.src], part);
          }
          a = bfly_sum(part);
          if (agg == NEAT_AGG_MEAN) a = a / float(cnt);
        } else if (agg == NEAT_AGG_PRODUCT) {
          float part = 1.0f;
          for (int k = lane; k < cnt; k += 32) {
            const EdgeRec e = ld_edge(er + beg + k);
            part *= e.w * smv[e.src];
          }
          a = bfly_prod(part);
        } else {
          float part = qnan();
          for (int k = lane; k < cnt; k += 32) {
            const EdgeRec e = ld_edge(er + beg + k);
            part = fmaxf(part, e.w * smv[e.src]);
          }
          a = bfly_max(part);
        }
      }
      const float v = act_apply(meta_act(meta), fmaf(resp, a, bias));
      if (lane == 0) smv[p0 + q] = v;
      __syncwarp();
    }
  }
  for (int j = lane; j < O; j += 32) orow[j] = smv[io[I + j]];
}

// ---- HyperNEAT substrate query ---------------------------------------------
// Query q = s * G^2 + t; cell c = j * G + i sits at (-1 + 2i/(G-1),
// -1 + 2j/(G-1)); the CPPN inputs are (x_s, y_s, x_t, y_t, 1).  G <= 128 keeps
// every query index in 32 bits.
//
// Item = (genome in queue order, chunk of tiles), claimed by a whole CTA; tile =
// 32 * SPL consecutive queries, lane l of its warp evaluating queries
// tile * 32 * SPL + k * 32 + l, k < SPL (every program record loaded serves
// SPL queries per lane).  The CTA copies the CPPN's compiled program (the
// transform's: 16-byte node records, 16-byte edge pairs, value rows) into
// shared memory, and as many of its warps as have room for a value array
// ([row][32][SPL] floats) walk tiles with the values in shared memory too: one
// broadcast pair load per two edges, one vector value load and one paired FMA
// per edge and query lane.  A CPPN whose value array does not fit falls back
// to the sample-parallel walk over the packed program with values in the
// warp's workspace slot.

// Query geometry and output of one item
struct HnTile {
  int G, G2, G4;
  float step, inv_g, thresh;
  int px, py, pX, pY, pb, po;  // positions of the five inputs and the output
  float *wg;                   // the genome's weights
};

// The tiles next() hands one warp (warp-uniform, -1 when done): coordinates
// into the input rows of the warp's value array v, walk(), thresholded
// outputs.  Value (row, query k of this lane) sits at
// v[(row * 32 + lane) * SPL + k] when LANE_MAJOR (the compiled walks: one
// vector access per row), else at v[(row * SPL + k) * 32 + lane] (the
// sample-parallel position walk).
template <int SPL, bool LANE_MAJOR, class Next, class Walk>
__device__ __forceinline__ void hn_tiles(const HnTile &t, float *v, Next next, Walk walk) {
  constexpr int RS = 32 * SPL;
  const int lane = threadIdx.x & 31;
  auto at = [&](int row, int k) -> float & {
    return LANE_MAJOR ? v[(row * 32 + lane) * SPL + k] : v[(row * SPL + k) * 32 + lane];
  };
#pragma unroll
  for (int k = 0; k < SPL; ++k) at(t.pb, k) = 1.0f;
  for (int tile = next(); tile >= 0; tile = next()) {
    const int q0 = tile * RS;
    const int sc0 = q0 / t.G2, tc0 = q0 - sc0 * t.G2 + lane;
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
      int sc = sc0, tc = tc0 + k * 32;
      if (tc >= t.G2) {
        const int d = tc / t.G2;
        sc += d;
        tc -= d * t.G2;
      }
      const int sj = int((float(sc) + 0.5f) * t.inv_g), si = sc - sj * t.G;
      const int tj = int((float(tc) + 0.5f) * t.inv_g), ti = tc - tj * t.G;
      at(t.px, k) = -1.0f + t.step * float(si);
      at(t.py, k) = -1.0f + t.step * float(sj);
      at(t.pX, k) = -1.0f + t.step * float(ti);
      at(t.pY, k) = -1.0f + t.step * float(tj);
    }
    walk();
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
      const int qi = q0 + k * 32 + lane;
      const float o = at(t.po, k);
      if (qi < t.G4) t.wg[qi] = fabsf(o) > t.thresh ? o : 0.0f;
    }
  }
}

// The tiles of one item for a warp whose value array is its workspace slot
// (tiles claimed from the CTA's counter *s_tile below t1; the compiled
// program read from global memory).  Out of line: its registers do not add
// to those of the staged walk it runs beside.
template <int SPL>
__device__ __noinline__ void hn_slot_tiles(const HnTile t, float *v, int *s_tile, int t1,
                                           const CNode *gcn, int nlive, const uint4 *cp, int I) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    v[(I * 32 + lane) * SPL + k] = 0.0f;
    v[((I + 1) * 32 + lane) * SPL + k] = 1.0f;
  }
  char *vb = reinterpret_cast<char *>(v + lane * SPL);
  auto claim = [&]() {
    int x = 0;
    if (lane == 0) x = atomicAdd(s_tile, 1);
    x = __shfl_sync(0xffffffffu, x, 0);
    return x < t1 ? x : -1;
  };
  // (the plain loop: the records loaded ahead would spill)
  hn_tiles<SPL, true>(t, v, claim, [&]() { cwalk<SPL, true, false>(gcn, nlive, cp, vb); });
}

template <int SPL>
__global__ void __launch_bounds__(512, 2) k_hyperneat(Ws w, int G, float thresh,
                                                   float *__restrict__ weights,
                                                   int chunks_per_genome, int tiles_per_chunk,
                                                   int smem_bytes) {
  constexpr int RS = 32 * SPL;
  extern __shared__ __align__(16) unsigned char hsm[];
  __shared__ int s_item, s_tile;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int N = w.N, I = w.I;
  const int prog_bytes = hn_prog_bytes(N, w.C);
  uint4 *s_nodes = reinterpret_cast<uint4 *>(hsm);  // CNode records
  uint4 *s_pairs = reinterpret_cast<uint4 *>(hsm + size_t(N) * sizeof(CNode));
  float *s_vals = reinterpret_cast<float *>(hsm + prog_bytes);
  // workspace slots of every warp of this CTA (N + 2 rows each), or none
  const size_t SLOT = size_t(N + 2) * RS;
  const bool slots_ok = w.sp_scratch != nullptr &&
                        size_t(blockIdx.x + 1) * nw * SLOT <= w.sp_scratch_floats;
  float *vg = slots_ok ? w.sp_scratch + (size_t(blockIdx.x) * nw + wid) * SLOT : nullptr;
  const int G2 = G * G, G4 = G2 * G2;
  const int tiles = (G4 + RS - 1) / RS;
  const int total = w.P * chunks_per_genome;
  const float step = 2.0f / float(G - 1);
  // cell c < 2^14: c / G = floor((c + 1/2) / G), whose fractional part stays
  // at least 1/(2G) away from an integer, far beyond the float rounding
  const float inv_g = 1.0f / float(G);
  for (;;) {
    if (threadIdx.x == 0) s_item = int(atomicAdd(w.counters + CTR_HN_ITEM, 1u));
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    const int q = item / chunks_per_genome, chunk = item - q * chunks_per_genome;
    const int g = w.qorder[q];
    const GenomeHdr h = w.hdr[g];
    float *wg = weights + size_t(g) * G4;
    const int t0 = chunk * tiles_per_chunk, t1 = min(t0 + tiles_per_chunk, tiles);
    const int32_t *io = w.pio + size_t(g) * 6;
    // warps with room for a value array of the compiled rows (CTA-uniform)
    const bool comp = w.cnode != nullptr && h.crows > 0;
    const int vwarps = comp ? min(nw, (smem_bytes - prog_bytes) / (h.crows * RS * 4)) : 0;
    if (h.status != 0u || (vwarps < 1 && !slots_ok)) {  // CTA-uniform
      if (h.status == 0u && lane == 0) atomicOr(w.counters + CTR_ERR, ERR_SP_NO_SCRATCH);
      for (int qi = t0 * RS + int(threadIdx.x); qi < min(t1 * RS, G4); qi += blockDim.x)
        wg[qi] = qnan();
      __syncthreads();  // s_item is rewritten by the next claim
      continue;
    }
    if (vwarps >= 1) {
      // the compiled program to shared memory
      const CNode *gcn = w.cnode + size_t(g) * N;
      const uint4 *cn = reinterpret_cast<const uint4 *>(gcn);
      const uint4 *cp = w.cpair + size_t(g) * cpair_cap(N, w.C);
      for (int i = threadIdx.x; i < h.nlive; i += blockDim.x) s_nodes[i] = __ldg(cn + i);
      for (int i = threadIdx.x; i < h.cpairs; i += blockDim.x) s_pairs[i] = __ldg(cp + i);
      if (threadIdx.x == 0) s_tile = t0;
      __syncthreads();
      // tiles claimed one at a time: the warps with a value array in shared
      // memory walk the staged program; the others (the CPPN's arrays fill the
      // shared memory before every warp has one) walk the same compiled
      // program from global memory with their arrays in their workspace slots
      // (the same arithmetic: the same bits), instead of waiting for the next
      // item
      auto claim = [&]() {
        int x = 0;
        if (lane == 0) x = atomicAdd(&s_tile, 1);
        x = __shfl_sync(0xffffffffu, x, 0);
        return x < t1 ? x : -1;
      };
      // inputs in rows 0..4, constants 0 and 1 in rows I and I + 1
      const HnTile t{G, G2, G4, step, inv_g, thresh, 0, 1, 2, 3, 4, w.cout[g], wg};
      if (wid < vwarps) {
        float *v = s_vals + size_t(wid) * h.crows * RS;  // shared memory
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
          v[(I * 32 + lane) * SPL + k] = 0.0f;
          v[((I + 1) * 32 + lane) * SPL + k] = 1.0f;
        }
        char *vb = reinterpret_cast<char *>(v + lane * SPL);
        const CNode *sn = reinterpret_cast<const CNode *>(s_nodes);
        hn_tiles<SPL, true>(t, v, claim, [&]() { cwalk<SPL, false>(sn, h.nlive, s_pairs, vb); });
      } else if (vg != nullptr) {
        hn_slot_tiles<SPL>(t, vg, &s_tile, t1, gcn, h.nlive, cp, I);
      }
    } else {
      const HnTile t{G, G2, G4, step, inv_g, thresh, io[0], io[1], io[2], io[3], io[4], io[5], wg};
      const NodeRec *nr = w.knode + h.node_off;
      const EdgeRec *er = w.kedge + h.edge_off;
      float *vl = vg + lane;
      int cur = t0 + wid - nw;
      auto next = [&]() {
        cur += nw;
        return cur < t1 ? cur : -1;
      };
      hn_tiles<SPL, false>(t, vg, next, [&]() {
        float *const scol[SPL] = {};
        walk_program<false, SPL>(nr, er, h.V, vl, scol, 0);
      });
    }
    __syncthreads();  // the staged program and s_item are reused by the next item
  }
  grid_done_reset(w.counters + CTR_HN_ITEM, w.counters + CTR_HN_DONE);
}

}  // namespace

size_t forward_sp_smem(int vcap, int warps, int spl) {
  return size_t(vcap) * 32 * spl * sizeof(float) * warps;
}

cudaError_t launch_forward_sp(const Ws &w, const float *inputs, int64_t stride, int S,
                              float *outputs, float *saved, const SpShape &sh, cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const size_t smem = forward_sp_smem(sh.vcap, sh.warps, sh.spl);
  const int tiles = (S + 32 * sh.spl - 1) / (32 * sh.spl);
  const dim3 grid(unsigned(sh.grid)), block(unsigned(sh.warps * 32));
  // outputs only on a plan with compiled programs: the compiled walk
  const bool comp = saved == nullptr && w.cnode != nullptr;
#define NEAT_SP(L, C)                                                                     \
  k_forward_sp<L, C><<<grid, block, smem, st>>>(w, inputs, stride, S, outputs, saved, tiles, \
                                                sh.vcap, sh.coop)
  switch (sh.spl * 2 + (comp ? 1 : 0)) {
    case 2: NEAT_SP(1, false); break;
    case 3: NEAT_SP(1, true); break;
    case 4: NEAT_SP(2, false); break;
    case 5: NEAT_SP(2, true); break;
    case 8: NEAT_SP(4, false); break;
    case 9: NEAT_SP(4, true); break;
    default: return cudaErrorInvalidValue;
  }
#undef NEAT_SP
  return cudaGetLastError();
}

cudaError_t launch_forward_plain(const Ws &w, const float *inputs, int64_t stride, int S,
                                 float *outputs, cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  if (S <= PLAIN_EDGE_S_MAX) {
    const dim3 grid(unsigned(w.P), unsigned(S));
    k_forward_plain_edges<<<grid, 32, size_t(w.N) * sizeof(float), st>>>(w, inputs, stride, S,
                                                                        outputs);
    return cudaGetLastError();
  }
  const size_t smem = size_t(w.N) * 32 * sizeof(float);
  const dim3 grid(unsigned(w.P), unsigned((S + 31) / 32));
  k_forward_plain<<<grid, 32, smem, st>>>(w, inputs, stride, S, outputs);
  return cudaGetLastError();
}

cudaError_t launch_forward_recurrent(const Ws &w, const float *inputs, int64_t stride, int S,
                                     int T, float *outputs, int spl, int warps, int grid,
                                     cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const int tiles = (S + 32 * spl - 1) / (32 * spl);
  if (spl == 2)
    k_forward_rec<2><<<grid, warps * 32, 0, st>>>(w, inputs, stride, S, T, outputs, tiles);
  else
    k_forward_rec<1><<<grid, warps * 32, 0, st>>>(w, inputs, stride, S, T, outputs, tiles);
  return cudaGetLastError();
}

int forward_rec_occupancy(int warps, int spl) {
  int n = 0;
  const cudaError_t e =
      spl == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_rec<2>, warps * 32, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_rec<1>, warps * 32, 0);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_hyperneat(const Ws &w, int G, float thresh, float *weights, int spl,
                             int warps, int ctas, int smem_bytes, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  const int64_t G4 = int64_t(G) * G * G * G;
  const int RS = 32 * spl;
  const int64_t tiles = (G4 + RS - 1) / RS;
  // items of 64 K, 32 K or 16 K queries, the largest that still gives every
  // CTA four items: a CTA's warps wait for the item's last tile and restage
  // the program between items, so larger items cost less (256 CPPNs on the
  // 32 x 32 grid, ms: 12.12 / 11.76 / 11.73 with 16 / 32 / 64 K), while
  // fewer items than CTAs would leave CTAs idle
  int q_item = 65536;
  while (q_item > 16384 && int64_t(w.P) * ((G4 + q_item - 1) / q_item) < 4LL * ctas) q_item >>= 1;
  const int tiles_per_chunk = std::max(1, q_item / RS);
  const int chunks = int((tiles + tiles_per_chunk - 1) / tiles_per_chunk);
  switch (spl) {
#define NEAT_HN(L)                                                                          \
  k_hyperneat<L><<<ctas, warps * 32, smem_bytes, st>>>(w, G, thresh, weights, chunks,       \
                                                       tiles_per_chunk, smem_bytes);         \
  break
    case 1: NEAT_HN(1);
    case 2: NEAT_HN(2);
    case 4: NEAT_HN(4);
#undef NEAT_HN
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace neat

namespace neat {
cudaError_t forward_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_forward_sp<1, false>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_sp<2, false>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_sp<4, false>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_sp<1, true>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_sp<2, true>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_sp<4, true>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_plain, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_hyperneat<1>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_hyperneat<2>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_hyperneat<4>, bytes);
  return e;
}
int forward_sp_occupancy(int warps, size_t smem, int spl) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (spl == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_sp<1, false>, warps * 32, smem);
  if (spl == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_sp<2, false>, warps * 32, smem);
  if (spl == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_sp<4, false>, warps * 32, smem);
  return e == cudaSuccess ? n : 0;
}
int hyperneat_occupancy(int spl, int warps, size_t smem) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  switch (spl) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hyperneat<1>, warps * 32, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hyperneat<2>, warps * 32, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hyperneat<4>, warps * 32, smem); break;
  }
  return e == cudaSuccess ? n : 0;
}
}  // namespace neat
