// Reverse mode of the calculation stage (the paper has no gradient; this is
// the adjoint of Sec. 3.3's forward rule v_k = act(b_k + r_k * a_k),
// a_k = agg_e(w_e * v_src(e))).  Given dL/dO it returns dL/dw (per connection
// row), dL/db and dL/dr (per node row) summed over samples, and dL/dx per
// sample.
//
// One CTA per genome (queue order, large genomes first).  Each warp handles
// 32-sample tiles (lane = sample): it reloads (or recomputes) the forward
// values, then walks the canonical order backwards.  A node's adjoint is
//   dL/dv_p = (pushed part) + sum over sum/mean consumers c of c_e w_e u_c,
// with u = dL/dz and c_e = r_c (sum) or r_c / n_c (mean).  The second term is
// PULLED by p from a per-genome list of its outgoing sum/mean edges (sorted
// by edge, so the rounding order is fixed), reading u_c where the consumer
// left it; product and max consumers, whose factor differs per sample, PUSH
// their terms into the adjoint slot of their sources (all in earlier
// frontiers, so never before those sources are visited) and sum dL/dw with
// warp butterflies.  Pulling keeps the walk free of read-modify-write chains.
//
// Nodes no output depends on (META_DEAD) have a zero adjoint: they are not
// visited, and their parameters' gradients stay 0.
//
// The cross-sample sums of a tile then run lane-parallel: lane per node for
// dL/db = sum_s u and dL/dr = sum_s u a, lane per sum/mean edge for
// dL/dw_e = c_e sum_s u_dst v_src, each into a lane-owned per-warp
// accumulator.  The per-warp accumulators are combined across warps in a
// fixed order: the result is deterministic (no floating-point atomics).
//
// Per-warp arrays are [V][33] floats: a lane's sample column (row p, column
// lane) and a lane's row (row p, columns s) both hit 32 distinct banks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

constexpr int RS = 33;  // row stride (floats) of the per-warp [V][RS] arrays

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// 4-byte asynchronous global -> shared copy (completes at cp_async_wait)
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// z[j] = act(z[j]) for four values of one activation: the four evaluations
// are independent and overlap.  Dispatch by a chain of two-way branches on
// the id (measured faster here than the multiway branch: 3.50 -> 3.32 ms per
// backward launch on 2,048 genomes at S = 4096).
template <int A>
__device__ __forceinline__ void act_same4(float (&z)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) z[j] = act_apply(A, z[j]);
}
__device__ __forceinline__ void act4(int act, float (&z)[4]) {
  if (is_id(act, NEAT_ACT_SIGMOID)) act_same4<NEAT_ACT_SIGMOID>(z);
  else if (is_id(act, NEAT_ACT_TANH)) act_same4<NEAT_ACT_TANH>(z);
  else if (is_id(act, NEAT_ACT_SIN)) act_same4<NEAT_ACT_SIN>(z);
  else if (is_id(act, NEAT_ACT_GAUSSIAN)) act_same4<NEAT_ACT_GAUSSIAN>(z);
  else if (is_id(act, NEAT_ACT_RELU)) act_same4<NEAT_ACT_RELU>(z);
  else if (is_id(act, NEAT_ACT_ABS)) act_same4<NEAT_ACT_ABS>(z);
}

// act_a(z) (the same values as act_apply), dispatched like act4
__device__ __forceinline__ float act_of(int a, float z) {
  if (is_id(a, NEAT_ACT_SIGMOID)) return act_apply(NEAT_ACT_SIGMOID, z);
  if (is_id(a, NEAT_ACT_TANH)) return act_apply(NEAT_ACT_TANH, z);
  if (is_id(a, NEAT_ACT_SIN)) return act_apply(NEAT_ACT_SIN, z);
  if (is_id(a, NEAT_ACT_GAUSSIAN)) return act_apply(NEAT_ACT_GAUSSIAN, z);
  if (is_id(a, NEAT_ACT_RELU)) return act_apply(NEAT_ACT_RELU, z);
  if (is_id(a, NEAT_ACT_ABS)) return act_apply(NEAT_ACT_ABS, z);
  return z;  // identity
}

// d act / dz (the same values as act_deriv), dispatched like act4
__device__ __forceinline__ float deriv_of(int a, float z, float v) {
  if (is_id(a, NEAT_ACT_SIGMOID)) return v * (1.0f - v);
  if (is_id(a, NEAT_ACT_TANH)) return 1.0f - v * v;
  if (is_id(a, NEAT_ACT_SIN)) return cosf(z);
  if (is_id(a, NEAT_ACT_GAUSSIAN)) return -2.0f * z * v;
  if (is_id(a, NEAT_ACT_RELU)) return z > 0.0f ? 1.0f : 0.0f;
  if (is_id(a, NEAT_ACT_ABS)) return z > 0.0f ? 1.0f : (z < 0.0f ? -1.0f : 0.0f);
  return 1.0f;  // identity
}

// Ascending bitonic sort of a[0..n2) by the whole CTA, n2 a power of two.
__device__ void bitonic_sort_u32(uint32_t *a, int n2) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t x = a[i], y = a[l];
          if (((i & k) == 0) == (x > y)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
}

__host__ __device__ inline int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Explicit shared-space loads with 32-bit addresses for the reverse walk's
// pulls and the cross-sample sums (the per-warp arrays are addressed through
// sizes read at run time); volatile with a memory clobber, so they keep
// their order with the walk's other accesses to the same arrays.
__device__ __forceinline__ unsigned sh_addr(const void *p) {
  return unsigned(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ float lds_f32(unsigned a) {
  float r;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(a) : "memory");
  return r;
}
__device__ __forceinline__ uint2 lds_u32x2(unsigned a) {
  uint2 r;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(a) : "memory");
  return r;
}

// Reads of a warp's [V][RS] arrays: explicit shared loads when the arrays sit
// in shared memory, plain loads when they sit in a workspace slot in global
// memory (the path of genomes too large for shared memory).
template <bool GM>
struct WArr {
  unsigned a;
  __device__ __forceinline__ explicit WArr(const float *p) : a(sh_addr(p)) {}
  __device__ __forceinline__ float operator[](unsigned i) const { return lds_f32(a + 4u * i); }
};
template <>
struct WArr<true> {
  const float *p;
  __device__ __forceinline__ explicit WArr(const float *q) : p(q) {}
  __device__ __forceinline__ float operator[](unsigned i) const { return p[i]; }
};

// One pulled edge: consumer position and c_e * w_e.
struct __align__(8) PullRec {
  int dst;
  float cw;
};

// Shared memory of a CTA: the genome's node and edge records; per edge c_e
// and its destination (-1: product/max); the pull lists (PullRec per
// sum/mean edge, grouped by source) with each position's range; the sort
// keys; then one block per working warp of
// bwd_warp_floats(V, E) floats: v, a, adjoint [V][RS] and the warp's
// accumulators for dL/dw [E], dL/db [V], dL/dr [V].  As many warps work as
// blocks of this genome's size fit; the others only join the barriers.
// (with_keys false: the sort keys live in the CTA's workspace slots instead)
__host__ __device__ inline size_t bwd_fixed_bytes(int N, int C, bool with_keys = true) {
  return sizeof(NodeRec) * size_t(N) + sizeof(EdgeRec) * size_t(C) +
         2 * sizeof(float) * size_t(C) + sizeof(PullRec) * size_t(C) +
         2 * sizeof(int) * size_t(N) +
         (with_keys ? sizeof(uint32_t) * size_t(pow2_at_least(C)) : 0);
}
__host__ __device__ inline size_t bwd_warp_floats(int V, int E) {
  return 3 * size_t(V) * RS + size_t(E) + 2 * size_t(V);
}

// GM = false: one CTA per genome (grid P), the warp arrays in shared memory
// after the records.  GM = true: a grid of fewer CTAs, each walking genomes
// blockIdx.x, blockIdx.x + gridDim.x, ... of the queue with its warps' arrays
// in its own workspace slots (blockDim / 32 blocks of bwd_warp_floats(N, C)
// floats at sp_scratch + blockIdx.x * that).
template <bool STORED, bool GM>
__global__ void k_backward(Ws w, const float *__restrict__ inputs, int64_t stride, int S,
                           const float *__restrict__ gout, const float *__restrict__ saved,
                           float *__restrict__ gw_out, float *__restrict__ gb_out,
                           float *__restrict__ gr_out, float *__restrict__ gi_out,
                           int smem_bytes) {
  extern __shared__ __align__(16) float sm[];
  const int N = w.N, C = w.C, I = w.I, O = w.O;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t cta_floats = size_t(blockDim.x >> 5) * bwd_warp_floats(N, C);
  if (GM && (w.sp_scratch == nullptr || (size_t(blockIdx.x) + 1) * cta_floats > w.sp_scratch_floats)) {
    // no slot for this CTA (the host sizes the grid so that this never
    // happens): report it; its genomes keep the gradients they had
    if (threadIdx.x == 0) atomicOr(w.counters + CTR_ERR, ERR_SP_NO_SCRATCH);
    return;
  }
  for (int qi = blockIdx.x; qi < w.P; qi += gridDim.x) {
  const int g = w.qorder[qi];
  const GenomeHdr h = w.hdr[g];
  for (int j = threadIdx.x; j < C; j += blockDim.x) gw_out[size_t(g) * C + j] = 0.0f;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    gb_out[size_t(g) * N + r] = 0.0f;
    gr_out[size_t(g) * N + r] = 0.0f;
  }
  const int tiles = (S + 31) / 32;
  if (h.status != 0u) {
    if (gi_out != nullptr)
      for (size_t i = threadIdx.x; i < size_t(S) * I; i += blockDim.x)
        gi_out[size_t(g) * S * I + i] = 0.0f;
    continue;  // (uniform over the CTA: nothing shared was touched)
  }
  const int V = h.V, E = h.E;
  NodeRec *nr = reinterpret_cast<NodeRec *>(sm);          // [N] node records
  EdgeRec *er = reinterpret_cast<EdgeRec *>(nr + N);      // [C] edge records
  float *ecoef = reinterpret_cast<float *>(er + C);       // [C] c_e of a sum/mean edge
  int *edst = reinterpret_cast<int *>(ecoef + C);         // [C] its destination (-1: product/max)
  PullRec *pull = reinterpret_cast<PullRec *>(edst + C);  // [C] pull lists
  int *pbeg = reinterpret_cast<int *>(pull + C);          // [N] pull list of position p:
  int *pend = pbeg + N;                                   // [N]   pull[pbeg[p] .. pend[p])
  // [pow2(C)] sort keys: in shared memory after the lists, or (GM) at the
  // start of the CTA's slots, which the warps' arrays only use after the sort
  float *wbase = GM ? w.sp_scratch + size_t(blockIdx.x) * cta_floats
                    : reinterpret_cast<float *>(reinterpret_cast<uint32_t *>(pend + N) +
                                                pow2_at_least(C));
  uint32_t *keys = GM ? reinterpret_cast<uint32_t *>(wbase) : reinterpret_cast<uint32_t *>(pend + N);
  const size_t pw = bwd_warp_floats(V, E);
  const int nwa = GM ? int(blockDim.x >> 5)
                     : min(int(blockDim.x >> 5),
                           int((size_t(smem_bytes) - bwd_fixed_bytes(N, C)) / (pw * sizeof(float))));
  float *v = wbase + size_t(wid) * pw + lane;  // values   [V][RS] (this lane's column)
  float *av = v + V * RS;                      // agg      [V][RS]
  float *dv = av + V * RS;                     // adjoints [V][RS]; u once a node is done
  float *accw = wbase + size_t(wid) * pw + 3 * V * RS;  // [E]
  float *accb = accw + E;                               // [V]
  float *accr = accb + V;                               // [V]

  // ---- per-genome setup: records, edge coefficients, pull lists
  const int32_t *io = w.pio + size_t(g) * (I + O);
  const int32_t *erow = w.kerow + h.edge_off;
  const int E2 = pow2_at_least(E);
  for (int p = threadIdx.x; p < V; p += blockDim.x) {
    nr[p] = w.knode[h.node_off + p];
    pbeg[p] = 0;
    pend[p] = 0;
  }
  for (int k = threadIdx.x; k < E; k += blockDim.x) er[k] = w.kedge[h.edge_off + k];
  if (!GM)
    for (size_t i = threadIdx.x; i < size_t(nwa) * pw; i += blockDim.x) wbase[i] = 0.0f;
  for (int p = threadIdx.x; p < V; p += blockDim.x) {
    const NodeRec n = w.knode[h.node_off + p];
    if (n.meta & META_INPUT) continue;
    const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
    // (a node no output depends on keeps its pull entries: it adds its zero
    // adjoint in the same place of each source's sum as without pruning)
    const bool lin = agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN;
    const float c = agg == NEAT_AGG_MEAN ? n.resp / float(cnt) : n.resp;
    for (int k = 0; k < cnt; ++k) {
      edst[n.in_begin + k] = lin ? p : -1;
      ecoef[n.in_begin + k] = c;
    }
  }
  __syncthreads();
  // keys (source << 16 | edge) of the sum/mean edges; the rest sort last
  for (int k = threadIdx.x; k < E2; k += blockDim.x)
    keys[k] = (k < E && edst[k] >= 0) ? (er[k].src << 16) | uint32_t(k) : 0xffffffffu;
  __syncthreads();
  bitonic_sort_u32(keys, E2);
  for (int i = threadIdx.x; i < E; i += blockDim.x) {
    const uint32_t key = keys[i];
    if (key == 0xffffffffu) continue;
    const int src = int(key >> 16), k = int(key & 0xffffu);
    pull[i].dst = edst[k];
    pull[i].cw = ecoef[k] * er[k].w;
    if (i == 0 || (keys[i - 1] >> 16) != uint32_t(src)) pbeg[src] = i;
    if (i + 1 == E || keys[i + 1] == 0xffffffffu || (keys[i + 1] >> 16) != uint32_t(src))
      pend[src] = i + 1;
  }
  __syncthreads();
  if (GM) {
    // the keys are done with; only the accumulators start at zero: every
    // value row a walk reads is written first in each tile (the rows of dead
    // positions are never read)
    const size_t acc = size_t(E) + 2 * size_t(V);
    for (size_t i = threadIdx.x; i < size_t(nwa) * acc; i += blockDim.x)
      wbase[(i / acc) * pw + 3 * size_t(V) * RS + i % acc] = 0.0f;
    __syncthreads();
  }

  for (int tile = wid; wid < nwa && tile < tiles; tile += nwa) {
    const int s = tile * 32 + lane;
    const bool active = s < S;
    // ---- forward values
    const float *in = inputs + size_t(g) * stride + size_t(active ? s : 0) * I;
    for (int i = 0; i < I; ++i) v[io[i] * RS] = active ? __ldg(in + i) : 0.0f;
    if (STORED) {
      // saved[g][p][s]: every position's line requested at once, straight
      // into shared memory
      const float *col = saved + size_t(g) * N * S + s;
      if (GM) {
        for (int p = 0; p < V; ++p)
          if (!(nr[p].meta & META_DEAD)) av[p * RS] = active ? __ldg(col + size_t(p) * S) : 0.0f;
      } else {
        if (active) {
          for (int p = 0; p < V; ++p)
            if (!(nr[p].meta & META_DEAD)) cp_async4(av + p * RS, col + size_t(p) * S);
        } else {
          for (int p = 0; p < V; ++p) av[p * RS] = 0.0f;
        }
        cp_async_wait();
      }
      // v = act(b + r a) of every node, four positions at a time
      for (int p = 0; p < V; p += 4) {
        NodeRec n[4];
        float z[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int pq = min(p + q, V - 1);
          n[q] = nr[pq];
          z[q] = fmaf(n[q].resp, av[pq * RS], n[q].bias);
        }
        const int act = meta_act(n[0].meta);
        if (act == meta_act(n[1].meta) && act == meta_act(n[2].meta) &&
            act == meta_act(n[3].meta)) {
          act4(act, z);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) z[q] = act_of(meta_act(n[q].meta), z[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (p + q < V && !(n[q].meta & (META_INPUT | META_DEAD))) v[(p + q) * RS] = z[q];
      }
    } else {
      for (int p = 0; p < V; ++p) {
        const NodeRec n = nr[p];
        if (n.meta & (META_INPUT | META_DEAD)) continue;
        const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
        const EdgeRec *e = er + n.in_begin;
        float a;
        if (cnt == 0) {
          a = 0.0f;
        } else if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
          float a0 = 0.0f, a1 = 0.0f;
          int k = 0;
          const unsigned ea = sh_addr(e);
          const WArr<GM> va(v);
          for (; k + 1 < cnt; k += 2) {
            const uint2 e0 = lds_u32x2(ea + 8u * unsigned(k)), e1 = lds_u32x2(ea + 8u * unsigned(k + 1));
            a0 = fmaf(__uint_as_float(e0.y), va[RS * e0.x], a0);
            a1 = fmaf(__uint_as_float(e1.y), va[RS * e1.x], a1);
          }
          if (k < cnt) a0 = fmaf(e[k].w, v[e[k].src * RS], a0);
          a = a0 + a1;
          if (agg == NEAT_AGG_MEAN) a = a / float(cnt);
        } else if (agg == NEAT_AGG_PRODUCT) {
          a = 1.0f;
          for (int k = 0; k < cnt; ++k) a *= e[k].w * v[e[k].src * RS];
        } else {
          a = e[0].w * v[e[0].src * RS];
          for (int k = 1; k < cnt; ++k) a = fmaxf(a, e[k].w * v[e[k].src * RS]);
        }
        av[p * RS] = a;
        v[p * RS] = act_of(meta_act(n.meta), fmaf(n.resp, a, n.bias));
      }
    }
    // ---- adjoints (inactive lanes carry zero adjoints throughout): the
    // pushed part starts as dL/dO
    for (int p = 0; p < V; ++p) dv[p * RS] = 0.0f;
    for (int o = 0; o < O; ++o)
      dv[io[I + o] * RS] += active ? __ldg(gout + (size_t(g) * S + s) * O + o) : 0.0f;
    for (int p = V - 1; p >= 0; --p) {
      const NodeRec n = nr[p];
      if (n.meta & META_DEAD) continue;  // zero adjoint, nothing to pass on
      // pulled part: sum over this position's sum/mean consumers
      const int b = pbeg[p], en = pend[p];
      float d0 = dv[p * RS], d1 = 0.0f;
      int i = b;
      const unsigned pla = sh_addr(pull);
      const WArr<GM> dva(dv);
      for (; i + 3 < en; i += 4) {
        const uint2 r0 = lds_u32x2(pla + 8u * unsigned(i)), r1 = lds_u32x2(pla + 8u * unsigned(i + 1)),
                    r2 = lds_u32x2(pla + 8u * unsigned(i + 2)), r3 = lds_u32x2(pla + 8u * unsigned(i + 3));
        const float u0 = dva[RS * r0.x], u1 = dva[RS * r1.x], u2 = dva[RS * r2.x],
                    u3 = dva[RS * r3.x];
        d0 = fmaf(__uint_as_float(r0.y), u0, d0);
        d1 = fmaf(__uint_as_float(r1.y), u1, d1);
        d0 = fmaf(__uint_as_float(r2.y), u2, d0);
        d1 = fmaf(__uint_as_float(r3.y), u3, d1);
      }
      for (; i < en; ++i) {
        const uint2 r0 = lds_u32x2(pla + 8u * unsigned(i));
        d0 = fmaf(__uint_as_float(r0.y), dva[RS * r0.x], d0);
      }
      const float d = d0 + d1;
      if (n.meta & META_INPUT) {
        dv[p * RS] = d;  // dL/dx
        continue;
      }
      const float a = av[p * RS];
      const float z = fmaf(n.resp, a, n.bias);
      const float u = d * deriv_of(meta_act(n.meta), z, v[p * RS]);
      dv[p * RS] = u;  // every consumer of p sits later and is done
      const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
      if (cnt == 0 || agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) continue;
      // product / max: push into the sources' adjoints (earlier frontiers)
      const float da = u * n.resp;
      const EdgeRec *e = er + n.in_begin;
      float *aw = accw + n.in_begin;
      if (agg == NEAT_AGG_PRODUCT) {
        // prod_{f != k} t_f from the product of the nonzero factors and the
        // number of zero factors
        float pnz = 1.0f;
        int nz = 0;
        for (int k = 0; k < cnt; ++k) {
          const float t = e[k].w * v[e[k].src * RS];
          if (t == 0.0f) ++nz; else pnz *= t;
        }
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = e[k];
          const float x = v[e0.src * RS];
          const float t = e0.w * x;
          float part;
          if (nz == 0) part = pnz / t;
          else if (nz == 1) part = (t == 0.0f) ? pnz : 0.0f;
          else part = 0.0f;
          const float dt = da * part;
          const float c = warp_sum(dt * x);
          if (lane == 0) aw[k] += c;
          dv[e0.src * RS] = fmaf(dt, e0.w, dv[e0.src * RS]);
        }
      } else {  // max: the first (lowest connection row) edge attaining the max
        int best = 0;
        float bt = 0.0f;
        int brow = 0x7fffffff;
        for (int k = 0; k < cnt; ++k) {
          const float t = e[k].w * v[e[k].src * RS];
          const int row = __ldg(erow + n.in_begin + k);
          const bool better = (k == 0) || (t > bt) || (bt != bt && t == t) ||
                              (t == bt && row < brow);
          if (better) {
            best = k;
            bt = t;
            brow = row;
          }
        }
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = e[k];
          const float x = v[e0.src * RS];
          const float dt = (k == best) ? da : 0.0f;
          const float c = warp_sum(dt * x);
          if (lane == 0) aw[k] += c;
          dv[e0.src * RS] = fmaf(dt, e0.w, dv[e0.src * RS]);
        }
      }
    }
    if (gi_out != nullptr && active)
      for (int i = 0; i < I; ++i) gi_out[(size_t(g) * S + s) * I + i] = dv[io[i] * RS];
    __syncwarp();
    // ---- cross-sample sums of this tile, lane-parallel over positions and
    // edges (inactive samples have u = 0 and add nothing)
    const float *vw = v - lane, *aww = av - lane, *dw = dv - lane;  // warp arrays
    for (int p = lane; p < V; p += 32) {
      if (nr[p].meta & (META_INPUT | META_DEAD)) continue;
      const WArr<GM> up(dw + p * RS), ap(aww + p * RS);
      float sb0 = 0.0f, sb1 = 0.0f, sr0 = 0.0f, sr1 = 0.0f;
#pragma unroll 8
      for (int q = 0; q < 32; q += 2) {
        const float u0 = up[q], u1 = up[q + 1];
        const float x0 = ap[q], x1 = ap[q + 1];
        sb0 += u0;
        sb1 += u1;
        sr0 = fmaf(u0, x0, sr0);
        sr1 = fmaf(u1, x1, sr1);
      }
      accb[p] += sb0 + sb1;
      accr[p] += sr0 + sr1;
    }
    for (int k = lane; k < E; k += 32) {
      const int dd = edst[k];
      // (an edge into a node no output depends on has a zero gradient: its
      // accumulator stays 0, and the values of dead sources are never read)
      if (dd < 0 || (nr[dd].meta & META_DEAD)) continue;
      const WArr<GM> up(dw + dd * RS), vp(vw + er[k].src * RS);
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll 8
      for (int q = 0; q < 32; q += 4) {
        s0 = fmaf(up[q], vp[q], s0);
        s1 = fmaf(up[q + 1], vp[q + 1], s1);
        s2 = fmaf(up[q + 2], vp[q + 2], s2);
        s3 = fmaf(up[q + 3], vp[q + 3], s3);
      }
      accw[k] = fmaf(ecoef[k], (s0 + s1) + (s2 + s3), accw[k]);
    }
    __syncwarp();
  }
  __syncthreads();
  // combine the per-warp partial sums in a fixed order and scatter to rows
  const size_t ow = 3 * size_t(V) * RS;  // accumulators inside a warp block
  for (int k = threadIdx.x; k < E; k += blockDim.x) {
    float sum = 0.0f;
    for (int ww = 0; ww < nwa; ++ww) sum += wbase[ww * pw + ow + k];
    gw_out[size_t(g) * C + erow[k]] = sum;
  }
  const int32_t *prow = w.prow + size_t(g) * N;
  for (int p = threadIdx.x; p < V; p += blockDim.x) {
    const int row = prow[p];
    if (row < I) continue;
    float sb = 0.0f, sr = 0.0f;
    for (int ww = 0; ww < nwa; ++ww) {
      sb += wbase[ww * pw + ow + E + p];
      sr += wbase[ww * pw + ow + E + V + p];
    }
    gb_out[size_t(g) * N + row] = sb;
    gr_out[size_t(g) * N + row] = sr;
  }
  __syncthreads();  // the next genome overwrites the records and the accumulators
  }
}

// out[j] = sum over genomes g in ascending order of x[g n + j], accumulated in
// double precision and rounded once: thread per element, eight genomes' loads
// in flight per step (coalesced across the warp: consecutive j).
__global__ void k_sum_genomes(const float *__restrict__ x, int P, int64_t n,
                              float *__restrict__ out) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
       j += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    int g = 0;
    for (; g + 8 <= P; g += 8) {
      float t[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) t[q] = __ldg(x + size_t(g + q) * size_t(n) + size_t(j));
#pragma unroll
      for (int q = 0; q < 8; ++q) acc += double(t[q]);
    }
    for (; g < P; ++g) acc += double(__ldg(x + size_t(g) * size_t(n) + size_t(j)));
    out[j] = float(acc);
  }
}

}  // namespace

cudaError_t launch_sum_genomes(const float *x, int P, int64_t n, float *out, int sm_count,
                               cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, int64_t(std::max(1, sm_count)) * 8);
  k_sum_genomes<<<unsigned(blocks), 256, 0, st>>>(x, P, n, out);
  return cudaGetLastError();
}

size_t backward_smem(int N, int C, int warps) {
  return bwd_fixed_bytes(N, C) + sizeof(float) * bwd_warp_floats(N, C) * size_t(warps);
}

size_t backward_fixed_smem(int N, int C) { return bwd_fixed_bytes(N, C, false); }

size_t backward_slot_floats(int N, int C) { return bwd_warp_floats(N, C); }

int backward_occupancy(bool global_values, int warps, int smem_bytes) {
  int occ = 0;
  const cudaError_t e =
      global_values ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_backward<true, true>,
                                                                    warps * 32, size_t(smem_bytes))
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_backward<true, false>,
                                                                    warps * 32, size_t(smem_bytes));
  return e == cudaSuccess ? occ : 0;
}

cudaError_t launch_backward(const Ws &w, const float *inputs, int64_t stride, int S,
                            const float *grad_out, const float *saved, float *gw, float *gb,
                            float *gr, float *gi, int warps, int smem_bytes, bool global_values,
                            int grid_ctas, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  const dim3 grid(unsigned(global_values ? grid_ctas : w.P)), block(unsigned(warps * 32));
#define NEAT_BWD(ST, GM)                                                                  \
  k_backward<ST, GM><<<grid, block, smem_bytes, st>>>(w, inputs, stride, S, grad_out, saved, gw, \
                                                      gb, gr, gi, smem_bytes)
  if (saved != nullptr) {
    if (global_values) NEAT_BWD(true, true);
    else NEAT_BWD(true, false);
  } else {
    if (global_values) NEAT_BWD(false, true);
    else NEAT_BWD(false, false);
  }
#undef NEAT_BWD
  return cudaGetLastError();
}

cudaError_t backward_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_backward<true, false>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_backward<false, false>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_backward<true, true>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_backward<false, true>, bytes);
  return e;
}

}  // namespace neat
