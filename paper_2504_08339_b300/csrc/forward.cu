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
//  k_hyperneat      the batched form with inputs generated in the kernel
//                   (substrate coordinates) and a threshold epilogue.
#include <cuda_runtime.h>

#include <cstdint>

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
// samples; inputs are left alone.
template <bool SAVE, int SPL>
__device__ __forceinline__ void eval_node(const NodeRec &n, int p, const EdgeRec *__restrict__ er,
                                          float *vl, float *const (&scol)[SPL], int S) {
  if (n.meta & META_INPUT) return;
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

// Item = (genome in queue order, tile of 32 * SPL samples); lane l evaluates
// samples tile * 32 * SPL + j * 32 + l, j < SPL.  The values of a genome with
// V <= vcap live in this warp's shared-memory array, the others in the warp's
// slot of the workspace value array (L1/L2-resident while in use).
//
// With `coop`, the items of the queue's first counters[CTR_SP_NBIG] genomes
// (the most expensive ones, E + 2V >= SP_COOP_COST) are taken by whole CTAs:
// the CTA's warps split each frontier's positions (no position of a frontier
// reads another's value) with a barrier between frontiers, in the slot of the
// CTA's first warp.  One warp walking such a genome alone would finish long
// after the rest of the grid.  The remaining items are claimed per warp.
template <int SPL>
__global__ void __launch_bounds__(512, 3)
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
  const size_t slot = size_t(blockIdx.x) * nw + wid;
  float *vg = (w.sp_scratch != nullptr && (slot + 1) * size_t(N) * RS <= w.sp_scratch_floats)
                  ? w.sp_scratch + slot * size_t(N) * RS
                  : nullptr;
  const int total = w.P * tiles;
  const int big_items = coop ? min(total, int(w.counters[CTR_SP_NBIG]) * tiles) : 0;

  // ---- CTA-wide items (vg of warp 0 is the CTA's slot: the grid is sized
  // so that every warp of it has one)
  float *vc = (w.sp_scratch != nullptr &&
               (size_t(blockIdx.x) * nw + 1) * size_t(N) * RS <= w.sp_scratch_floats)
                  ? w.sp_scratch + size_t(blockIdx.x) * nw * size_t(N) * RS
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
        if (saved != nullptr)
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
    float *v = h.V <= vcap ? vs : vg;
    int sj[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) sj[j] = tile * RS + j * 32 + lane;
    if (h.status != 0u || v == nullptr) {
      if (v == nullptr && lane == 0) atomicOr(w.counters + CTR_ERR, ERR_SP_NO_SCRATCH);
#pragma unroll
      for (int j = 0; j < SPL; ++j)
        if (sj[j] < S)
          for (int o = 0; o < O; ++o) out[(size_t(g) * S + sj[j]) * O + o] = qnan();
      continue;
    }
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
    if (saved != nullptr) {
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
  grid_done_reset(w.counters + CTR_FWD_ITEM, w.counters + CTR_FWD_DONE, w.counters + CTR_FWD_BIG);
}

// Recurrent calculation (T synchronous iterations; inputs clamped, v^0 = 0
// elsewhere, outputs v^T).  Warps claim (genome, 32-sample tile) items from
// the size-sorted queue; the warp's workspace slot holds two [N][32] value
// buffers, v^{t-1} (read) and v^t (written), swapped after every iteration.
__global__ void __launch_bounds__(512, 3)
    k_forward_rec(Ws w, const float *__restrict__ inputs, int64_t stride, int S, int T,
                  float *__restrict__ out, int tiles) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int N = w.N, I = w.I, O = w.O;
  const size_t slot = size_t(blockIdx.x) * (blockDim.x >> 5) + wid;
  float *buf = (w.sp_scratch != nullptr && (slot + 1) * 2 * size_t(N) * 32 <= w.sp_scratch_floats)
                   ? w.sp_scratch + slot * 2 * size_t(N) * 32
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
    const int s = tile * 32 + lane;
    const bool active = s < S;
    float *orow = out + (size_t(g) * S + (active ? s : 0)) * O;
    if (h.status != 0u || buf == nullptr) {
      if (buf == nullptr && lane == 0) atomicOr(w.counters + CTR_ERR, ERR_SP_NO_SCRATCH);
      if (active)
        for (int o = 0; o < O; ++o) orow[o] = qnan();
      continue;
    }
    float *a = buf + lane, *b = buf + size_t(N) * 32 + lane;
    const int V = h.V;
    for (int p = 0; p < V; ++p) {
      a[p * 32] = 0.0f;
      b[p * 32] = 0.0f;
    }
    const int32_t *io = w.pio + size_t(g) * (I + O);
    const float *in = inputs + size_t(g) * stride + size_t(active ? s : 0) * I;
    for (int i = 0; i < I; ++i) {
      const float x = active ? __ldg(in + i) : 0.0f;
      a[io[i] * 32] = x;
      b[io[i] * 32] = x;
    }
    const NodeRec *nr = w.knode + h.node_off;
    const EdgeRec *er = w.kedge + h.edge_off;
    for (int t = 0; t < T; ++t) {
      for (int p = 0; p < V; ++p) {
        const NodeRec n = ld_node(nr + p);
        if (n.meta & META_INPUT) continue;
        float ag[1];
        node_agg<1>(n, er, a, ag);
        b[p * 32] = act_apply(meta_act(n.meta), fmaf(n.resp, ag[0], n.bias));
      }
      float *tmp = a;
      a = b;
      b = tmp;
    }
    if (active)
      for (int o = 0; o < O; ++o) orow[o] = a[io[I + o] * 32];
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

// HyperNEAT substrate query: item = (genome in queue order, chunk of 32-query
// tiles).  Query q = s * G^2 + t; cell c = j * G + i sits at
// (-1 + 2i/(G-1), -1 + 2j/(G-1)); inputs (x_s, y_s, x_t, y_t, 1).
__global__ void k_hyperneat(Ws w, int G, float thresh, float *__restrict__ weights,
                            int chunks_per_genome, int tiles_per_chunk) {
  extern __shared__ __align__(16) float smv[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int N = w.N;
  float *v = smv + size_t(wid) * N * 32;
  const int64_t G2 = int64_t(G) * G, G4 = G2 * G2;
  const int total = w.P * chunks_per_genome;
  const float step = 2.0f / float(G - 1);
  for (;;) {
    int item = 0;
    if (lane == 0) item = int(atomicAdd(w.counters + CTR_HN_ITEM, 1u));
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int q = item / chunks_per_genome, chunk = item - q * chunks_per_genome;
    const int g = w.qorder[q];
    const GenomeHdr h = w.hdr[g];
    float *wg = weights + size_t(g) * G4;
    const int32_t *io = w.pio + size_t(g) * 6;
    const NodeRec *nr = w.knode + h.node_off;
    const EdgeRec *er = w.kedge + h.edge_off;
    const int64_t t0 = int64_t(chunk) * tiles_per_chunk;
    for (int64_t tile = t0; tile < t0 + tiles_per_chunk; ++tile) {
      const int64_t qi = tile * 32 + lane;
      if (tile * 32 >= G4) break;
      const bool active = qi < G4;
      if (h.status != 0u) {
        if (active) wg[qi] = qnan();
        continue;
      }
      const int64_t sc = active ? qi / G2 : 0, tc = active ? qi - sc * G2 : 0;
      const int si = int(sc % G), sj = int(sc / G), ti = int(tc % G), tj = int(tc / G);
      v[io[0] * 32 + lane] = -1.0f + step * float(si);
      v[io[1] * 32 + lane] = -1.0f + step * float(sj);
      v[io[2] * 32 + lane] = -1.0f + step * float(ti);
      v[io[3] * 32 + lane] = -1.0f + step * float(tj);
      v[io[4] * 32 + lane] = 1.0f;
      float *const scol[1] = {nullptr};
      walk_program<false, 1>(nr, er, h.V, v + lane, scol, 0);
      const float o = v[io[5] * 32 + lane];
      if (active) wg[qi] = fabsf(o) > thresh ? o : 0.0f;
    }
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
  switch (sh.spl) {
    case 1: k_forward_sp<1><<<grid, block, smem, st>>>(w, inputs, stride, S, outputs, saved, tiles,
                                                       sh.vcap, sh.coop); break;
    case 2: k_forward_sp<2><<<grid, block, smem, st>>>(w, inputs, stride, S, outputs, saved, tiles,
                                                       sh.vcap, sh.coop); break;
    case 4: k_forward_sp<4><<<grid, block, smem, st>>>(w, inputs, stride, S, outputs, saved, tiles,
                                                       sh.vcap, sh.coop); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_forward_plain(const Ws &w, const float *inputs, int64_t stride, int S,
                                 float *outputs, cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const size_t smem = size_t(w.N) * 32 * sizeof(float);
  const dim3 grid(unsigned(w.P), unsigned((S + 31) / 32));
  k_forward_plain<<<grid, 32, smem, st>>>(w, inputs, stride, S, outputs);
  return cudaGetLastError();
}

cudaError_t launch_forward_recurrent(const Ws &w, const float *inputs, int64_t stride, int S,
                                     int T, float *outputs, int warps, int grid, cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const int tiles = (S + 31) / 32;
  k_forward_rec<<<grid, warps * 32, 0, st>>>(w, inputs, stride, S, T, outputs, tiles);
  return cudaGetLastError();
}

int forward_rec_occupancy(int warps) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_rec, warps * 32, 0) !=
      cudaSuccess)
    return 0;
  return n;
}

cudaError_t launch_hyperneat(const Ws &w, int G, float thresh, float *weights, int warps,
                             int ctas, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  const size_t smem = forward_sp_smem(w.N, warps, 1);
  const int64_t G4 = int64_t(G) * G * G * G;
  const int64_t tiles = (G4 + 31) / 32;
  const int tiles_per_chunk = 16;
  const int chunks = int((tiles + tiles_per_chunk - 1) / tiles_per_chunk);
  k_hyperneat<<<ctas, warps * 32, smem, st>>>(w, G, thresh, weights, chunks, tiles_per_chunk);
  return cudaGetLastError();
}

}  // namespace neat

namespace neat {
cudaError_t forward_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_forward_sp<1>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_sp<2>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_sp<4>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_plain, bytes);
  if (e != cudaSuccess) return e;
  return set_dyn_smem_limit(k_hyperneat, bytes);
}
int forward_sp_occupancy(int warps, size_t smem, int spl) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (spl == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_sp<1>, warps * 32, smem);
  if (spl == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_sp<2>, warps * 32, smem);
  if (spl == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_sp<4>, warps * 32, smem);
  return e == cudaSuccess ? n : 0;
}
int hyperneat_occupancy(int warps, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hyperneat, warps * 32, smem) !=
      cudaSuccess)
    return 0;
  return n;
}
}  // namespace neat
