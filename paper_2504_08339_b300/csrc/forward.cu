// Calculation stage (TensorNEAT Sec. 3.3): v[inputs] = I, then in canonical
// order v[k] = act(b + r * agg_e(w_e * v[src_e])); O = v[outputs].
//
// Sample-parallel forms: a warp owns one genome and 32 samples; lane l walks
// the genome's program for sample l with node values in shared memory laid
// out [position][lane] (conflict-free), program records read with warp-uniform
// (broadcast) loads.  No lane ever reads another lane's values, so the walk
// needs no synchronisation at all.
//
//  k_forward_sp     persistent grid, warps claim (genome, 32-sample tile)
//                   items from a device work queue in size-sorted order over
//                   the ragged-packed programs (the batched form).
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

// Aggregated input a = agg_e(w_e * v[src_e]) of one node for this lane's
// sample; v is the warp's [position][32] value array.
__device__ __forceinline__ float node_agg(const NodeRec &n, const EdgeRec *__restrict__ er,
                                          const float *v, int lane) {
  const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
  const EdgeRec *e = er + n.in_begin;
  if (cnt == 0) return 0.0f;
  if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
    float a0 = 0.0f, a1 = 0.0f;
    int k = 0;
    for (; k + 1 < cnt; k += 2) {
      const EdgeRec e0 = ld_edge(e + k), e1 = ld_edge(e + k + 1);
      a0 = fmaf(e0.w, v[e0.src * 32 + lane], a0);
      a1 = fmaf(e1.w, v[e1.src * 32 + lane], a1);
    }
    if (k < cnt) {
      const EdgeRec e0 = ld_edge(e + k);
      a0 = fmaf(e0.w, v[e0.src * 32 + lane], a0);
    }
    const float a = a0 + a1;
    return agg == NEAT_AGG_MEAN ? a / float(cnt) : a;
  }
  if (agg == NEAT_AGG_PRODUCT) {
    float a = 1.0f;
    for (int k = 0; k < cnt; ++k) {
      const EdgeRec e0 = ld_edge(e + k);
      a *= e0.w * v[e0.src * 32 + lane];
    }
    return a;
  }
  // max: fmax fold
  EdgeRec e0 = ld_edge(e);
  float a = e0.w * v[e0.src * 32 + lane];
  for (int k = 1; k < cnt; ++k) {
    e0 = ld_edge(e + k);
    a = fmaxf(a, e0.w * v[e0.src * 32 + lane]);
  }
  return a;
}

// Walk positions [0, V) of a ragged program (inputs already in v).
template <bool SAVE>
__device__ __forceinline__ void walk_program(const NodeRec *__restrict__ nr,
                                             const EdgeRec *__restrict__ er, int V, float *v,
                                             int lane, float *saved_row) {
  for (int p = 0; p < V; ++p) {
    const NodeRec n = ld_node(nr + p);
    if (n.meta & META_INPUT) continue;
    const float a = node_agg(n, er, v, lane);
    v[p * 32 + lane] = act_apply(meta_act(n.meta), fmaf(n.resp, a, n.bias));
    if (SAVE) saved_row[p] = a;
  }
}

__device__ __forceinline__ void grid_done_reset(uint32_t *item_ctr, uint32_t *done_ctr) {
  // the last CTA to finish returns the queue counters to zero, so every launch
  // (including graph replays) starts from a clean queue
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(done_ctr, 1u);
    if (t == gridDim.x - 1) {
      atomicExch(item_ctr, 0u);
      atomicExch(done_ctr, 0u);
    }
  }
}

__global__ void k_forward_sp(Ws w, const float *__restrict__ inputs, int64_t stride, int S,
                             float *__restrict__ out, float *__restrict__ saved, int tiles) {
  extern __shared__ __align__(16) float smv[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int N = w.N, I = w.I, O = w.O;
  float *v = smv + size_t(wid) * N * 32;
  const int total = w.P * tiles;
  for (;;) {
    int item = 0;
    if (lane == 0) item = int(atomicAdd(w.counters + CTR_FWD_ITEM, 1u));
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= total) break;
    const int q = item / tiles, tile = item - q * tiles;
    const int g = w.qorder[q];
    const GenomeHdr h = w.hdr[g];
    const int s = tile * 32 + lane;
    const bool active = s < S;
    float *orow = out + (size_t(g) * S + (active ? s : 0)) * O;
    if (h.status != 0u) {
      if (active)
        for (int j = 0; j < O; ++j) orow[j] = qnan();
      continue;
    }
    const int32_t *io = w.pio + size_t(g) * (I + O);
    const float *in = inputs + size_t(g) * stride + size_t(active ? s : 0) * I;
    for (int i = 0; i < I; ++i) v[io[i] * 32 + lane] = active ? __ldg(in + i) : 0.0f;
    const NodeRec *nr = w.knode + h.node_off;
    const EdgeRec *er = w.kedge + h.edge_off;
    if (saved != nullptr && active)
      walk_program<true>(nr, er, h.V, v, lane, saved + (size_t(g) * S + s) * N);
    else
      walk_program<false>(nr, er, h.V, v, lane, nullptr);
    if (active)
      for (int j = 0; j < O; ++j) orow[j] = v[io[I + j] * 32 + lane];
  }
  grid_done_reset(w.counters + CTR_FWD_ITEM, w.counters + CTR_FWD_DONE);
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
    const float a = node_agg(n, er, smv, lane);
    smv[p * 32 + lane] = act_apply(meta_act(n.meta), fmaf(n.resp, a, n.bias));
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
      walk_program<false>(nr, er, h.V, v, lane, nullptr);
      const float o = v[io[5] * 32 + lane];
      if (active) wg[qi] = fabsf(o) > thresh ? o : 0.0f;
    }
  }
  grid_done_reset(w.counters + CTR_HN_ITEM, w.counters + CTR_HN_DONE);
}

}  // namespace

size_t forward_sp_smem(int N, int warps) { return size_t(N) * 32 * sizeof(float) * warps; }

cudaError_t launch_forward_sp(const Ws &w, const float *inputs, int64_t stride, int S,
                              float *outputs, float *saved, int warps, int grid,
                              cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const size_t smem = forward_sp_smem(w.N, warps);
  const int tiles = (S + 31) / 32;
  k_forward_sp<<<grid, warps * 32, smem, st>>>(w, inputs, stride, S, outputs, saved, tiles);
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

cudaError_t launch_hyperneat(const Ws &w, int G, float thresh, float *weights, int warps,
                             int ctas, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  const size_t smem = forward_sp_smem(w.N, warps);
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
  cudaError_t e = set_dyn_smem_limit(k_forward_sp, bytes);
  if (e != cudaSuccess) return e;
  e = set_dyn_smem_limit(k_forward_plain, bytes);
  if (e != cudaSuccess) return e;
  return set_dyn_smem_limit(k_hyperneat, bytes);
}
int forward_sp_occupancy(int warps, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_sp, warps * 32, smem) !=
      cudaSuccess)
    return 0;
  return n;
}
int hyperneat_occupancy(int warps, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hyperneat, warps * 32, smem) !=
      cudaSuccess)
    return 0;
  return n;
}
}  // namespace neat
