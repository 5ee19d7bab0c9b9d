// Reverse mode of the calculation stage (the paper has no gradient; this is
// the adjoint of Sec. 3.3's forward rule v_k = act(b_k + r_k * a_k),
// a_k = agg_e(w_e * v_src(e))).  Given dL/dO it returns dL/dw (per connection
// row), dL/db and dL/dr (per node row) summed over samples, and dL/dx per
// sample.
//
// One CTA per genome (queue order, large genomes first).  Each warp handles
// 32-sample tiles: it recomputes (or reloads) the forward values, then walks
// the canonical order backwards with per-lane adjoints in shared memory; the
// walk only propagates adjoints (each node's u = dL/dz overwrites its
// adjoint).  The cross-sample sums then run lane-parallel over the tile:
// lane per node for dL/db = sum_s u and dL/dr = sum_s u a, lane per edge for
// dL/dw_e = c_e sum_s u_dst v_src (sum: c = r, mean: c = r / n), each into a
// lane-owned per-warp accumulator; product and max edges, whose factor
// differs per sample, are summed with warp butterflies during the walk.  The
// per-warp accumulators are combined across warps in a fixed order: the
// result is deterministic (no floating-point atomics).
//
// Per-warp arrays are [N][33] floats: a lane's sample column (row p, column
// lane) and a lane's row (row p, columns s) both hit 32 distinct banks.
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

constexpr int RS = 33;  // row stride (floats) of the per-warp [N][RS] arrays

// z[j] = act(z[j]) for four nodes of one activation: the four evaluations
// are independent and overlap
template <int A>
__device__ __forceinline__ void act_same4(float (&z)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) z[j] = act_apply(A, z[j]);
}
__device__ __forceinline__ void act4(int act, float (&z)[4]) {
  switch (act) {
    case NEAT_ACT_IDENTITY: break;
    case NEAT_ACT_SIGMOID: act_same4<NEAT_ACT_SIGMOID>(z); break;
    case NEAT_ACT_TANH: act_same4<NEAT_ACT_TANH>(z); break;
    case NEAT_ACT_RELU: act_same4<NEAT_ACT_RELU>(z); break;
    case NEAT_ACT_SIN: act_same4<NEAT_ACT_SIN>(z); break;
    case NEAT_ACT_GAUSSIAN: act_same4<NEAT_ACT_GAUSSIAN>(z); break;
    default: act_same4<NEAT_ACT_ABS>(z); break;
  }
}

// Shared memory of a CTA: the genome's node and edge records, c_e and the
// destination of every edge, then one block per working warp of
// bwd_warp_floats(V, E) floats: v, a, adjoint [V][RS] and the warp's
// accumulators for dL/dw [E], dL/db [V], dL/dr [V].  As many warps work as
// blocks of this genome's size fit; the others only join the barriers.
__host__ __device__ inline size_t bwd_fixed_bytes(int N, int C) {
  return sizeof(NodeRec) * size_t(N) + sizeof(EdgeRec) * size_t(C) + 2 * sizeof(float) * size_t(C);
}
__host__ __device__ inline size_t bwd_warp_floats(int V, int E) {
  return 3 * size_t(V) * RS + size_t(E) + 2 * size_t(V);
}

template <bool STORED>
__global__ void k_backward(Ws w, const float *__restrict__ inputs, int64_t stride, int S,
                           const float *__restrict__ gout, const float *__restrict__ saved,
                           float *__restrict__ gw_out, float *__restrict__ gb_out,
                           float *__restrict__ gr_out, float *__restrict__ gi_out,
                           int smem_bytes) {
  extern __shared__ __align__(16) float sm[];
  const int N = w.N, C = w.C, I = w.I, O = w.O;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = w.qorder[blockIdx.x];
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
    return;
  }
  const int V = h.V, E = h.E;
  NodeRec *nr = reinterpret_cast<NodeRec *>(sm);      // [N] the genome's node records
  EdgeRec *er = reinterpret_cast<EdgeRec *>(nr + N);  // [C] and edge records
  float *ecoef = reinterpret_cast<float *>(er + C);   // [C] c_e of a sum/mean edge
  int *edst = reinterpret_cast<int *>(ecoef + C);     // [C] its destination (-1: product/max)
  float *wbase = reinterpret_cast<float *>(edst + C);
  const size_t pw = bwd_warp_floats(V, E);
  const int nwa = min(int(blockDim.x >> 5),
                      int((size_t(smem_bytes) - bwd_fixed_bytes(N, C)) / (pw * sizeof(float))));
  float *v = wbase + size_t(wid) * pw;  // values   [V][RS]
  float *av = v + V * RS;               // agg      [V][RS]
  float *dv = av + V * RS;              // adjoints [V][RS]; u once a node is done
  float *accw = dv + V * RS;            // [E]
  float *accb = accw + E;               // [V]
  float *accr = accb + V;               // [V]

  const int32_t *io = w.pio + size_t(g) * (I + O);
  const int32_t *erow = w.kerow + h.edge_off;
  for (int p = threadIdx.x; p < V; p += blockDim.x) nr[p] = w.knode[h.node_off + p];
  for (int k = threadIdx.x; k < E; k += blockDim.x) er[k] = w.kedge[h.edge_off + k];
  for (size_t i = threadIdx.x; i < size_t(nwa) * pw; i += blockDim.x) wbase[i] = 0.0f;
  for (int p = threadIdx.x; p < V; p += blockDim.x) {
    const NodeRec n = w.knode[h.node_off + p];
    if (n.meta & META_INPUT) continue;
    const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
    const bool lin = agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN;
    const float c = agg == NEAT_AGG_MEAN ? n.resp / float(cnt) : n.resp;
    for (int k = 0; k < cnt; ++k) {
      edst[n.in_begin + k] = lin ? p : -1;
      ecoef[n.in_begin + k] = c;
    }
  }
  __syncthreads();

  for (int tile = wid; wid < nwa && tile < tiles; tile += nwa) {
    const int s = tile * 32 + lane;
    const bool active = s < S;
    const size_t srow = size_t(g) * S + (active ? s : 0);
    // ---- forward values
    const float *in = inputs + size_t(g) * stride + size_t(active ? s : 0) * I;
    for (int i = 0; i < I; ++i) v[io[i] * RS + lane] = active ? __ldg(in + i) : 0.0f;
    if (STORED) {
      // saved[g][p][s]: one 128-byte line per position, all issued at once
      const float *col = saved + size_t(g) * N * S + (active ? s : 0);
#pragma unroll 4
      for (int p = 0; p < V; ++p) av[p * RS + lane] = active ? __ldg(col + size_t(p) * S) : 0.0f;
    }
    if (STORED) {
      // v = act(b + r a) of every node, four positions at a time
      for (int p = 0; p < V; p += 4) {
        NodeRec n[4];
        float z[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int q = min(p + j, V - 1);
          n[j] = nr[q];
          z[j] = fmaf(n[j].resp, av[q * RS + lane], n[j].bias);
        }
        const int act = meta_act(n[0].meta);
        if (act == meta_act(n[1].meta) && act == meta_act(n[2].meta) &&
            act == meta_act(n[3].meta)) {
          act4(act, z);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) z[j] = act_apply(meta_act(n[j].meta), z[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (p + j < V && !(n[j].meta & META_INPUT)) v[(p + j) * RS + lane] = z[j];
      }
    }
    for (int p = 0; !STORED && p < V; ++p) {
      const NodeRec n = nr[p];
      if (n.meta & META_INPUT) continue;
      float a;
      {
        const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
        const EdgeRec *e = er + n.in_begin;
        if (cnt == 0) {
          a = 0.0f;
        } else if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
          float a0 = 0.0f, a1 = 0.0f;
          int k = 0;
          for (; k + 1 < cnt; k += 2) {
            const EdgeRec e0 = e[k], e1 = e[k + 1];
            a0 = fmaf(e0.w, v[e0.src * RS + lane], a0);
            a1 = fmaf(e1.w, v[e1.src * RS + lane], a1);
          }
          if (k < cnt) {
            const EdgeRec e0 = e[k];
            a0 = fmaf(e0.w, v[e0.src * RS + lane], a0);
          }
          a = a0 + a1;
          if (agg == NEAT_AGG_MEAN) a = a / float(cnt);
        } else if (agg == NEAT_AGG_PRODUCT) {
          a = 1.0f;
          for (int k = 0; k < cnt; ++k) {
            const EdgeRec e0 = e[k];
            a *= e0.w * v[e0.src * RS + lane];
          }
        } else {
          EdgeRec e0 = e[0];
          a = e0.w * v[e0.src * RS + lane];
          for (int k = 1; k < cnt; ++k) {
            e0 = e[k];
            a = fmaxf(a, e0.w * v[e0.src * RS + lane]);
          }
        }
      }
      av[p * RS + lane] = a;
      v[p * RS + lane] = act_apply(meta_act(n.meta), fmaf(n.resp, a, n.bias));
    }
    // ---- adjoints (inactive lanes carry zero adjoints throughout)
    for (int p = 0; p < V; ++p) dv[p * RS + lane] = 0.0f;
    for (int j = 0; j < O; ++j)
      dv[io[I + j] * RS + lane] += active ? __ldg(gout + srow * O + j) : 0.0f;
    for (int p = V - 1; p >= 0; --p) {
      const NodeRec n = nr[p];
      if (n.meta & META_INPUT) continue;
      const float a = av[p * RS + lane];
      const float z = fmaf(n.resp, a, n.bias);
      const float u = dv[p * RS + lane] * act_deriv(meta_act(n.meta), z, v[p * RS + lane]);
      dv[p * RS + lane] = u;  // every consumer of p sits later and is done
      const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
      if (cnt == 0) continue;
      const float da = u * n.resp;
      const EdgeRec *e = er + n.in_begin;
      float *aw = accw + n.in_begin;
      if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
        const float dt = agg == NEAT_AGG_MEAN ? da / float(cnt) : da;
        // the sources of one node are distinct (duplicate edges are rejected),
        // so four read-modify-writes can be in flight at once
        int k = 0;
        for (; k + 3 < cnt; k += 4) {
          const EdgeRec e0 = e[k], e1 = e[k + 1], e2 = e[k + 2],
                        e3 = e[k + 3];
          const float d0 = dv[e0.src * RS + lane], d1 = dv[e1.src * RS + lane],
                      d2 = dv[e2.src * RS + lane], d3 = dv[e3.src * RS + lane];
          dv[e0.src * RS + lane] = fmaf(dt, e0.w, d0);
          dv[e1.src * RS + lane] = fmaf(dt, e1.w, d1);
          dv[e2.src * RS + lane] = fmaf(dt, e2.w, d2);
          dv[e3.src * RS + lane] = fmaf(dt, e3.w, d3);
        }
        for (; k < cnt; ++k) {
          const EdgeRec e0 = e[k];
          dv[e0.src * RS + lane] = fmaf(dt, e0.w, dv[e0.src * RS + lane]);
        }
      } else if (agg == NEAT_AGG_PRODUCT) {
        // prod_{f != k} t_f from the product of the nonzero factors and the
        // number of zero factors
        float pnz = 1.0f;
        int nz = 0;
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = e[k];
          const float t = e0.w * v[e0.src * RS + lane];
          if (t == 0.0f) ++nz; else pnz *= t;
        }
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = e[k];
          const float t = e0.w * v[e0.src * RS + lane];
          float part;
          if (nz == 0) part = pnz / t;
          else if (nz == 1) part = (t == 0.0f) ? pnz : 0.0f;
          else part = 0.0f;
          const float dt = da * part;
          const float c = warp_sum(dt * v[e0.src * RS + lane]);
          if (lane == 0) aw[k] += c;
          dv[e0.src * RS + lane] = fmaf(dt, e0.w, dv[e0.src * RS + lane]);
        }
      } else {  // max: the first (lowest connection row) edge attaining the max
        int best = 0;
        float bt = 0.0f;
        int brow = 0x7fffffff;
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = e[k];
          const float t = e0.w * v[e0.src * RS + lane];
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
          const float dt = (k == best) ? da : 0.0f;
          const float c = warp_sum(dt * v[e0.src * RS + lane]);
          if (lane == 0) aw[k] += c;
          dv[e0.src * RS + lane] = fmaf(dt, e0.w, dv[e0.src * RS + lane]);
        }
      }
    }
    if (gi_out != nullptr && active)
      for (int i = 0; i < I; ++i) gi_out[srow * I + i] = dv[io[i] * RS + lane];
    __syncwarp();
    // ---- cross-sample sums of this tile, lane-parallel (inactive samples
    // have u = 0 and add nothing)
    for (int p = lane; p < V; p += 32) {
      if (nr[p].meta & META_INPUT) continue;
      const float *up = dv + p * RS, *ap = av + p * RS;
      float sb0 = 0.0f, sb1 = 0.0f, sr0 = 0.0f, sr1 = 0.0f;
#pragma unroll 8
      for (int q = 0; q < 32; q += 2) {
        sb0 += up[q];
        sb1 += up[q + 1];
        sr0 = fmaf(up[q], ap[q], sr0);
        sr1 = fmaf(up[q + 1], ap[q + 1], sr1);
      }
      accb[p] += sb0 + sb1;
      accr[p] += sr0 + sr1;
    }
    for (int k = lane; k < E; k += 32) {
      const int d = edst[k];
      if (d < 0) continue;
      const float *up = dv + d * RS, *vp = v + er[k].src * RS;
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
    float s = 0.0f;
    for (int ww = 0; ww < nwa; ++ww) s += wbase[ww * pw + ow + k];
    gw_out[size_t(g) * C + erow[k]] = s;
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
}

}  // namespace

size_t backward_smem(int N, int C, int warps) {
  return bwd_fixed_bytes(N, C) + sizeof(float) * bwd_warp_floats(N, C) * size_t(warps);
}

cudaError_t launch_backward(const Ws &w, const float *inputs, int64_t stride, int S,
                            const float *grad_out, const float *saved, float *gw, float *gb,
                            float *gr, float *gi, int warps, int smem_bytes, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  if (saved != nullptr)
    k_backward<true><<<w.P, warps * 32, smem_bytes, st>>>(w, inputs, stride, S, grad_out, saved,
                                                          gw, gb, gr, gi, smem_bytes);
  else
    k_backward<false><<<w.P, warps * 32, smem_bytes, st>>>(w, inputs, stride, S, grad_out,
                                                           nullptr, gw, gb, gr, gi, smem_bytes);
  return cudaGetLastError();
}

cudaError_t backward_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_backward<true>, bytes);
  if (e != cudaSuccess) return e;
  return set_dyn_smem_limit(k_backward<false>, bytes);
}

}  // namespace neat
