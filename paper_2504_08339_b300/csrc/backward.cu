// Reverse mode of the calculation stage (the paper has no gradient; this is
// the adjoint of Sec. 3.3's forward rule v_k = act(b_k + r_k * a_k),
// a_k = agg_e(w_e * v_src(e))).  Given dL/dO it returns dL/dw (per connection
// row), dL/db and dL/dr (per node row) summed over samples, and dL/dx per
// sample.
//
// One CTA per genome (queue order, large genomes first).  Each warp handles
// 32-sample tiles: it recomputes (or reloads) the forward values, then walks
// the canonical order backwards with per-lane adjoints delta[position][lane]
// in shared memory.  Cross-sample sums are warp butterflies into per-warp
// accumulators, combined across warps in a fixed order: the result is
// deterministic (no floating-point atomics).
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

__device__ __forceinline__ EdgeRec ld_edge(const EdgeRec *p) {
  const uint2 x = __ldg(reinterpret_cast<const uint2 *>(p));
  EdgeRec e;
  e.src = x.x;
  e.w = __uint_as_float(x.y);
  return e;
}

template <bool STORED>
__global__ void k_backward(Ws w, const float *__restrict__ inputs, int64_t stride, int S,
                           const float *__restrict__ gout, const float *__restrict__ saved,
                           float *__restrict__ gw_out, float *__restrict__ gb_out,
                           float *__restrict__ gr_out, float *__restrict__ gi_out) {
  extern __shared__ __align__(16) float sm[];
  const int N = w.N, C = w.C, I = w.I, O = w.O;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = w.qorder[blockIdx.x];
  const GenomeHdr h = w.hdr[g];
  float *v = sm + size_t(wid) * 3 * N * 32;  // values   [N][32]
  float *av = v + N * 32;                    // agg      [N][32]
  float *dv = av + N * 32;                   // adjoints [N][32]
  float *accw = sm + size_t(nw) * 3 * N * 32;  // [nw][C]
  float *accb = accw + nw * C;                 // [nw][N]
  float *accr = accb + nw * N;                 // [nw][N]

  for (int i = threadIdx.x; i < nw * (C + 2 * N); i += blockDim.x) accw[i] = 0.0f;
  for (int j = threadIdx.x; j < C; j += blockDim.x) gw_out[size_t(g) * C + j] = 0.0f;
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    gb_out[size_t(g) * N + r] = 0.0f;
    gr_out[size_t(g) * N + r] = 0.0f;
  }
  __syncthreads();
  const int tiles = (S + 31) / 32;
  if (h.status != 0u) {
    if (gi_out != nullptr)
      for (size_t i = threadIdx.x; i < size_t(S) * I; i += blockDim.x)
        gi_out[size_t(g) * S * I + i] = 0.0f;
    return;
  }
  const int V = h.V;
  const int32_t *io = w.pio + size_t(g) * (I + O);
  const NodeRec *nr = w.knode + h.node_off;
  const EdgeRec *er = w.kedge + h.edge_off;
  const int32_t *erow = w.kerow + h.edge_off;

  for (int tile = wid; tile < tiles; tile += nw) {
    const int s = tile * 32 + lane;
    const bool active = s < S;
    const size_t srow = size_t(g) * S + (active ? s : 0);
    // ---- forward values
    const float *in = inputs + size_t(g) * stride + size_t(active ? s : 0) * I;
    for (int i = 0; i < I; ++i) v[io[i] * 32 + lane] = active ? __ldg(in + i) : 0.0f;
    for (int p = 0; p < V; ++p) {
      const NodeRec n = nr[p];
      if (n.meta & META_INPUT) {
        av[p * 32 + lane] = 0.0f;
        continue;
      }
      float a;
      if (STORED) {
        a = active ? __ldg(saved + srow * N + p) : 0.0f;
      } else {
        const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
        const EdgeRec *e = er + n.in_begin;
        if (cnt == 0) {
          a = 0.0f;
        } else if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
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
          a = a0 + a1;
          if (agg == NEAT_AGG_MEAN) a = a / float(cnt);
        } else if (agg == NEAT_AGG_PRODUCT) {
          a = 1.0f;
          for (int k = 0; k < cnt; ++k) {
            const EdgeRec e0 = ld_edge(e + k);
            a *= e0.w * v[e0.src * 32 + lane];
          }
        } else {
          EdgeRec e0 = ld_edge(e);
          a = e0.w * v[e0.src * 32 + lane];
          for (int k = 1; k < cnt; ++k) {
            e0 = ld_edge(e + k);
            a = fmaxf(a, e0.w * v[e0.src * 32 + lane]);
          }
        }
      }
      av[p * 32 + lane] = a;
      v[p * 32 + lane] = act_apply(meta_act(n.meta), fmaf(n.resp, a, n.bias));
    }
    // ---- adjoints
    for (int p = 0; p < V; ++p) dv[p * 32 + lane] = 0.0f;
    for (int j = 0; j < O; ++j)
      dv[io[I + j] * 32 + lane] += active ? __ldg(gout + srow * O + j) : 0.0f;
    for (int p = V - 1; p >= 0; --p) {
      const NodeRec n = nr[p];
      if (n.meta & META_INPUT) continue;
      const float a = av[p * 32 + lane];
      const float z = fmaf(n.resp, a, n.bias);
      const float u = dv[p * 32 + lane] * act_deriv(meta_act(n.meta), z, v[p * 32 + lane]);
      const float sb = warp_sum(u), sr = warp_sum(u * a);
      if (lane == 0) {
        accb[wid * N + p] += sb;
        accr[wid * N + p] += sr;
      }
      const int cnt = meta_cnt(n.meta), agg = meta_agg(n.meta);
      if (cnt == 0) continue;
      const float da = u * n.resp;
      const EdgeRec *e = er + n.in_begin;
      float *aw = accw + wid * C + n.in_begin;
      if (agg == NEAT_AGG_SUM || agg == NEAT_AGG_MEAN) {
        const float dt = agg == NEAT_AGG_MEAN ? da / float(cnt) : da;
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = ld_edge(e + k);
          const float c = warp_sum(dt * v[e0.src * 32 + lane]);
          if (lane == 0) aw[k] += c;
          dv[e0.src * 32 + lane] = fmaf(dt, e0.w, dv[e0.src * 32 + lane]);
        }
      } else if (agg == NEAT_AGG_PRODUCT) {
        // prod_{f != k} t_f from the product of the nonzero factors and the
        // number of zero factors
        float pnz = 1.0f;
        int nz = 0;
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = ld_edge(e + k);
          const float t = e0.w * v[e0.src * 32 + lane];
          if (t == 0.0f) ++nz; else pnz *= t;
        }
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = ld_edge(e + k);
          const float t = e0.w * v[e0.src * 32 + lane];
          float part;
          if (nz == 0) part = pnz / t;
          else if (nz == 1) part = (t == 0.0f) ? pnz : 0.0f;
          else part = 0.0f;
          const float dt = da * part;
          const float c = warp_sum(dt * v[e0.src * 32 + lane]);
          if (lane == 0) aw[k] += c;
          dv[e0.src * 32 + lane] = fmaf(dt, e0.w, dv[e0.src * 32 + lane]);
        }
      } else {  // max: the first (lowest connection row) edge attaining the max
        int best = 0;
        float bt = 0.0f;
        int brow = 0x7fffffff;
        for (int k = 0; k < cnt; ++k) {
          const EdgeRec e0 = ld_edge(e + k);
          const float t = e0.w * v[e0.src * 32 + lane];
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
          const EdgeRec e0 = ld_edge(e + k);
          const float dt = (k == best) ? da : 0.0f;
          const float c = warp_sum(dt * v[e0.src * 32 + lane]);
          if (lane == 0) aw[k] += c;
          dv[e0.src * 32 + lane] = fmaf(dt, e0.w, dv[e0.src * 32 + lane]);
        }
      }
    }
    if (gi_out != nullptr && active)
      for (int i = 0; i < I; ++i) gi_out[srow * I + i] = dv[io[i] * 32 + lane];
  }
  __syncthreads();
  // combine the per-warp partial sums in a fixed order and scatter to rows
  for (int k = threadIdx.x; k < h.E; k += blockDim.x) {
    float s = 0.0f;
    for (int ww = 0; ww < nw; ++ww) s += accw[ww * C + k];
    gw_out[size_t(g) * C + erow[k]] = s;
  }
  const int32_t *prow = w.prow + size_t(g) * N;
  for (int p = threadIdx.x; p < V; p += blockDim.x) {
    const int row = prow[p];
    if (row < I) continue;
    float sb = 0.0f, sr = 0.0f;
    for (int ww = 0; ww < nw; ++ww) {
      sb += accb[ww * N + p];
      sr += accr[ww * N + p];
    }
    gb_out[size_t(g) * N + row] = sb;
    gr_out[size_t(g) * N + row] = sr;
  }
}

}  // namespace

size_t backward_smem(int N, int C, int warps) {
  return sizeof(float) * (size_t(warps) * 3 * N * 32 + size_t(warps) * (C + 2 * N));
}

cudaError_t launch_backward(const Ws &w, const float *inputs, int64_t stride, int S,
                            const float *grad_out, const float *saved, float *gw, float *gb,
                            float *gr, float *gi, int warps, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  const size_t smem = backward_smem(w.N, w.C, warps);
  if (saved != nullptr)
    k_backward<true><<<w.P, warps * 32, smem, st>>>(w, inputs, stride, S, grad_out, saved, gw,
                                                    gb, gr, gi);
  else
    k_backward<false><<<w.P, warps * 32, smem, st>>>(w, inputs, stride, S, grad_out, nullptr, gw,
                                                     gb, gr, gi);
  return cudaGetLastError();
}

cudaError_t backward_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_backward<true>, bytes);
  if (e != cudaSuccess) return e;
  return set_dyn_smem_limit(k_backward<false>, bytes);
}

}  // namespace neat
