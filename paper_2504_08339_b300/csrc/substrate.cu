// HyperNEAT substrate evaluation: the two-sheet substrate of the query grid
// (an input sheet and an output sheet of K = G^2 cells; the query's weight
// w[s][t] connects input cell s to output cell t), y_t = act(sum_s w[s][t] x_s)
// for every input pattern x of every genome: Y[g] = act(X[g] W[g]).
//
// k_substrate: one CTA per 64 x 64 output tile of one genome; 32-deep slices
// of X (transposed) and W staged in shared memory; each thread accumulates a
// 4 x 4 block in registers over k in ascending order (a fixed summation
// order: results are deterministic), then applies the activation.
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

constexpr int BM = 64, BN = 64, BK = 32;

template <int ACT>
__global__ void __launch_bounds__(256) k_substrate(const float *__restrict__ w, int K,
                                                   const float *__restrict__ x,
                                                   int64_t stride, int S,
                                                   float *__restrict__ y) {
  __shared__ float xs[BK][BM + 4];  // X tile, transposed: xs[k][row]
  __shared__ float ws[BK][BN + 4];  // W tile: ws[k][col]
  const int g = blockIdx.z;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float *xg = x + size_t(g) * stride;
  const float *wg = w + size_t(g) * K * K;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += BK) {
    // X tile: 64 rows x 32 k; thread loads 8 (consecutive k across a warp)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * 256, r = e >> 5, kk = e & 31;
      const int gr = row0 + r, gk = k0 + kk;
      xs[kk][r] = (gr < S && gk < K) ? __ldg(xg + size_t(gr) * K + gk) : 0.0f;
    }
    // W tile: 32 k x 64 columns (consecutive columns across a warp)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * 256, kk = e >> 6, c = e & 63;
      const int gk = k0 + kk, gc = col0 + c;
      ws[kk][c] = (gk < K && gc < K) ? __ldg(wg + size_t(gk) * K + gc) : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = xs[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = ws[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty * 4 + i;
    if (r >= S) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx * 4 + j;
      if (c < K) y[(size_t(g) * S + r) * K + c] = act_apply(ACT, acc[i][j]);
    }
  }
}

}  // namespace

cudaError_t launch_substrate(const float *w, int P, int K, const float *x, int64_t stride, int S,
                             int act, float *y, cudaStream_t st) {
  if (P == 0 || S == 0) return cudaSuccess;
  const dim3 grid(unsigned((K + BN - 1) / BN), unsigned((S + BM - 1) / BM), unsigned(P));
  switch (act) {
#define NEAT_SUB(A) k_substrate<A><<<grid, 256, 0, st>>>(w, K, x, stride, S, y); break
    case NEAT_ACT_IDENTITY: NEAT_SUB(NEAT_ACT_IDENTITY);
    case NEAT_ACT_SIGMOID: NEAT_SUB(NEAT_ACT_SIGMOID);
    case NEAT_ACT_TANH: NEAT_SUB(NEAT_ACT_TANH);
    case NEAT_ACT_RELU: NEAT_SUB(NEAT_ACT_RELU);
    case NEAT_ACT_SIN: NEAT_SUB(NEAT_ACT_SIN);
    case NEAT_ACT_GAUSSIAN: NEAT_SUB(NEAT_ACT_GAUSSIAN);
    case NEAT_ACT_ABS: NEAT_SUB(NEAT_ACT_ABS);
#undef NEAT_SUB
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace neat

extern "C" neat_status neat_substrate_forward(const float *weights, int P, int K,
                                              const float *inputs, int64_t in_pop_stride, int S,
                                              int act, float *outputs, cudaStream_t stream) {
  if (P < 0 || K < 1 || S < 0 || act < 0 || act > NEAT_ACT_ABS || P > 65535)
    return NEAT_ERR_ARG;
  if (P == 0 || S == 0) return NEAT_OK;
  if (weights == nullptr || inputs == nullptr || outputs == nullptr ||
      (reinterpret_cast<uintptr_t>(weights) % 4) != 0 || (reinterpret_cast<uintptr_t>(inputs) % 4) != 0 ||
      (reinterpret_cast<uintptr_t>(outputs) % 4) != 0)
    return NEAT_ERR_ARG;
  if (in_pop_stride != 0 && in_pop_stride < int64_t(S) * K) return NEAT_ERR_ARG;
  if ((int64_t(S) + 63) / 64 > 65535) return NEAT_ERR_UNSUPPORTED;
  return neat::cuda_error_status(
      neat::launch_substrate(weights, P, K, inputs, in_pop_stride, S, act, outputs, stream));
}
