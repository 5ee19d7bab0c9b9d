// Tensorized operations of TensorNEAT Sec. 3.2 on the padded population
// tensors, in place: node / connection addition writes the new row at the
// first NaN row (a node row is free when its key is NaN, a connection row
// when either key is), removal writes NaN over a row, attribute modification
// assigns one non-key column.  Each genome has a list of K operations of 8
// floats (kind, row, v0..v5), applied in order:
//   1 add node (v0..v4)   2 remove node row   3 add connection (v0..v3)
//   4 remove connection row   5 node[row][v0] = v1 (column 1..4)
//   6 conn[row][v0] = v1 (column 2..3)   anything else: nothing
// An operation without a free row or with a row / column out of range changes
// nothing and sets bit k (k < 32) of the genome's op status.
//
// One warp per genome: the first free row is found 32 rows at a time with a
// ballot; the lanes write the row's columns; __syncwarp orders each
// operation's writes before the next one's reads.
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

__device__ __forceinline__ bool row_in(float r, int rows) {
  return r >= 0.0f && r < float(rows) && r == floorf(r);
}

// first free row of a [rows][cols] table (key columns: 0, and 1 for
// connections), or -1
__device__ __forceinline__ int first_free(const float *t, int rows, int cols, bool conn,
                                          int lane) {
  for (int base = 0; base < rows; base += 32) {
    const int r = base + lane;
    bool pad = false;
    if (r < rows) {
      const float *row = t + size_t(r) * cols;
      pad = isnan(row[0]) || (conn && isnan(row[1]));
    }
    const unsigned m = __ballot_sync(0xffffffffu, pad);
    if (m) return base + __ffs(m) - 1;
  }
  return -1;
}

__global__ void __launch_bounds__(256) k_apply_ops(float *__restrict__ nodes,
                                                   float *__restrict__ conns, int P, int N, int C,
                                                   const float *__restrict__ ops, int K,
                                                   uint32_t *__restrict__ op_status) {
  const int lane = threadIdx.x & 31;
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g >= P) return;
  float *gn = nodes + size_t(g) * N * 5;
  float *gc = conns + size_t(g) * C * 4;
  uint32_t st = 0;
  for (int k = 0; k < K; ++k) {
    const float *op = ops + (size_t(g) * K + k) * 8;
    const float kind = __ldg(op), rowf = __ldg(op + 1);
    bool ok = true;
    if (kind == 1.0f || kind == 3.0f) {
      const bool conn = kind == 3.0f;
      const int cols = conn ? 4 : 5;
      float *t = conn ? gc : gn;
      const int r = first_free(t, conn ? C : N, cols, conn, lane);
      if (r < 0) ok = false;
      else if (lane < cols) t[size_t(r) * cols + lane] = __ldg(op + 2 + lane);
    } else if (kind == 2.0f || kind == 4.0f) {
      const bool conn = kind == 4.0f;
      const int cols = conn ? 4 : 5;
      if (!row_in(rowf, conn ? C : N)) ok = false;
      else if (lane < cols)
        (conn ? gc : gn)[size_t(rowf) * cols + lane] = __int_as_float(0x7fc00000);
    } else if (kind == 5.0f || kind == 6.0f) {
      const bool conn = kind == 6.0f;
      const int cols = conn ? 4 : 5, lo = conn ? 2 : 1;
      const float col = __ldg(op + 2);
      if (!row_in(rowf, conn ? C : N) || !(col >= float(lo) && col <= float(cols - 1) &&
                                           col == floorf(col)))
        ok = false;
      else if (lane == 0) (conn ? gc : gn)[size_t(rowf) * cols + size_t(col)] = __ldg(op + 3);
    }
    if (!ok && k < 32) st |= 1u << k;
    __syncwarp();  // this operation's writes before the next one's reads
  }
  if (lane == 0 && op_status != nullptr) op_status[g] = st;
}

}  // namespace

cudaError_t launch_apply_ops(float *nodes, float *conns, int P, int N, int C, const float *ops,
                             int K, uint32_t *op_status, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  k_apply_ops<<<(P + 7) / 8, 256, 0, st>>>(nodes, conns, P, N, C, ops, K, op_status);
  return cudaGetLastError();
}

}  // namespace neat

extern "C" neat_status neat_apply_ops(float *nodes, float *conns, int P, int N, int C,
                                      const float *ops, int K, uint32_t *op_status,
                                      cudaStream_t stream) {
  if (P < 0 || N < 1 || N > NEAT_MAX_NODES || C < 1 || C > NEAT_MAX_CONNS || K < 0)
    return NEAT_ERR_UNSUPPORTED;
  if (P == 0) return NEAT_OK;
  if (nodes == nullptr || conns == nullptr || (K > 0 && ops == nullptr) ||
      (reinterpret_cast<uintptr_t>(nodes) % 4) != 0 || (reinterpret_cast<uintptr_t>(conns) % 4) != 0 ||
      (reinterpret_cast<uintptr_t>(ops) % 4) != 0 ||
      (op_status != nullptr && (reinterpret_cast<uintptr_t>(op_status) % 4) != 0))
    return NEAT_ERR_ARG;
  return neat::cuda_error_status(
      neat::launch_apply_ops(nodes, conns, P, N, C, ops, K, op_status, stream));
}
