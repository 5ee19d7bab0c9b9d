// Shared-memory read bandwidth probe: the peak behind the on-chip term of the
// forward/backward roofline (node-value reads and writes are on-chip traffic;
// the L1 and shared memory share one 128-byte-per-clock data path per SM).
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kWords = 4096;  // uint4 words: 64 KiB per CTA
constexpr int kUnroll = 8;

// Thread t of iteration it reads words (t + u * 512 + it) mod 4096, u < 8:
// consecutive threads read consecutive 16-byte words (no bank conflicts), and
// the shift by `it` keeps the loads inside the loop.  32-bit word w of the
// array holds w * 0x9E3779B1.
__global__ void __launch_bounds__(kThreads) k_smem_probe(int iters, uint32_t *sink) {
  extern __shared__ uint4 buf[];  // kWords words
  const int t = threadIdx.x;
  for (int i = t; i < kWords; i += kThreads) {
    const uint32_t w = uint32_t(i) * 4u;
    buf[i] = make_uint4(w * 0x9E3779B1u, (w + 1u) * 0x9E3779B1u, (w + 2u) * 0x9E3779B1u,
                        (w + 3u) * 0x9E3779B1u);
  }
  __syncthreads();
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint4 x = buf[(t + u * kThreads + it) & (kWords - 1)];
      acc.x ^= x.x;
      acc.y ^= x.y;
      acc.z ^= x.z;
      acc.w ^= x.w;
    }
  }
  sink[size_t(blockIdx.x) * kThreads + t] = acc.x ^ acc.y ^ acc.z ^ acc.w;
}

}  // namespace

extern "C" neat_status neat_probe_smem_read(int blocks, int iters, uint32_t *sink,
                                            cudaStream_t stream) {
  if (blocks < 1 || iters < 0 || sink == nullptr || (reinterpret_cast<uintptr_t>(sink) % 4) != 0)
    return NEAT_ERR_ARG;
  const int bytes = kWords * int(sizeof(uint4));
  const cudaError_t e =
      cudaFuncSetAttribute(k_smem_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return neat::cuda_error_status(e);
  k_smem_probe<<<blocks, kThreads, bytes, stream>>>(iters, sink);
  return neat::cuda_error_status(cudaGetLastError());
}
