// neat_forward_noalloc: transformation + batched forward in one call, with
// every byte of working memory taken from a fixed array compiled into the
// library instead of a caller- or library-allocated workspace.
//
// Some callers cannot allocate device memory at the moment they evaluate a
// population: code running inside an allocator-free region (a real-time
// control loop that must not touch the CUDA allocator, a host runtime whose
// memory pool is owned by another framework, a plugin that is handed only
// input and output buffers).  They still provide inputs and outputs; this
// entry point uses NEAT_NOALLOC_SCRATCH_BYTES of static device memory for the
// plan workspace and the transform's order / layer tensors.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and raises the kernels'
// shared-memory limits; make that first call before any stream capture.
// Every call shares the one array: calls that overlap on the GPU (two streams,
// or two host threads on one device) race on it and must be serialised by the
// caller.  The array keeps the last call's contents; each call clears the
// queue counters it depends on before use.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "neat_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NEAT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
int g_smem_optin[kMaxDevices] = {};

// per-device set-up: address of the array, SM count, shared-memory limits
cudaError_t setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_ptr[dev] != nullptr) return cudaSuccess;
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  int sms = 0, optin = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = neat::transform_set_smem_limit(optin);
  if (e == cudaSuccess) e = neat::forward_set_smem_limit(optin);
  if (e == cudaSuccess) e = neat::lvl_set_smem_limit(optin);
  if (e != cudaSuccess) return e;
  g_sm_count[dev] = sms;
  g_smem_optin[dev] = optin;
  g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// bytes of the array a population of these sizes uses (0 for invalid sizes):
// the plan regions this call touches (headers, padded and packed programs,
// both queue orders, counters; not the small-S batches, the compiled
// programs or the workspace value slots) and the transform's order, layer and
// layer-count arrays, each region rounded up to 256 bytes
size_t scratch_needed(int P, int N, int C, int I, int O) {
  if (P < 0 || I < 1 || O < 1 || N < I + O || N > NEAT_MAX_NODES || C < 1 || C > NEAT_MAX_CONNS)
    return 0;
  const neat::Layout L = neat::make_layout(P, N, C, I, O);
  const size_t pn = sizeof(int32_t) * size_t(P) * N;
  return L.base + 2 * align256(pn) + align256(sizeof(int32_t) * size_t(P));
}

// warps per CTA and shared memory of the sample-parallel forward with every
// genome's values in shared memory
void sp_launch_shape(int N, int &warps, size_t &smem) {
  warps = 8;
  while (warps > 1 && neat::forward_sp_smem(N, warps, 1) > size_t(96 * 1024)) --warps;
  smem = neat::forward_sp_smem(N, warps, 1);
}

}  // namespace

extern "C" neat_status neat_forward_noalloc(const float *nodes, const float *conns, int P, int N,
                                            int C, int I, int O, const float *inputs,
                                            int64_t in_pop_stride, int S, float *outputs,
                                            uint32_t *gstatus, cudaStream_t stream) {
  const size_t need = scratch_needed(P, N, C, I, O);
  if (need == 0) return NEAT_ERR_UNSUPPORTED;
  if (need > size_t(NEAT_NOALLOC_SCRATCH_BYTES)) return NEAT_ERR_WORKSPACE;  // beyond the fixed array
  if (S < 0) return NEAT_ERR_ARG;
  if (P == 0) return NEAT_OK;
  if (nodes == nullptr || conns == nullptr || gstatus == nullptr ||
      (reinterpret_cast<uintptr_t>(conns) % 16) != 0 || (reinterpret_cast<uintptr_t>(nodes) % 4) != 0 ||
      (reinterpret_cast<uintptr_t>(gstatus) % 4) != 0)
    return NEAT_ERR_ARG;
  if (S > 0 && (inputs == nullptr || outputs == nullptr ||
                (reinterpret_cast<uintptr_t>(inputs) % 4) != 0 ||
                (reinterpret_cast<uintptr_t>(outputs) % 4) != 0))
    return NEAT_ERR_ARG;
  if (in_pop_stride != 0 && in_pop_stride < int64_t(S) * I) return NEAT_ERR_ARG;
  // (genome, 32-sample tile) work items are counted in 32 bits
  if (int64_t(P) * ((int64_t(S) + 31) / 32) > int64_t(INT32_MAX)) return NEAT_ERR_UNSUPPORTED;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return neat::cuda_error_status(e);
  if (dev < 0 || dev >= kMaxDevices) return NEAT_ERR_UNSUPPORTED;
  e = setup_device(dev);
  if (e != cudaSuccess) return neat::cuda_error_status(e);
  // every shape check before the first launch
  if (neat::transform_smem(N, C) > size_t(g_smem_optin[dev])) return NEAT_ERR_UNSUPPORTED;
  int warps = 1;
  size_t smem = 0;
  sp_launch_shape(N, warps, smem);
  if (S > 0 && smem > size_t(g_smem_optin[dev])) return NEAT_ERR_UNSUPPORTED;

  unsigned char *base = g_scratch_ptr[dev];
  const neat::Layout L = neat::make_layout(P, N, C, I, O);
  neat::Ws w = neat::make_ws(base, L, P, N, C, I, O);
  // only the base regions of the layout live in the array
  w.lvl_goff = nullptr;
  w.lvl_first = nullptr;
  w.lvl_loc = nullptr;
  w.lvl_arena = nullptr;
  w.cnode = nullptr;
  w.cpair = nullptr;
  w.cout = nullptr;
  w.clay = nullptr;
  w.sp_scratch = nullptr;
  w.sp_scratch_floats = 0;
  int32_t *order = reinterpret_cast<int32_t *>(base + L.base);
  int32_t *layer = reinterpret_cast<int32_t *>(base + L.base +
                                               align256(sizeof(int32_t) * size_t(P) * N));
  int32_t *n_layers = reinterpret_cast<int32_t *>(base + L.base +
                                                  2 * align256(sizeof(int32_t) * size_t(P) * N));

  // the queue counters and the failure word must start at zero (the array
  // keeps the last call's state)
  e = cudaMemsetAsync(base + L.counters, 0, sizeof(uint32_t) * 64, stream);
  if (e == cudaSuccess)
    e = neat::launch_transform(w, nodes, conns, order, layer, n_layers, gstatus, stream);
  if (e == cudaSuccess) e = neat::launch_queue_build(w, 0, stream);
  if (e == cudaSuccess && S > 0) {
    const int occ = std::max(1, neat::forward_sp_occupancy(warps, smem, 1));
    const int64_t items = int64_t(P) * ((S + 31) / 32);
    const int grid = int(std::max<int64_t>(
        1, std::min<int64_t>(int64_t(g_sm_count[dev]) * occ, (items + warps - 1) / warps)));
    const neat::SpShape sh{warps, 1, N, grid, 0};
    e = neat::launch_forward_sp(w, inputs, in_pop_stride, S, outputs, nullptr, sh, stream);
  }
  return neat::cuda_error_status(e);
}
