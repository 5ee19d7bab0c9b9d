// Host side of the C ABI declared in include/neat.h: the plan object,
// argument checks, launch-shape choices, and the exported entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>

#include "neat_internal.cuh"

struct neat_plan {
  int device;
  int P, N, C, I, O;
  void *ws;
  size_t ws_bytes;
  neat::Layout L;
  neat::Ws w;
  int sm_count;
  int smem_optin;
  neat_tuning tune;
  int transformed;  // 0: none, 1: feed-forward (neat_transform), 2: recurrent
  // 1 while the plan's last call was a transform: a level forward then must
  // not overlap the kernel before it (the batch programs' writer)
  int after_transform;
};

namespace {

constexpr int kVersion = 100;  // 0.1.0

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool sizes_ok(int P, int N, int C, int I, int O) {
  return P >= 0 && I >= 1 && O >= 1 && N >= I + O && N <= NEAT_MAX_NODES && C >= 1 &&
         C <= NEAT_MAX_CONNS && P <= (1 << 24);
}

thread_local int g_last_cuda_error = 0;

neat_status cuda_status(cudaError_t e) { return neat::cuda_error_status(e); }

// Launch shape of the sample-parallel forward for S samples per genome.
// Every genome's values live in its warp's workspace slot (measured faster
// than shared-memory value arrays on every workload: the L1 caches them and
// many more warps fit on an SM); the slots bound the grid, which is kept to
// whole multiples of the SM count.
neat::SpShape sp_shape(const neat_plan *p, int S, bool compiled = true) {
  neat::SpShape sh{};
  // 8 warps; 4 for large genomes, whose most expensive members are evaluated
  // CTA-wide (smaller CTAs: more of them work on the big genomes at once,
  // measured 8 % faster on the uneven population)
  sh.warps = p->tune.warps_per_cta > 0 ? p->tune.warps_per_cta : (p->N > 256 ? 4 : 8);
  // the compiled walk (outputs only) takes two samples a lane from S = 64 (a
  // tile of 64 samples; uneven genomes at S = 64, us per launch, one / two a
  // lane: 266 / 204 for 256 genomes, 385 / 318 for 2,048, 1,067 / 886 for
  // 16,384); the position walk (saved aggregates) and smaller S one
  // (differentiation forward with saved aggregates, 2,048 genomes at S =
  // 4096: 1,065 us with one, 1,137 with two)
  sh.spl = p->tune.samples_per_lane > 0 ? p->tune.samples_per_lane
                                        : (compiled && S >= 64 ? 2 : 1);
  sh.vcap = 0;
  sh.coop = 1;
  const int slots = neat::sp_scratch_slots(p->w, sh.spl);
  const int occ = std::max(1, neat::forward_sp_occupancy(sh.warps, 0, sh.spl));
  const int64_t tiles = (int64_t(S) + 32 * sh.spl - 1) / (32 * sh.spl);
  const int64_t items = int64_t(p->P) * tiles;
  int64_t cap = std::min<int64_t>(int64_t(p->sm_count) * occ, slots / sh.warps);
  if (cap >= p->sm_count) cap = cap / p->sm_count * p->sm_count;
  const int64_t grid = std::min<int64_t>(cap, (items + sh.warps - 1) / sh.warps);
  sh.grid = int(std::max<int64_t>(1, grid));
  return sh;
}

int small_s_max(const neat_plan *p) {
  return p->tune.small_s_max != 0 ? p->tune.small_s_max : 8;  // -1: never
}

// Per-warp shared memory of the level-synchronous forward above which the
// sample-parallel forward takes small S too (fewer than three warps per SM).
constexpr size_t kLvlWarpMaxBytes = 72 * 1024;

bool lvl_fits(const neat_plan *p, int S) {
  const size_t wb = neat::lvl_warp_bytes(p->w, neat::lvl_tile(S));
  return wb <= kLvlWarpMaxBytes && wb <= size_t(p->smem_optin);
}

// Warps per CTA of the level-synchronous forward: the tuning's lvl_threads,
// else the CTA size (8, 4, 2 or 1 warps) that keeps the most warps resident
// per SM (each warp owns a batch buffer, so the per-SM shared memory is what
// limits them).
int lvl_warps(const neat_plan *p, int st, int *occ_out) {
  const size_t wb = neat::lvl_warp_bytes(p->w, st);
  int best = 0, best_w = 1, best_occ = 1;
  for (int wp : {8, 4, 2, 1}) {
    if (p->tune.lvl_threads > 0 && wp != p->tune.lvl_threads / 32) continue;
    const int occ = neat::forward_lvl_occupancy(wp, wb * size_t(wp), st);
    if (occ * wp > best) { best = occ * wp; best_w = wp; best_occ = occ; }
  }
  if (best == 0) {  // the tuning's CTA size does not fit: fall back to one warp
    best_w = 1;
    best_occ = std::max(1, neat::forward_lvl_occupancy(1, wb, st));
  }
  if (occ_out) *occ_out = best_occ;
  return best_w;
}

// Polls of a staging wait before the level kernel gives up on a batch.
int wait_polls(const neat_plan *p) {
  return p->tune.wait_polls == 0 ? (1 << 22) : (p->tune.wait_polls < 0 ? 0 : p->tune.wait_polls);
}

// Backward CTA: 16 warps over all the shared memory a CTA may have; each
// genome runs on as many warps as its per-warp blocks fit (smaller genomes,
// more warps).
constexpr int kBackwardWarps = 16;
// warps of a backward CTA whose warp arrays sit in workspace slots
constexpr int kBackwardGlobalWarps = 8;

neat_status check_inputs(const neat_plan *p, const float *inputs, int64_t stride, int S) {
  if (S < 0) return NEAT_ERR_ARG;
  if (S == 0 || p->P == 0) return NEAT_OK;
  if (inputs == nullptr || !aligned(inputs, 4)) return NEAT_ERR_ARG;
  if (stride != 0 && stride < int64_t(S) * p->I) return NEAT_ERR_ARG;
  // the persistent kernels count (genome, 32-sample tile) work items in 32 bits
  if (int64_t(p->P) * ((int64_t(S) + 31) / 32) > int64_t(INT32_MAX)) return NEAT_ERR_UNSUPPORTED;
  return NEAT_OK;
}

// copy (and optionally clear) the plan's device failure word
__global__ void k_read_errors(uint32_t *word, uint32_t *dst, int clear) {
  const uint32_t v = *word;
  *dst = v;
  if (clear) *word = 0u;
}

}  // namespace

namespace neat {
neat_status cuda_error_status(cudaError_t e) {
  if (e == cudaSuccess) return NEAT_OK;
  g_last_cuda_error = int(e);
  return NEAT_ERR_CUDA;
}
}  // namespace neat

extern "C" {

int neat_version(void) { return kVersion; }

int neat_last_cuda_error(void) { return g_last_cuda_error; }

const char *neat_status_string(neat_status s) {
  switch (s) {
    case NEAT_OK: return "ok";
    case NEAT_ERR_ARG: return "invalid argument";
    case NEAT_ERR_CUDA: return "CUDA error";
    case NEAT_ERR_WORKSPACE: return "workspace too small";
    case NEAT_ERR_UNSUPPORTED: return "unsupported size";
    case NEAT_ERR_STATE: return "plan not transformed (for this network type)";
    case NEAT_ERR_TIMEOUT: return "a bounded device wait gave up (outputs of its genomes are NaN)";
  }
  return "unknown status";
}

size_t neat_workspace_bytes(int P, int N, int C, int I, int O) {
  if (!sizes_ok(P, N, C, I, O)) return 0;
  return neat::make_layout(P, N, C, I, O).total;
}

neat_status neat_plan_create(neat_plan **out, int P, int N, int C, int I, int O, void *workspace,
                             size_t workspace_bytes) {
  if (out == nullptr) return NEAT_ERR_ARG;
  *out = nullptr;
  if (!sizes_ok(P, N, C, I, O)) return NEAT_ERR_UNSUPPORTED;
  const neat::Layout L = neat::make_layout(P, N, C, I, O);
  if (workspace == nullptr || !aligned(workspace, 256)) return NEAT_ERR_ARG;
  if (workspace_bytes < L.total) return NEAT_ERR_WORKSPACE;
  neat_plan *p = new (std::nothrow) neat_plan;
  if (p == nullptr) return NEAT_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->P = P; p->N = N; p->C = C; p->I = I; p->O = O;
  p->ws = workspace;
  p->ws_bytes = workspace_bytes;
  p->L = L;
  p->w = neat::make_ws(workspace, L, P, N, C, I, O);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  if (e == cudaSuccess && neat::transform_smem(N, C) > size_t(p->smem_optin))
    e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = neat::transform_set_smem_limit(p->smem_optin);
  if (e == cudaSuccess) e = neat::forward_set_smem_limit(p->smem_optin);
  if (e == cudaSuccess) e = neat::backward_set_smem_limit(p->smem_optin);
  if (e == cudaSuccess) e = neat::lvl_set_smem_limit(p->smem_optin);
  // zero the headers and queue counters so a plan is in a defined state
  if (e == cudaSuccess) e = cudaMemset(static_cast<char *>(workspace) + L.hdr, 0,
                                       sizeof(neat::GenomeHdr) * size_t(P));
  if (e == cudaSuccess) e = cudaMemset(static_cast<char *>(workspace) + L.counters, 0,
                                       sizeof(uint32_t) * 64);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete p;
    return cuda_status(e);
  }
  *out = p;
  return NEAT_OK;
}

neat_status neat_plan_destroy(neat_plan *plan) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  delete plan;
  return NEAT_OK;
}

neat_status neat_plan_set_tuning(neat_plan *plan, const neat_tuning *t) {
  if (plan == nullptr || t == nullptr) return NEAT_ERR_ARG;
  if (t->warps_per_cta < 0 || t->warps_per_cta > 16) return NEAT_ERR_ARG;
  if (!(t->samples_per_lane == 0 || t->samples_per_lane == 1 || t->samples_per_lane == 2 ||
        t->samples_per_lane == 4))
    return NEAT_ERR_ARG;
  if (t->lvl_threads < 0 || t->lvl_threads > 256 || (t->lvl_threads % 32) != 0)
    return NEAT_ERR_ARG;
  if (t->small_s_max < -1 || t->small_s_max > 64) return NEAT_ERR_ARG;
  if (t->lvl_budget_kb != 0 && (t->lvl_budget_kb * 1024 < neat::LVL_MIN_BUDGET ||
                                t->lvl_budget_kb * 1024 > neat::LVL_MAX_BUDGET))
    return NEAT_ERR_ARG;
  if (t->prune_dead != 0 && t->prune_dead != 1) return NEAT_ERR_ARG;
  if (t->wait_polls < -1) return NEAT_ERR_ARG;
  if (t->bwd_global != 0 && t->bwd_global != 1) return NEAT_ERR_ARG;
  plan->tune = *t;
  return NEAT_OK;
}

neat_status neat_plan_get_tuning(const neat_plan *plan, neat_tuning *t) {
  if (plan == nullptr || t == nullptr) return NEAT_ERR_ARG;
  *t = plan->tune;
  const neat::SpShape sh = sp_shape(plan, 32);
  if (t->warps_per_cta == 0) t->warps_per_cta = sh.warps;
  // (samples_per_lane 0 stays 0: each forward picks it from its S)
  if (t->lvl_threads == 0) t->lvl_threads = 32 * lvl_warps(plan, 1, nullptr);
  if (t->small_s_max == 0) t->small_s_max = small_s_max(plan);
  // (lvl_budget_kb 0 stays 0: the transform picks the budget per population)
  if (t->wait_polls == 0) t->wait_polls = wait_polls(plan);
  return NEAT_OK;
}

neat_status neat_plan_device_errors(neat_plan *plan, uint32_t *errors, int clear,
                                    cudaStream_t stream) {
  if (plan == nullptr || errors == nullptr || !aligned(errors, 4)) return NEAT_ERR_ARG;
  k_read_errors<<<1, 1, 0, stream>>>(plan->w.counters + neat::CTR_ERR, errors, clear ? 1 : 0);
  return cuda_status(cudaGetLastError());
}

neat_status neat_plan_check(neat_plan *plan, cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  uint32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, plan->w.counters + neat::CTR_ERR, sizeof(word),
                                  cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e == cudaSuccess && word != 0u)
    e = cudaMemsetAsync(plan->w.counters + neat::CTR_ERR, 0, sizeof(uint32_t), stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (word & NEAT_DEV_TIMEOUT) return NEAT_ERR_TIMEOUT;
  if (word & NEAT_DEV_NO_SCRATCH) return NEAT_ERR_WORKSPACE;
  return NEAT_OK;
}

neat_status neat_plan_validate(const neat_plan *plan, uint32_t *bits, cudaStream_t stream) {
  if (plan == nullptr || bits == nullptr || !aligned(bits, 4)) return NEAT_ERR_ARG;
  if (plan->transformed == 0) return NEAT_ERR_STATE;
  return cuda_status(neat::launch_validate(plan->w, plan->L, plan->transformed == 1 ? 1 : 0, bits,
                                           plan->sm_count, stream));
}

neat_status neat_transform(neat_plan *plan, const float *nodes, const float *conns, int32_t *order,
                           int32_t *layer, int32_t *n_layers, uint32_t *gstatus,
                           cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  if (plan->P > 0) {
    if (nodes == nullptr || conns == nullptr || order == nullptr || layer == nullptr ||
        n_layers == nullptr || gstatus == nullptr)
      return NEAT_ERR_ARG;
    if (!aligned(nodes, 4) || !aligned(conns, 16) || !aligned(order, 4) || !aligned(layer, 4) ||
        !aligned(n_layers, 4) || !aligned(gstatus, 4))
      return NEAT_ERR_ARG;
  }
  plan->after_transform = 1;  // (set before any launch: also on a failure below)
  // the batch budget is fixed by the transform that builds the batches
  plan->w.prune = plan->tune.prune_dead == 1 ? 1 : 0;
  plan->w.lvl_budget =
      neat::lvl_budget(plan->N, plan->C, plan->I, plan->O, plan->tune.lvl_budget_kb * 1024);
  // a new population: the device error word starts clean
  cudaError_t e = cudaMemsetAsync(plan->w.counters + neat::CTR_ERR, 0, sizeof(uint32_t), stream);
  if (e == cudaSuccess) e = neat::launch_transform(plan->w, nodes, conns, order, layer, n_layers, gstatus,
                                         stream);
  if (e == cudaSuccess) e = neat::launch_queue_build(plan->w, 0, stream);
  // without a budget knob the batches are cut to fill the resident warps of a
  // one-sample forward (the rollout step's form)
  int target = 0;
  if (plan->tune.lvl_budget_kb == 0) {
    int occ = 1;
    const int warps = lvl_warps(plan, 1, &occ);
    target = plan->sm_count * std::max(1, occ) * warps;
  }
  if (e == cudaSuccess)
    e = neat::launch_lvl_build(plan->w, target,
                               neat::lvl_min_budget(plan->N, plan->C, plan->I, plan->O), stream);
  if (e != cudaSuccess) return cuda_status(e);
  plan->transformed = 1;
  return NEAT_OK;
}

neat_status neat_forward(neat_plan *plan, const float *inputs, int64_t in_pop_stride, int S,
                         float *outputs, float *saved, cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  if (plan->transformed != 1) return NEAT_ERR_STATE;
  neat_status s = check_inputs(plan, inputs, in_pop_stride, S);
  if (s != NEAT_OK) return s;
  if (S == 0 || plan->P == 0) return NEAT_OK;
  if (outputs == nullptr || !aligned(outputs, 4) || (saved && !aligned(saved, 4)))
    return NEAT_ERR_ARG;
  if (saved == nullptr && S <= small_s_max(plan) && lvl_fits(plan, S)) {
    // few samples per genome: level-synchronous batches of genomes, one per warp
    const int st = neat::lvl_tile(S);
    int occ = 1;
    const int warps = lvl_warps(plan, st, &occ);
    const int64_t want = (int64_t(plan->P) + warps - 1) / warps;  // batches <= P
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(plan->sm_count) * occ, want)));
    // programmatic dependent launch unless the previous call was a transform
    const int pdl = plan->after_transform ? 0 : 1;
    plan->after_transform = 0;
    return cuda_status(neat::launch_forward_lvl(plan->w, inputs, in_pop_stride, S, outputs, warps,
                                                grid, wait_polls(plan), pdl, stream));
  }
  const neat::SpShape sh = sp_shape(plan, S, saved == nullptr && plan->w.cnode != nullptr);
  if (int64_t(sh.grid) * sh.warps > neat::sp_scratch_slots(plan->w, sh.spl))
    return NEAT_ERR_UNSUPPORTED;
  return cuda_status(neat::launch_forward_sp(plan->w, inputs, in_pop_stride, S, outputs, saved, sh,
                                             stream));
}

neat_status neat_forward_plain(neat_plan *plan, const float *inputs, int64_t in_pop_stride, int S,
                               float *outputs, cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  if (plan->transformed != 1) return NEAT_ERR_STATE;
  neat_status s = check_inputs(plan, inputs, in_pop_stride, S);
  if (s != NEAT_OK) return s;
  if (S == 0 || plan->P == 0) return NEAT_OK;
  if (outputs == nullptr || !aligned(outputs, 4)) return NEAT_ERR_ARG;
  if ((S + 31) / 32 > 65535) return NEAT_ERR_UNSUPPORTED;
  return cuda_status(neat::launch_forward_plain(plan->w, inputs, in_pop_stride, S, outputs, stream));
}

neat_status neat_backward(neat_plan *plan, const float *inputs, int64_t in_pop_stride, int S,
                          const float *grad_outputs, const float *saved, float *grad_weight,
                          float *grad_bias, float *grad_response, float *grad_inputs,
                          cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  if (plan->transformed != 1) return NEAT_ERR_STATE;
  neat_status s = check_inputs(plan, inputs, in_pop_stride, S);
  if (s != NEAT_OK) return s;
  if (plan->P == 0) return NEAT_OK;
  if (grad_weight == nullptr || grad_bias == nullptr || grad_response == nullptr)
    return NEAT_ERR_ARG;
  if (S > 0 && grad_outputs == nullptr) return NEAT_ERR_ARG;
  if (!aligned(grad_weight, 4) || !aligned(grad_bias, 4) || !aligned(grad_response, 4) ||
      (grad_outputs && !aligned(grad_outputs, 4)) || (saved && !aligned(saved, 4)) ||
      (grad_inputs && !aligned(grad_inputs, 4)))
    return NEAT_ERR_ARG;
  const bool fits = neat::backward_smem(plan->N, plan->C, 1) <= size_t(plan->smem_optin);
  if (fits && plan->tune.bwd_global == 0) {
    const int smem = int(std::min<size_t>(size_t(plan->smem_optin),
                                          neat::backward_smem(plan->N, plan->C, kBackwardWarps)));
    return cuda_status(neat::launch_backward(plan->w, inputs, in_pop_stride, S, grad_outputs,
                                             saved, grad_weight, grad_bias, grad_response,
                                             grad_inputs, kBackwardWarps, smem, false, 0, stream));
  }
  // per-warp arrays in workspace slots: the records and pull lists must still
  // fit in shared memory, and one CTA's slots in the workspace
  const size_t fixed = neat::backward_fixed_smem(plan->N, plan->C);
  if (fixed > size_t(plan->smem_optin)) return NEAT_ERR_UNSUPPORTED;
  const size_t cta_floats = size_t(kBackwardGlobalWarps) *
                            neat::backward_slot_floats(plan->N, plan->C);
  const int64_t slots = plan->w.sp_scratch ? int64_t(plan->w.sp_scratch_floats / cta_floats) : 0;
  const int occ = neat::backward_occupancy(true, kBackwardGlobalWarps, int(fixed));
  int64_t ctas = std::min<int64_t>({int64_t(plan->P), int64_t(plan->sm_count) * std::max(1, occ),
                                    slots});
  if (ctas < 1) return NEAT_ERR_WORKSPACE;
  return cuda_status(neat::launch_backward(plan->w, inputs, in_pop_stride, S, grad_outputs, saved,
                                           grad_weight, grad_bias, grad_response, grad_inputs,
                                           kBackwardGlobalWarps, int(fixed), true, int(ctas),
                                           stream));
}

neat_status neat_sum_genomes(const float *x, int P, int64_t n, float *out, cudaStream_t stream) {
  if (P < 0 || n < 0) return NEAT_ERR_ARG;
  if (n == 0) return NEAT_OK;
  if (out == nullptr || !aligned(out, 4) || (P > 0 && (x == nullptr || !aligned(x, 4))))
    return NEAT_ERR_ARG;
  // the two ranges may not overlap
  const uintptr_t xb = reinterpret_cast<uintptr_t>(x), ob = reinterpret_cast<uintptr_t>(out);
  if (P > 0 && xb < ob + sizeof(float) * size_t(n) && ob < xb + sizeof(float) * size_t(P) * size_t(n))
    return NEAT_ERR_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = neat::launch_sum_genomes(x, P, n, out, sms, stream);
  return cuda_status(e);
}

neat_status neat_hyperneat_query(neat_plan *plan, int grid, float thresh, float *weights,
                                 cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  if (plan->transformed != 1) return NEAT_ERR_STATE;
  if (plan->I != 5 || plan->O != 1) return NEAT_ERR_UNSUPPORTED;
  if (grid < 2 || grid > 128) return NEAT_ERR_ARG;
  if (plan->P == 0) return NEAT_OK;
  if (weights == nullptr || !aligned(weights, 4)) return NEAT_ERR_ARG;
  // four queries a lane, 16-warp CTAs (256 CPPNs of 64 nodes on the 32 x 32
  // grid, ms: 12.12 against 12.63 with two a lane; 16 / 8 / 4 warps a CTA at
  // two a lane: 12.63 / 12.67 / 13.91)
  const int spl = plan->tune.samples_per_lane > 0 ? plan->tune.samples_per_lane : 4;
  const int warps = plan->tune.warps_per_cta > 0 ? plan->tune.warps_per_cta : 16;
  // shared memory per CTA: an SM's share for about 32 resident warps (the
  // staged program plus as many value arrays as fit), less the static part
  int per_sm = 0, reserved = 0;
  cudaError_t e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                         plan->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, plan->device);
  if (e != cudaSuccess) return cuda_status(e);
  const int want = std::max(1, 32 / warps);
  const int prog = neat::hn_prog_bytes(plan->N, plan->C);
  int smem = std::min(plan->smem_optin, per_sm / want - reserved) - 1024;
  // a CTA holds at least the program and one value array of a full-size
  // genome (fewer CTAs per SM for large N, C)
  const int64_t rows_max = int64_t(plan->N + 2) * 32 * spl * 4;
  if (smem < prog + rows_max) smem = plan->smem_optin - 1024;
  if (smem < prog) return NEAT_ERR_UNSUPPORTED;
  const int occ = std::max(1, neat::hyperneat_occupancy(spl, warps, size_t(smem)));
  int64_t ctas = int64_t(plan->sm_count) * occ;
  if (rows_max + prog > smem) {  // some genomes may use workspace slots: one per warp
    ctas = std::min<int64_t>(ctas, neat::sp_scratch_slots(plan->w, spl) / warps);
    if (ctas >= plan->sm_count) ctas -= ctas % plan->sm_count;
  }
  if (ctas < 1) return NEAT_ERR_UNSUPPORTED;
  return cuda_status(neat::launch_hyperneat(plan->w, grid, thresh, weights, spl, warps,
                                            int(ctas), smem, stream));
}

neat_status neat_hyperneat_substrate(neat_plan *plan, int grid, float thresh, const float *inputs,
                                     int64_t in_pop_stride, int S, int act, float *weights,
                                     float *outputs, cudaStream_t stream) {
  neat_status s = neat_hyperneat_query(plan, grid, thresh, weights, stream);
  if (s != NEAT_OK) return s;
  return neat_substrate_forward(weights, plan->P, grid * grid, inputs, in_pop_stride, S, act,
                                outputs, stream);
}

neat_status neat_mutate_transform(neat_plan *plan, float *nodes, float *conns, const float *ops,
                                  int K, uint32_t *op_status, int32_t *order, int32_t *layer,
                                  int32_t *n_layers, uint32_t *gstatus, cudaStream_t stream) {
  if (plan == nullptr || K < 0) return NEAT_ERR_ARG;
  if (plan->P > 0 && (K > 0 && ops == nullptr)) return NEAT_ERR_ARG;
  if (plan->P > 0 && ((K > 0 && !aligned(ops, 4)) || (op_status && !aligned(op_status, 4))))
    return NEAT_ERR_ARG;
  if (plan->P > 0 && (nodes == nullptr || conns == nullptr)) return NEAT_ERR_ARG;
  if (plan->P > 0 && K > 0) {
    if (!aligned(nodes, 4) || !aligned(conns, 16)) return NEAT_ERR_ARG;
    cudaError_t e = neat::launch_apply_ops(nodes, conns, plan->P, plan->N, plan->C, ops, K,
                                           op_status, stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return neat_transform(plan, nodes, conns, order, layer, n_layers, gstatus, stream);
}

neat_status neat_transform_recurrent(neat_plan *plan, const float *nodes, const float *conns,
                                     uint32_t *gstatus, cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  if (plan->P > 0) {
    if (nodes == nullptr || conns == nullptr || gstatus == nullptr) return NEAT_ERR_ARG;
    if (!aligned(nodes, 4) || !aligned(conns, 16) || !aligned(gstatus, 4)) return NEAT_ERR_ARG;
  }
  cudaError_t e = neat::launch_transform(plan->w, nodes, conns, nullptr, nullptr, nullptr, gstatus,
                                         stream, 1);
  if (e == cudaSuccess) e = neat::launch_queue_build(plan->w, 0, stream);
  if (e != cudaSuccess) return cuda_status(e);
  plan->transformed = 2;
  plan->after_transform = 1;
  return NEAT_OK;
}

neat_status neat_forward_recurrent(neat_plan *plan, const float *inputs, int64_t in_pop_stride,
                                   int S, int T, float *outputs, cudaStream_t stream) {
  if (plan == nullptr) return NEAT_ERR_ARG;
  if (plan->transformed == 0) return NEAT_ERR_STATE;
  if (T < 0 || T > (1 << 16)) return NEAT_ERR_ARG;
  neat_status s = check_inputs(plan, inputs, in_pop_stride, S);
  if (s != NEAT_OK) return s;
  if (S == 0 || plan->P == 0) return NEAT_OK;
  if (outputs == nullptr || !aligned(outputs, 4)) return NEAT_ERR_ARG;
  // 8 warps per CTA (the tuning's warps_per_cta if set); one sample per lane
  // (the tuning's samples_per_lane, 1 or 2, if set: two measured 25 % slower
  // on 10,000 genomes at S = 64, T = 8); two value buffers per warp bound the
  // grid, kept to whole multiples of the SM count
  const int warps = plan->tune.warps_per_cta > 0 ? plan->tune.warps_per_cta : 8;
  const int spl = plan->tune.samples_per_lane > 0 ? std::min(plan->tune.samples_per_lane, 2) : 1;
  const int slots = neat::sp_scratch_slots(plan->w, 2 * spl);
  const int occ = std::max(1, neat::forward_rec_occupancy(warps, spl));
  const int64_t items = int64_t(plan->P) * ((S + 32 * spl - 1) / (32 * spl));
  int64_t cap = std::min<int64_t>(int64_t(plan->sm_count) * occ, slots / warps);
  if (cap >= plan->sm_count) cap = cap / plan->sm_count * plan->sm_count;
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(cap, (items + warps - 1) / warps)));
  if (int64_t(grid) * warps > slots) return NEAT_ERR_UNSUPPORTED;
  return cuda_status(neat::launch_forward_recurrent(plan->w, inputs, in_pop_stride, S, T, outputs,
                                                    spl, warps, grid, stream));
}

}  // extern "C"
