// Level-synchronous batched forward for small sample counts (one or a few
// input vectors per genome, e.g. one observation per rollout step).
//
// With S = 1 a single genome offers only the few independent nodes of one
// layer at a time, so genomes are evaluated in small BATCHES: all their
// layer-r nodes are independent of each other (Sec. 3.3's order only requires
// each node to follow its inputs), so a round evaluates the layer-r nodes of
// every genome in the batch.  Each batch belongs to one warp, which stages the
// batch program into its own shared-memory buffer and runs the rounds with
// __syncwarp only: a shallow batch never waits for a deep one, and no
// CTA-wide barrier sits in a round.  A round has two passes: one lane per
// 4-edge chunk of incoming connections (the partial of the task's
// aggregation), then one lane per node (combine the partials, bias, response,
// activation).  The node pass evaluates each activation function present in
// the round once for the whole warp (a warp-uniform branch per function), so
// the mixed activations of a round cost one evaluation of each kind.
//
// Transform time (k_lvl_plan, k_lvl_build): genomes in layer-sorted queue
// order are cut into batches whose programs fit the per-warp buffer, and each
// batch program is written contiguously (see BatchHead in neat_internal.cuh).
// Run time (k_forward_lvl): a warp claims a batch and stages its program with
// two bulk copies (cp.async.bulk with mbarrier completion and bounded waits):
// the head part (genome ids, I/O slots, round table) first, so the step's
// input loads are issued while the tasks and edges are still in flight.
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

__device__ __forceinline__ int pow2_ceil_d(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ---------------------------------------------------------------------------
// Batch assignment (one CTA).  Every thread takes a contiguous run of the
// layer-sorted queue (at least 128 genomes) and cuts it greedily: a genome
// joins the current batch unless the batch's byte bound would exceed the
// per-warp buffer, its value slots the slot cap, or it holds LVL_MAX_GENOMES.
// Runs never share a batch, so the cut is exact and parallel; a run ends with
// one partly filled batch.  Batch b's program sits at arena offset
// goff[first genome of b] + LVL_BATCH_FIXED * b, goff being the prefix of the
// genome byte bounds in queue order.
constexpr int PLAN_THREADS = 1024;

__global__ void __launch_bounds__(PLAN_THREADS) k_lvl_plan(Ws w) {
  __shared__ long long sb[32];
  __shared__ int sn[32];
  const int P = w.P, T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int I = w.I, O = w.O, cap = w.lvl_budget, scap = w.lvl_slots;
  const int per = max(128, (P + T - 1) / T);
  const int q0 = min(tid * per, P), q1 = min(q0 + per, P);
  auto genome = [&](int q, int &pb, int &V) {
    const GenomeHdr h = w.hdr[w.qlvl[q]];
    const bool ok = h.status == 0u;
    pb = lvl_genome_bytes(h.nlive, h.nch, h.L, I, O, ok);  // tasks: the evaluated nodes
    V = ok ? h.V : 0;
  };
  // pass 1: batches and bytes of this thread's run
  int nb = 0;
  long long by = 0;
  {
    int cb = 0, cs = 0, cg = 0;
    for (int q = q0; q < q1; ++q) {
      int pb, V;
      genome(q, pb, V);
      if (cg == 0 || cg == LVL_MAX_GENOMES || cb + pb > cap || cs + V > scap) {
        ++nb;
        cb = LVL_BATCH_FIXED;
        cs = 0;
        cg = 0;
      }
      cb += pb;
      cs += V;
      ++cg;
      by += pb;
    }
  }
  // exclusive scans over the threads
  int xn = nb;
  long long xb = by;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int yn = __shfl_up_sync(0xffffffffu, xn, d);
    const long long yb = __shfl_up_sync(0xffffffffu, xb, d);
    if (lane >= d) { xn += yn; xb += yb; }
  }
  if (lane == 31) { sn[wid] = xn; sb[wid] = xb; }
  __syncthreads();
  if (wid == 0) {
    int a = lane < (T >> 5) ? sn[lane] : 0;
    long long c = lane < (T >> 5) ? sb[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int ya = __shfl_up_sync(0xffffffffu, a, d);
      const long long yc = __shfl_up_sync(0xffffffffu, c, d);
      if (lane >= d) { a += ya; c += yc; }
    }
    if (lane < (T >> 5)) { sn[lane] = a; sb[lane] = c; }
  }
  __syncthreads();
  // pass 2: first genome of each batch, genome byte offsets
  {
    int b = (wid > 0 ? sn[wid - 1] : 0) + xn - nb - 1;
    long long off = (wid > 0 ? sb[wid - 1] : 0) + xb - by;
    int cb = 0, cs = 0, cg = 0;
    for (int q = q0; q < q1; ++q) {
      int pb, V;
      genome(q, pb, V);
      if (cg == 0 || cg == LVL_MAX_GENOMES || cb + pb > cap || cs + V > scap) {
        ++b;
        w.lvl_first[b] = q;
        cb = LVL_BATCH_FIXED;
        cs = 0;
        cg = 0;
      }
      cb += pb;
      cs += V;
      ++cg;
      w.lvl_goff[q] = int(off);
      off += pb;
    }
  }
  if (tid == T - 1) {
    const int total = sn[(T >> 5) - 1];
    w.lvl_first[total] = P;
    w.counters[CTR_NBATCH] = uint32_t(total);
  }
}

// ---------------------------------------------------------------------------
// one CTA per batch: gather, sort and write the batch program
constexpr int BLD_THREADS = 256;

__global__ void __launch_bounds__(BLD_THREADS) k_lvl_build(Ws w) {
  __shared__ int g_id[LVL_MAX_GENOMES + 1], g_V[LVL_MAX_GENOMES + 1], g_L[LVL_MAX_GENOMES + 1];
  __shared__ int g_noff[LVL_MAX_GENOMES + 1], g_eoff[LVL_MAX_GENOMES + 1];
  __shared__ int g_slot[LVL_MAX_GENOMES + 1], g_NL[LVL_MAX_GENOMES + 1];
  __shared__ int s_nslots, s_ntasks, s_nrounds, s_bad;
  __shared__ int wbuf[33];
  extern __shared__ __align__(16) unsigned char dsm[];
  uint64_t *keys = reinterpret_cast<uint64_t *>(dsm);               // [LVL_MAX_SLOTS]
  int *cnt = reinterpret_cast<int *>(dsm + 8 * LVL_MAX_SLOTS);      // [LVL_MAX_SLOTS + 1]

  const int b = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int nb = int(w.counters[CTR_NBATCH]);
  if (b >= nb) return;
  const int I = w.I, O = w.O, pcap = w.lvl_pcap;
  const int q0 = w.lvl_first[b], q1 = w.lvl_first[b + 1];
  const int ng = q1 - q0;
  if (tid == 0) s_bad = (ng < 1 || ng > LVL_MAX_GENOMES) ? 1 : 0;
  __syncthreads();
  if (s_bad) return;  // cannot happen by construction of the cut
  for (int k = tid; k < ng; k += T) {
    const int g = w.qlvl[q0 + k];
    const GenomeHdr h = w.hdr[g];
    const bool ok = h.status == 0u;
    g_id[k] = g;
    g_V[k] = ok ? h.V : 0;
    g_L[k] = ok ? h.L : 0;
    g_NL[k] = ok ? h.nlive : 0;
    g_noff[k] = h.node_off;
    g_eoff[k] = h.edge_off;
  }
  __syncthreads();
  if (tid == 0) {
    int s = 0, nt = 0;
    for (int k = 0; k < ng; ++k) {
      g_slot[k] = s;
      s += g_V[k];
      nt += g_NL[k];
    }
    g_slot[ng] = s;
    s_nslots = s;
    s_ntasks = nt;
  }
  __syncthreads();
  const int nslots = s_nslots, ntasks = s_ntasks;
  if (nslots > w.lvl_slots) return;  // cannot happen by construction of the cut
  const int n2 = pow2_ceil_d(max(nslots, 1));
  // task keys: (layer, act, -cnt, genome, position); inputs and the nodes no
  // output depends on sort last (they are not tasks)
  for (int i = tid; i < n2; i += T) {
    uint64_t key = ~0ull;
    if (i < nslots) {
      int k = 0;
      while (g_slot[k + 1] <= i) ++k;
      const int p = i - g_slot[k];
      const NodeRec n = w.knode[g_noff[k] + p];
      if (!(n.meta & (META_INPUT | META_DEAD))) {
        const uint64_t lay = uint64_t(w.player[size_t(g_id[k]) * w.N + p]);
        key = (lay << 33) | (uint64_t(meta_act(n.meta)) << 30) |
              (uint64_t(16383 - meta_cnt(n.meta)) << 16) | (uint64_t(k) << 10) | uint64_t(p);
      }
    }
    keys[i] = key;
  }
  __syncthreads();
  for (int kk = 2; kk <= n2; kk <<= 1)
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < (n2 >> 1); i += T) {
        const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
        const int hi = lo + j;
        const uint64_t x = keys[lo], y = keys[hi];
        const bool up = (lo & kk) == 0;
        if ((x > y) == up) {
          keys[lo] = y;
          keys[hi] = x;
        }
      }
      __syncthreads();
    }
  // 4-edge chunks of each task
  for (int j = tid; j < ntasks; j += T) cnt[j] = (16383 - int((keys[j] >> 16) & 0x3fffu) + 3) >> 2;
  __syncthreads();
  // exclusive scan of chunk counts -> first chunk of each task
  {
    const int per = (ntasks + T - 1) / T;
    const int lo = min(tid * per, ntasks), hi = min(lo + per, ntasks);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    int x = s;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wbuf[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int a = lane < (T >> 5) ? wbuf[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, a, d);
        if (lane >= d) a += y;
      }
      if (lane < (T >> 5)) wbuf[lane] = a;
    }
    __syncthreads();
    int base = (wid > 0 ? wbuf[wid - 1] : 0) + x - s;
    for (int i = lo; i < hi; ++i) {
      const int c = cnt[i];
      cnt[i] = base;
      base += c;
    }
    if (tid == 0) cnt[ntasks] = wbuf[(T >> 5) - 1];
    __syncthreads();
  }
  const int nchunks = cnt[ntasks];
  // rounds: one layer each, split where a layer exceeds pcap chunks (a single
  // task never does: pcap >= the chunks of a node's in-degree)
  auto new_round = [&](int j, int cur, int in, int nc) {
    return j == 0 || int(keys[j] >> 33) != cur || in + nc > pcap;
  };
  if (tid == 0) {
    int R = 0, in = 0, cur = -1;
    for (int j = 0; j < ntasks; ++j) {
      const int nc = cnt[j + 1] - cnt[j];
      if (new_round(j, cur, in, nc)) {
        ++R;
        in = 0;
        cur = int(keys[j] >> 33);
      }
      in += nc;
    }
    s_nrounds = R;
  }
  __syncthreads();
  const int nrounds = s_nrounds;
  // program layout: head part (header, gio, round table), then tasks and edges
  const int G = 1 + I + O;
  const int off_gio = int(sizeof(BatchHead));
  const int off_round = (off_gio + 4 * ng * G + 15) & ~15;
  const int off_task = (off_round + 4 * (nrounds + 1) + 15) & ~15;
  const int off_eslot = off_task + int(sizeof(TaskRec)) * ntasks;
  const int off_ew = (off_eslot + 8 * nchunks + 15) & ~15;
  const int bytes = (off_ew + 16 * nchunks + 15) & ~15;
  const int arena_off = w.lvl_goff[q0] + LVL_BATCH_FIXED * b;
  unsigned char *base = w.lvl_arena + arena_off;
  uint32_t *rt = reinterpret_cast<uint32_t *>(base + off_round);
  TaskRec *tasks = reinterpret_cast<TaskRec *>(base + off_task);
  uint16_t *eslot = reinterpret_cast<uint16_t *>(base + off_eslot);
  float *ew = reinterpret_cast<float *>(base + off_ew);
  int *gio = reinterpret_cast<int *>(base + off_gio);
  if (tid == 0) {
    BatchHead hd;
    hd.n_genomes = ng; hd.n_slots = nslots; hd.n_rounds = nrounds; hd.n_tasks = ntasks;
    hd.n_chunks = nchunks; hd.off_round = off_round; hd.off_task = off_task;
    hd.off_eslot = off_eslot; hd.off_gio = off_gio; hd.prog_bytes = bytes; hd.off_ew = off_ew;
    hd.pad = 0;
    *reinterpret_cast<BatchHead *>(base) = hd;
    BatchLoc loc;
    loc.off = arena_off;
    loc.bytes = bytes;
    loc.head = off_task;
    loc.pad = 0;
    w.lvl_loc[b] = loc;
    // round table (same walk as above)
    int R = 0, in = 0, cur = -1;
    for (int j = 0; j < ntasks; ++j) {
      const int nc = cnt[j + 1] - cnt[j];
      if (new_round(j, cur, in, nc)) {
        rt[R++] = uint32_t(j) | (uint32_t(cnt[j]) << 16);
        in = 0;
        cur = int(keys[j] >> 33);
      }
      in += nc;
    }
    rt[R] = uint32_t(ntasks) | (uint32_t(nchunks) << 16);
  }
  // task records and their padded edge chunks
  for (int j = tid; j < ntasks; j += T) {
    const uint64_t key = keys[j];
    const int k = int((key >> 10) & 63u), p = int(key & 1023u);
    const NodeRec n = w.knode[g_noff[k] + p];
    const int c = meta_cnt(n.meta), agg = meta_agg(n.meta);
    TaskRec t;
    t.bias = n.bias;
    // mean: fold 1/n into the response, so that the round combines partial
    // sums the same way for sum and mean (r (s / n) -> (r / n) s, both
    // rounded once)
    t.resp = (agg == NEAT_AGG_MEAN && c > 0) ? n.resp / float(c) : n.resp;
    t.chunk = uint32_t(cnt[j]);
    t.meta = task_meta(c, meta_act(n.meta), agg, g_slot[k] + p);
    tasks[j] = t;
    const EdgeRec *src = w.kedge + g_eoff[k] + n.in_begin;
    const int e0 = 4 * cnt[j], e1 = 4 * cnt[j + 1];
    for (int e = 0; e < e1 - e0; ++e) {
      if (e < c) {
        const EdgeRec er = src[e];
        const uint32_t tag = (e & 3) == 0 ? uint32_t(agg) << LVL_SLOT_BITS : 0u;
        eslot[e0 + e] = uint16_t(uint32_t(g_slot[k] + int(er.src)) | tag);
        ew[e0 + e] = er.w;
      } else {
        eslot[e0 + e] = 0xffffu;
        ew[e0 + e] = 0.0f;
      }
    }
  }
  // genome ids and input / output slots (-1 for a rejected genome)
  for (int i = tid; i < ng * G; i += T) {
    const int k = i / G, f = i - k * G;
    const int g = g_id[k];
    int val;
    if (f == 0) val = g;
    else if (g_V[k] == 0) val = -1;
    else val = g_slot[k] + w.pio[size_t(g) * (I + O) + (f - 1)];
    gio[i] = val;
  }
}

// ---------------------------------------------------------------------------
// Bounded mbarrier wait on a phase parity: at most `polls` try_wait polls
// (none for polls <= 0).  Returns whether the phase completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, int polls) {
  uint32_t done = 0;
  for (int it = 0; it < polls && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
  }
  return done != 0;
}
constexpr int DRAIN_POLLS = 1 << 22;

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, int bytes, uint32_t mbar) {
  for (int off = 0; off < bytes; off += 16384) {
    const int n = min(16384, bytes - off);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst + uint32_t(off)),
        "l"(static_cast<const unsigned char *>(src) + off), "r"(n), "r"(mbar)
        : "memory");
  }
}

// Shared-memory accesses of the rounds as explicit shared-space instructions
// (the batch arrays are addressed through offsets read at run time; generic
// accesses to them measured slower).  Volatile: never moved across the
// round's __syncwarp.
__device__ __forceinline__ unsigned sh_addr(const void *p) {
  return unsigned(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ float lds_f32(const float *p) {
  float r;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(sh_addr(p)) : "memory");
  return r;
}
__device__ __forceinline__ float4 lds_f32x4(const float4 *p) {
  float4 r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "r"(sh_addr(p))
               : "memory");
  return r;
}
__device__ __forceinline__ uint2 lds_u32x2(const uint2 *p) {
  uint2 r;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(sh_addr(p)) : "memory");
  return r;
}
__device__ __forceinline__ uint32_t lds_u32(const uint32_t *p) {
  uint32_t r;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(sh_addr(p)) : "memory");
  return r;
}
__device__ __forceinline__ TaskRec lds_task(const TaskRec *p) {
  uint32_t b, r, c, m;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(b), "=r"(r), "=r"(c), "=r"(m)
               : "r"(sh_addr(p))
               : "memory");
  TaskRec t;
  t.bias = __uint_as_float(b);
  t.resp = __uint_as_float(r);
  t.chunk = c;
  t.meta = m;
  return t;
}
__device__ __forceinline__ void sts_f32(float *p, float x) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(sh_addr(p)), "f"(x) : "memory");
}

// Activation of one value per lane, each function present among the warp's
// lanes evaluated once (warp-uniform branches; lanes of other activations
// keep their own result).  Called by all 32 lanes.  The same functions as
// act_apply: sigmoid 1 / (1 + e^-z) and gaussian e^(-z^2) share one expf.
__device__ __forceinline__ float act_warp(int a, float z) {
  constexpr unsigned full = 0xffffffffu;
  float y = z;  // identity
  if (a == NEAT_ACT_RELU) y = fmaxf(z, 0.0f);
  if (a == NEAT_ACT_ABS) y = fabsf(z);
  if (__any_sync(full, a == NEAT_ACT_SIGMOID || a == NEAT_ACT_GAUSSIAN)) {
    const float e = expf(a == NEAT_ACT_SIGMOID ? -z : -(z * z));
    if (a == NEAT_ACT_SIGMOID) y = 1.0f / (1.0f + e);
    if (a == NEAT_ACT_GAUSSIAN) y = e;
  }
  if (__any_sync(full, a == NEAT_ACT_TANH)) {
    const float t = tanhf(z);
    if (a == NEAT_ACT_TANH) y = t;
  }
  if (__any_sync(full, a == NEAT_ACT_SIN)) {
    const float s = sinf(z);
    if (a == NEAT_ACT_SIN) y = s;
  }
  return y;
}

// One round of a warp's batch: tasks [t0, t1), chunks [c0, c1).
//  chunk pass: one lane per (4-edge chunk, sample): the partial of the
//    chunk's aggregation (sum: fma chain; product; max, NaN-ignoring) over
//    its real edges into part[];
//  node pass: one lane per (task, sample): the task's partials combined with
//    its aggregation (a mean's 1/n is folded into its response), then
//    v[slot] = act(b + r a).
template <int ST>
__device__ __forceinline__ void warp_round(const TaskRec *__restrict__ tasks,
                                           const uint2 *__restrict__ eslot,
                                           const float4 *__restrict__ ew, float *part, float *v,
                                           int t0, int t1, int c0, int c1, int lane) {
  const int na = (c1 - c0) * ST;
  for (int it = lane; it < na; it += 32) {
    const int c = c0 + (ST == 1 ? it : it / ST);
    const int s = ST == 1 ? 0 : it % ST;
    const uint2 sl = lds_u32x2(eslot + c);
    const float4 w4 = lds_f32x4(ew + c);
    const uint32_t e0 = sl.x & 0xffffu;
    const uint32_t q[4] = {e0 & (LVL_MAX_SLOTS - 1u), sl.x >> 16, sl.y & 0xffffu, sl.y >> 16};
    const float wq[4] = {w4.x, w4.y, w4.z, w4.w};
    const int agg = int(e0 >> LVL_SLOT_BITS);
    float sum = 0.0f, prod = 1.0f, mx = qnan();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k == 0 || q[k] != 0xffffu) {
        const float x = lds_f32(v + q[k] * ST + s);
        sum = fmaf(wq[k], x, sum);
        const float tv = wq[k] * x;
        prod *= tv;
        mx = fmaxf(mx, tv);
      }
    }
    sts_f32(part + it, agg == NEAT_AGG_PRODUCT ? prod : (agg == NEAT_AGG_MAX ? mx : sum));
  }
  __syncwarp();
  const int nt = (t1 - t0) * ST;
  for (int base = 0; base < nt; base += 32) {
    const int it = base + lane;
    int act = NEAT_ACT_IDENTITY, dst = -1;
    float z = 0.0f;
    if (it < nt) {
      const int t = t0 + (ST == 1 ? it : it / ST);
      const int s = ST == 1 ? 0 : it % ST;
      const TaskRec tk = lds_task(tasks + t);
      const int cnt = task_cnt(tk.meta), agg = task_agg(tk.meta);
      const int pc = int(tk.chunk) - c0, nc = (cnt + 3) >> 2;
      float sum = 0.0f, prod = 1.0f, mx = qnan();
      // partials four at a time: the loads of a group are in flight together
      for (int k = 0; k < nc; k += 4) {
        float p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = k + u < nc ? lds_f32(part + (pc + k + u) * ST + s) : 0.0f;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (k + u < nc) {
            sum += p[u];
            prod *= p[u];
            mx = fmaxf(mx, p[u]);
          }
      }
      // empty aggregation: 0 for every aggregation
      const float a = nc == 0 ? 0.0f
                    : agg == NEAT_AGG_PRODUCT ? prod
                    : agg == NEAT_AGG_MAX ? mx : sum;
      z = fmaf(tk.resp, a, tk.bias);
      act = task_act(tk.meta);
      dst = task_slot(tk.meta) * ST + s;
    }
    const float y = act_warp(act, z);
    if (dst >= 0) sts_f32(v + dst, y);
  }
  __syncwarp();
}

// NaN outputs for the genomes of batch b (read from the queue, not from the
// staged copy) after a staging wait gave up
__device__ void nan_batch_outputs(const Ws &w, int b, int S, float *__restrict__ out, int lane) {
  const int q0 = w.lvl_first[b], q1 = w.lvl_first[b + 1];
  const int per = S * w.O;
  for (int it = lane; it < (q1 - q0) * per; it += 32) {
    const int k = it / per, r = it - k * per;
    out[size_t(w.qlvl[q0 + k]) * per + r] = qnan();
  }
}

constexpr int LVL_MAX_WARPS = 8;

template <int ST>
__global__ void __launch_bounds__(32 * LVL_MAX_WARPS) k_forward_lvl(
    Ws w, const float *__restrict__ inputs, int64_t stride, int S, float *__restrict__ out,
    int warp_bytes, int vals_bytes, int polls) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2 * LVL_MAX_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int I = w.I, O = w.O, G = 1 + I + O;
  const int cap = w.lvl_budget;
  unsigned char *buf = sm + size_t(wid) * warp_bytes;
  float *v = reinterpret_cast<float *>(buf + cap);
  float *part = reinterpret_cast<float *>(buf + cap + vals_bytes);
  const uint32_t mb0 = uint32_t(__cvta_generic_to_shared(&mbar[2 * wid]));
  const uint32_t mb1 = uint32_t(__cvta_generic_to_shared(&mbar[2 * wid + 1]));
  const uint32_t buf_a = uint32_t(__cvta_generic_to_shared(buf));
  const int nbatch = int(w.counters[CTR_NBATCH]);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // the step's inputs towards L2, one 128-byte line per thread of the grid
  // (every address inside the inputs): the batches' input loads then hit L2
  if (stride >= 0) {
    const size_t total = size_t(w.P - 1) * size_t(stride) + size_t(S) * I;
    const size_t lines = (total + 31) / 32;
    for (size_t l = size_t(blockIdx.x) * blockDim.x + threadIdx.x; l < lines;
         l += size_t(gridDim.x) * blockDim.x)
      asm volatile("prefetch.L2 [%0];" ::"l"(inputs + l * 32));
  }
  const int nwarps = gridDim.x * nw;
  uint32_t parity = 0;
  // the first batch of each warp is its own index, later ones are claimed in
  // order of finishing: no contended atomic at the start of the launch
  int b = blockIdx.x * nw + wid;
  while (b < nbatch) {
    const BatchLoc loc = w.lvl_loc[b];
    const unsigned char *src = w.lvl_arena + loc.off;
    if (lane == 0) {
      // the head part (up to off_task) and the rest, each on its own mbarrier;
      // the previous batch's reads of the buffer are ordered before the copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb0),
                   "r"(loc.head)
                   : "memory");
      bulk_g2s(buf_a, src, loc.head, mb0);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb1),
                   "r"(loc.bytes - loc.head)
                   : "memory");
      bulk_g2s(buf_a + uint32_t(loc.head), src + loc.head, loc.bytes - loc.head, mb1);
    }
    bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(mb0, parity, polls));
    if (ok) {
      const BatchHead hd = *reinterpret_cast<const BatchHead *>(buf);
      const int *gio = reinterpret_cast<const int *>(buf + hd.off_gio);
      const uint32_t *rt = reinterpret_cast<const uint32_t *>(buf + hd.off_round);
      const TaskRec *tasks = reinterpret_cast<const TaskRec *>(buf + hd.off_task);
      const uint2 *eslot = reinterpret_cast<const uint2 *>(buf + hd.off_eslot);
      const float4 *ew = reinterpret_cast<const float4 *>(buf + hd.off_ew);
      for (int s0 = 0; s0 < S; s0 += ST) {
        // inputs (for the first tile while tasks and edges are still arriving)
        for (int it = lane; it < hd.n_genomes * I * ST; it += 32) {
          const int s = it % ST, r = it / ST, k = r / I, i = r - k * I;
          const int slot = gio[k * G + 1 + i];
          if (slot < 0) continue;
          const int gs = s0 + s;
          v[slot * ST + s] =
              gs < S ? __ldg(inputs + size_t(gio[k * G]) * stride + size_t(gs) * I + i) : 0.0f;
        }
        if (s0 == 0) ok = __all_sync(0xffffffffu, mbar_wait_bounded(mb1, parity, polls));
        __syncwarp();
        if (!ok) break;
        for (int r = 0; r < hd.n_rounds; ++r) {
          const uint32_t r0 = lds_u32(rt + r), r1 = lds_u32(rt + r + 1);
          warp_round<ST>(tasks, eslot, ew, part, v, int(r0 & 0xffffu), int(r1 & 0xffffu),
                         int(r0 >> 16), int(r1 >> 16), lane);
        }
        for (int it = lane; it < hd.n_genomes * O * ST; it += 32) {
          const int s = it % ST, r = it / ST, k = r / O, j = r - k * O;
          const int gs = s0 + s;
          if (gs >= S) continue;
          const int slot = gio[k * G + 1 + I + j];
          out[(size_t(gio[k * G]) * S + gs) * O + j] = slot < 0 ? qnan() : v[slot * ST + s];
        }
        __syncwarp();
      }
    }
    if (!ok) {
      // a staging wait gave up: report it, let both copies land (bounded)
      // before the buffer is reused, and NaN this batch's outputs
      if (lane == 0) atomicOr(w.counters + CTR_ERR, ERR_TMA_TIMEOUT);
      const bool drained = __all_sync(0xffffffffu, mbar_wait_bounded(mb0, parity, DRAIN_POLLS) &&
                                                       mbar_wait_bounded(mb1, parity, DRAIN_POLLS));
      nan_batch_outputs(w, b, S, out, lane);
      __syncwarp();
      if (!drained) break;  // the buffer may still be written: this warp stops
    }
    parity ^= 1u;
    int nxt = 0;
    if (lane == 0) nxt = nwarps + int(atomicAdd(w.counters + CTR_LVL_ITEM, 1u));
    b = __shfl_sync(0xffffffffu, nxt, 0);
  }
  // the last warp to finish resets the claim counters for the next launch
  if (lane == 0) {
    __threadfence();
    const unsigned t = atomicAdd(w.counters + CTR_LVL_DONE, 1u);
    if (t == unsigned(nwarps) - 1u) {
      atomicExch(w.counters + CTR_LVL_ITEM, 0u);
      atomicExch(w.counters + CTR_LVL_DONE, 0u);
    }
  }
}

}  // namespace

int lvl_tile(int S) { return S >= 4 ? 4 : (S >= 2 ? 2 : 1); }

size_t lvl_vals_bytes(const Ws &w, int st_samples) {
  return (sizeof(float) * size_t(w.lvl_slots) * st_samples + 15) & ~size_t(15);
}

size_t lvl_warp_bytes(const Ws &w, int st_samples) {
  const size_t part = (sizeof(float) * size_t(w.lvl_pcap) * st_samples + 15) & ~size_t(15);
  return (size_t(w.lvl_budget) + lvl_vals_bytes(w, st_samples) + part + 127) & ~size_t(127);
}

cudaError_t launch_lvl_build(const Ws &w, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  k_lvl_plan<<<1, PLAN_THREADS, 0, st>>>(w);
  const size_t smem = 8 * size_t(LVL_MAX_SLOTS) + 4 * size_t(LVL_MAX_SLOTS + 1);
  k_lvl_build<<<w.lvl_max_batches, BLD_THREADS, smem, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_forward_lvl(const Ws &w, const float *inputs, int64_t stride, int S,
                               float *outputs, int warps, int grid, int polls, cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const int ST = lvl_tile(S);
  const int wb = int(lvl_warp_bytes(w, ST)), vb = int(lvl_vals_bytes(w, ST));
  const size_t smem = size_t(wb) * warps;
  const int threads = 32 * warps;
  if (ST == 1)
    k_forward_lvl<1><<<grid, threads, smem, st>>>(w, inputs, stride, S, outputs, wb, vb, polls);
  else if (ST == 2)
    k_forward_lvl<2><<<grid, threads, smem, st>>>(w, inputs, stride, S, outputs, wb, vb, polls);
  else
    k_forward_lvl<4><<<grid, threads, smem, st>>>(w, inputs, stride, S, outputs, wb, vb, polls);
  return cudaGetLastError();
}

cudaError_t lvl_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_forward_lvl<1>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_lvl<2>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_lvl<4>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_lvl_build, bytes);
  return e;
}

int forward_lvl_occupancy(int warps, size_t smem, int st_samples) {
  int n = 0;
  cudaError_t e;
  if (st_samples == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_lvl<1>, 32 * warps, smem);
  else if (st_samples == 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_lvl<2>, 32 * warps, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_lvl<4>, 32 * warps, smem);
  return e == cudaSuccess ? n : 0;
}

}  // namespace neat
