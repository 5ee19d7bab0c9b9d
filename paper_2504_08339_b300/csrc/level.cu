// Level-synchronous batched forward for small sample counts (one or a few
// input vectors per genome, e.g. one observation per rollout step).
//
// With S = 1 a single genome offers only the few independent nodes of one
// layer at a time, so genomes are evaluated in small BATCHES: all their
// layer-r nodes are independent of each other (Sec. 3.3's order only requires
// each node to follow its inputs), so a round evaluates the layer-r nodes of
// every genome in the batch.  Each batch belongs to one warp, which runs the
// rounds with __syncwarp only: a shallow batch never waits for a deep one, and
// no CTA-wide barrier sits in a round.  A round has two passes: one lane per
// 4-edge chunk of incoming connections (the partial of the task's
// aggregation), then one lane per node (combine the partials, bias, response,
// activation), the nodes of mixed activations evaluated side by side without
// divergent branches.
//
// Transform time (k_lvl_plan, k_lvl_build): genomes in layer-sorted queue
// order are cut into batches under a byte budget, and each batch program is
// written contiguously (see BatchHead in neat_internal.cuh).
// Run time (k_forward_lvl): a warp takes its first batch by its index and
// claims the next ones from a counter.  It stages the batch's head part
// (header and I/O slots) into its shared memory with a bulk copy
// (cp.async.bulk, mbarrier completion, bounded wait) and reads the round
// table, task records and edge chunks straight from global memory (L2), each
// round's records one round ahead: the shared memory a warp holds is only its
// head part, its value slots and its chunk partials, so that many warps fit
// on an SM whatever the batch size.
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
// budget, its value slots the slot cap (less the two constant slots), or it
// already holds as many genomes as the head cap allows (at most
// LVL_MAX_GENOMES).
// Runs never share a batch, so the cut is exact and parallel; a run ends with
// one partly filled batch.  Batch b's program sits at arena offset
// goff[first genome of b] + LVL_BATCH_FIXED * b, goff being the prefix of the
// genome byte bounds in queue order.
constexpr int PLAN_THREADS = 1024;

// Populations of at most PLAN_STAGED genomes first stage every genome's
// (byte bound, slots) pair in shared memory, all loads independent, so that
// the runs' sequential cuts read shared memory instead of waiting on two
// dependent global loads a genome.
constexpr int PLAN_STAGED = 20480;

// target > 0 (no budget set by the caller): the budget is the smallest one,
// in steps of LVL_BUDGET_STEP from budget_lo, whose cut gives at most
// `target` batches (the warps resident at once): more batches than warps
// leave some warps a second batch after the rest are done (measured 26 %
// slower on 10,000 genomes at 14 KiB), far fewer leave warps idle and the
// rounds wider.  The batch count does not grow with the budget, so a binary
// search over the same greedy cut finds it.
constexpr int LVL_BUDGET_STEP = 128;

__global__ void __launch_bounds__(PLAN_THREADS) k_lvl_plan(Ws w, int target, int budget_lo) {
  __shared__ long long sb[32];
  __shared__ int sn[32];
  __shared__ int s_count;
  extern __shared__ int2 sgen[];  // [P] (byte bound, slots) when staged
  const int P = w.P, T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int I = w.I, O = w.O, scap = w.lvl_slots - LVL_CONST_SLOTS;
  int cap = w.lvl_budget;
  const int per = max(128, (P + T - 1) / T);
  // genomes per batch: the staged head (header, 4 B per genome id and I/O
  // slot, alignment) fits the warp's head buffer
  const int gmax = min(LVL_MAX_GENOMES,
                       (lvl_head_cap(I, O) - int(sizeof(BatchHead)) - 15) / (4 * (1 + I + O)));
  const int q0 = min(tid * per, P), q1 = min(q0 + per, P);
  auto load = [&](int q) {
    const GenomeHdr h = w.hdr[w.qlvl[q]];
    const bool ok = h.status == 0u;
    // tasks: the evaluated nodes
    return make_int2(lvl_genome_bytes(h.nlive, h.nch, h.L, I, O, ok), ok ? h.V : 0);
  };
  const bool staged = P <= PLAN_STAGED;
  if (staged) {
    for (int q = tid; q < P; q += T) sgen[q] = load(q);
    __syncthreads();
  }
  auto genome = [&](int q, int &pb, int &V) {
    const int2 x = staged ? sgen[q] : load(q);
    pb = x.x;
    V = x.y;
  };
  // batches of the cut at budget B (every thread calls it)
  auto count = [&](int B) {
    int nb = 0, cb = 0, cs = 0, cg = 0;
    for (int q = q0; q < q1; ++q) {
      int pb, V;
      genome(q, pb, V);
      if (cg == 0 || cg == gmax || cb + pb > B || cs + V > scap) {
        ++nb;
        cb = LVL_BATCH_FIXED;
        cs = 0;
        cg = 0;
      }
      cb += pb;
      cs += V;
      ++cg;
    }
    if (tid == 0) s_count = 0;
    __syncthreads();
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, d);
    if (lane == 0 && nb) atomicAdd(&s_count, nb);
    __syncthreads();
    const int c = s_count;
    __syncthreads();
    return c;
  };
  if (target > 0) {
    int lo = (budget_lo + LVL_BUDGET_STEP - 1) / LVL_BUDGET_STEP, hi = LVL_MAX_BUDGET / LVL_BUDGET_STEP;
    while (lo < hi) {  // (uniform over the CTA)
      const int mid = (lo + hi) >> 1;
      if (count(mid * LVL_BUDGET_STEP) <= target) hi = mid;
      else lo = mid + 1;
    }
    cap = lo * LVL_BUDGET_STEP;
  }
  // pass 1: batches and bytes of this thread's run
  int nb = 0;
  long long by = 0;
  {
    int cb = 0, cs = 0, cg = 0;
    for (int q = q0; q < q1; ++q) {
      int pb, V;
      genome(q, pb, V);
      if (cg == 0 || cg == gmax || cb + pb > cap || cs + V > scap) {
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
      if (cg == 0 || cg == gmax || cb + pb > cap || cs + V > scap) {
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
    // the forward's 64-bit claim counter (counters[CTR_LVL_ITEM..+1])
    *reinterpret_cast<unsigned long long *>(w.counters + CTR_LVL_ITEM) = 0ull;
  }
}

// ---------------------------------------------------------------------------
// one CTA per batch: gather, sort and write the batch program
constexpr int BLD_THREADS = 256;

__global__ void __launch_bounds__(BLD_THREADS) k_lvl_build(Ws w) {
  __shared__ int g_id[LVL_MAX_GENOMES + 1], g_V[LVL_MAX_GENOMES + 1];
  __shared__ int g_noff[LVL_MAX_GENOMES + 1], g_eoff[LVL_MAX_GENOMES + 1];
  __shared__ int g_slot[LVL_MAX_GENOMES + 1], g_NL[LVL_MAX_GENOMES + 1];
  __shared__ int s_nslots, s_ntasks, s_nrounds, s_bad;
  __shared__ unsigned s_acts;
  __shared__ uint32_t rsb[LVL_MAX_SLOTS / 32];  // round-start bits of the tasks
  __shared__ int wpre[LVL_MAX_SLOTS / 32];      // round starts before each word
  __shared__ int wbuf[33];
  extern __shared__ __align__(16) unsigned char dsm[];
  // sort keys [pow2(lvl_slots)], chunk offsets [lvl_slots + 1]: a batch holds
  // at most lvl_slots value slots, and so fewer tasks
  uint64_t *keys = reinterpret_cast<uint64_t *>(dsm);
  int *cnt = reinterpret_cast<int *>(dsm + 8 * size_t(pow2_ceil_d(w.lvl_slots)));

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
    g_NL[k] = ok ? h.nlive : 0;
    g_noff[k] = h.node_off;
    g_eoff[k] = h.edge_off;
  }
  __syncthreads();
  if (tid == 0) {
    int s = LVL_CONST_SLOTS, nt = 0;  // slots 0 and 1 hold the constants 0 and 1
    for (int k = 0; k < ng; ++k) {
      g_slot[k] = s;
      s += g_V[k];
      nt += g_NL[k];
    }
    g_slot[ng] = s;
    s_nslots = s;
    s_ntasks = nt;
    s_acts = 0u;
  }
  __syncthreads();
  const int nslots = s_nslots, ntasks = s_ntasks;
  if (nslots > w.lvl_slots) return;  // cannot happen by construction of the cut
  // sort keys over the genome slots (slot i + LVL_CONST_SLOTS)
  const int ngs = nslots - LVL_CONST_SLOTS;
  const int n2 = pow2_ceil_d(max(ngs, 1));
  // task keys: (layer, activation class, act, -cnt, genome, position), the
  // classes ordered exp-family (sigmoid, tanh, gaussian), cheap (identity,
  // relu, abs), sine: a round's first 32 tasks then rarely hold a sine and
  // the next 32 rarely an exp-family node, and the forward evaluates only
  // the functions a 32-task pass holds.  Inputs and the nodes no output
  // depends on sort last (they are not tasks).
  for (int i = tid; i < n2; i += T) {
    uint64_t key = ~0ull;
    if (i < ngs) {
      int k = 0;
      while (g_slot[k + 1] <= i + LVL_CONST_SLOTS) ++k;
      const int p = i + LVL_CONST_SLOTS - g_slot[k];
      const NodeRec n = w.knode[g_noff[k] + p];
      if (!(n.meta & (META_INPUT | META_DEAD))) {
        const uint64_t lay = uint64_t(w.player[size_t(g_id[k]) * w.N + p]);
        const int a = meta_act(n.meta);
        const uint64_t cls = ((ACT_BIT_EXP >> a) & 1u) ? 0u : (a == NEAT_ACT_SIN ? 2u : 1u);
        key = (lay << 35) | (cls << 33) | (uint64_t(a) << 30) |
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
  // task never does: pcap >= the chunks of a node's in-degree).  Round starts
  // are bits of rsb: every layer start, and the splits that the thread owning
  // a layer's start finds by walking that layer (layers in parallel); a
  // round's index is the number of starts before it (word prefix + popc).
  for (int i = tid; i < LVL_MAX_SLOTS / 32; i += T) rsb[i] = 0u;
  __syncthreads();
  auto lay_of = [&](int j) { return int(keys[j] >> 35); };
  for (int j = tid; j < ntasks; j += T) {
    if (j > 0 && lay_of(j) == lay_of(j - 1)) continue;
    atomicOr(&rsb[j >> 5], 1u << (j & 31));
    const int l = lay_of(j);
    int in = cnt[j + 1] - cnt[j];
    for (int k = j + 1; k < ntasks && lay_of(k) == l; ++k) {
      const int nc = cnt[k + 1] - cnt[k];
      if (in + nc > pcap) {
        atomicOr(&rsb[k >> 5], 1u << (k & 31));
        in = 0;
      }
      in += nc;
    }
  }
  __syncthreads();
  const int nwords = (ntasks + 31) >> 5;
  if (tid < 32) {  // exclusive prefix of the words' start counts (4 words a lane)
    int c[4], tot = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int wi = 4 * tid + q;
      c[q] = wi < nwords ? __popc(rsb[wi]) : 0;
      tot += c[q];
    }
    int x = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (tid >= d) x += y;
    }
    int base = x - tot;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      wpre[4 * tid + q] = base;
      base += c[q];
    }
    if (tid == 31) s_nrounds = x;
  }
  __syncthreads();
  const int nrounds = s_nrounds;
  // program layout: head part (header, gio), then round table, tasks and edges
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
    hd.act_mask = 0u;  // set once the task records are written
    *reinterpret_cast<BatchHead *>(base) = hd;
    BatchLoc loc;
    loc.off = arena_off;
    loc.bytes = bytes;
    loc.head = off_round;
    loc.pad = 0;
    w.lvl_loc[b] = loc;
    rt[nrounds] = uint32_t(ntasks) | (uint32_t(nchunks) << 16);
  }
  // round table: the first task and chunk of every round
  for (int j = tid; j < ntasks; j += T) {
    const uint32_t word = rsb[j >> 5], bit = 1u << (j & 31);
    if (word & bit)
      rt[wpre[j >> 5] + __popc(word & (bit - 1u))] = uint32_t(j) | (uint32_t(cnt[j]) << 16);
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
    atomicOr(&s_acts, 1u << meta_act(n.meta));
    const EdgeRec *src = w.kedge + g_eoff[k] + n.in_begin;
    const int e0 = 4 * cnt[j], e1 = 4 * cnt[j + 1];
    for (int e = 0; e < e1 - e0; ++e) {
      const uint32_t tag = (e & 3) == 0 ? uint32_t(agg) << LVL_SLOT_BITS : 0u;
      uint32_t slot;
      float wt;
      if (e < c) {
        const EdgeRec er = src[e];
        slot = uint32_t(g_slot[k] + int(er.src));
        wt = er.w;
      } else if (agg == NEAT_AGG_PRODUCT) {  // w 1 on the constant 1: a factor 1
        slot = 1u;
        wt = 1.0f;
      } else if (agg == NEAT_AGG_MAX) {      // the chunk's first edge again
        const EdgeRec er = src[e & ~3];
        slot = uint32_t(g_slot[k] + int(er.src));
        wt = er.w;
      } else {                               // w 0 on the constant 0: a term 0
        slot = 0u;
        wt = 0.0f;
      }
      eslot[e0 + e] = uint16_t(slot | tag);
      ew[e0 + e] = wt;
    }
  }
  __syncthreads();
  if (tid == 0) reinterpret_cast<BatchHead *>(base)->act_mask = s_acts;
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
// on 32-bit shared addresses (no generic pointer arithmetic or address
// conversion per access).  Volatile: never moved across the round's
// __syncwarp.
__device__ __forceinline__ unsigned sh_addr(const void *p) {
  return unsigned(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ float lds_f32_a(uint32_t a) {
  float r;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(a) : "memory");
  return r;
}
__device__ __forceinline__ void sts_f32_a(uint32_t a, float x) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(x) : "memory");
}

// Activation of one value per lane, the lanes holding nodes of mixed
// activations.  `mask` (bit a: some task of the pass, or of a superset such
// as the whole batch, has activation a; the same on every lane) names the
// evaluations needed: one exponential (and e^x - 1) per lane
// serves sigmoid, tanh and gaussian (act_exp_arg), one reciprocal sigmoid and
// tanh, one sine the sin nodes; each is evaluated on every lane and the
// lane's result selected, so no branch diverges (but for sine arguments
// beyond 6.5e6, which take sinf).
__device__ __forceinline__ float act_lanes(int a, float z, uint32_t mask) {
  float y = sel_eq<NEAT_ACT_RELU>(a, fmaxf(z, 0.0f), z);
  y = sel_eq<NEAT_ACT_ABS>(a, fabsf(z), y);
  if (mask & ACT_BIT_EXP) {
    float e, m;  // e^x and e^x - 1 of the lane's argument
    am::exp_expm1_cw(act_exp_arg(a, z), e, m);
    const float q = am::rcp_nr(2.0f + m);  // 1 / (1 + e^x)
    y = sel_eq<NEAT_ACT_SIGMOID>(a, q, y);
    y = sel_eq<NEAT_ACT_GAUSSIAN>(a, e, y);
    // tanh |z| = -(e^{-2|z|} - 1) / (1 + e^{-2|z|})
    if (mask & (1u << NEAT_ACT_TANH)) y = sel_eq<NEAT_ACT_TANH>(a, copysignf(-m * q, z), y);
  }
  if (mask & ACT_BIT_SIN) {
    const float zs = sel_eq<NEAT_ACT_SIN>(a, z, 0.0f);
    float sn = am::sin_cw(zs);
    if (fabsf(zs) > am::SIN_ARG_MAX) sn = sinf(zs);  // rare
    y = sel_eq<NEAT_ACT_SIN>(a, sn, y);
  }
  return y;
}

// A batch program's arrays: the round table, task records and edge chunks in
// global memory (read-only for the kernel, L2-resident within a rollout), the
// value slots and chunk partials as shared addresses.
struct BatchArrays {
  const uint32_t *rt;
  const uint4 *tasks;
  const uint2 *eslot;
  const uint4 *ew;
  uint32_t part, v;  // shared addresses
};
struct ChunkRec {
  uint2 sl;
  uint4 w;  // the four weights (bits)
};
__device__ __forceinline__ ChunkRec ld_chunk(const BatchArrays &ba, int c) {
  ChunkRec r;
  r.sl = __ldg(ba.eslot + c);
  r.w = __ldg(ba.ew + c);
  return r;
}
__device__ __forceinline__ TaskRec ld_task(const BatchArrays &ba, int t) {
  const uint4 q = __ldg(ba.tasks + t);
  TaskRec r;
  r.bias = __uint_as_float(q.x);
  r.resp = __uint_as_float(q.y);
  r.chunk = q.z;
  r.meta = q.w;
  return r;
}

// partial of one chunk for sample s of ST: the edges' terms folded with the
// task's aggregation (sum: fma chain; product; max, NaN-ignoring; padding
// edges are neutral for it, so every lane runs the same instructions)
template <int ST>
__device__ __forceinline__ float chunk_partial(const ChunkRec &r, uint32_t v, int s) {
  const int agg = int((r.sl.x >> LVL_SLOT_BITS) & 3u);
  const uint32_t vs = v + 4u * uint32_t(s);
  const float x0 = lds_f32_a(vs + 4u * ST * (r.sl.x & (LVL_MAX_SLOTS - 1u)));
  const float x1 = lds_f32_a(vs + 4u * ST * (r.sl.x >> 16));
  const float x2 = lds_f32_a(vs + 4u * ST * (r.sl.y & 0xffffu));
  const float x3 = lds_f32_a(vs + 4u * ST * (r.sl.y >> 16));
  const float w0 = __uint_as_float(r.w.x), w1 = __uint_as_float(r.w.y),
              w2 = __uint_as_float(r.w.z), w3 = __uint_as_float(r.w.w);
  const float sum = fmaf(w3, x3, fmaf(w2, x2, fmaf(w1, x1, w0 * x0)));
  const float p0 = w0 * x0, p1 = w1 * x1, p2 = w2 * x2, p3 = w3 * x3;
  const float prod = ((p0 * p1) * p2) * p3;
  const float mx = fmaxf(fmaxf(fmaxf(p0, p1), p2), p3);
  return sel_eq<NEAT_AGG_PRODUCT>(agg, prod, sel_eq<NEAT_AGG_MAX>(agg, mx, sum));
}

// aggregate of one task from its chunk partials (sample s of ST): the first
// two partials (nc <= 2 for three tasks in four) with the second masked out
// when absent, the rest (in-degrees above 8) in a loop.  Index pc + 1 stays
// inside the partial buffer (it holds the round's chunks plus 4, per sample).
template <int ST>
__device__ __forceinline__ float task_aggregate(const TaskRec &tk, uint32_t part, int c0, int s) {
  const int cnt = task_cnt(tk.meta), agg = task_agg(tk.meta);
  const int nc = (cnt + 3) >> 2;
  const uint32_t pa = part + 4u * uint32_t((int(tk.chunk) - c0) * ST + s);
  const float p0 = lds_f32_a(pa), p1 = lds_f32_a(pa + 4u * ST);
  const bool two = nc >= 2;
  float sum = p0 + sel_if(two, p1, 0.0f);
  float prod = p0 * sel_if(two, p1, 1.0f);
  float mx = fmaxf(p0, sel_if(two, p1, qnan()));
  for (int k = 2; k < nc; ++k) {
    const float p = lds_f32_a(pa + 4u * uint32_t(k * ST));
    sum += p;
    prod *= p;
    mx = fmaxf(mx, p);
  }
  // empty aggregation: 0 for every aggregation
  return sel_if(nc == 0, 0.0f,
                sel_eq<NEAT_AGG_PRODUCT>(agg, prod, sel_eq<NEAT_AGG_MAX>(agg, mx, sum)));
}

// One round of a warp's batch, ST samples per lane item: tasks [t0, t1),
// chunks [c0, c1), records read as they are needed (the form for several
// samples per genome, where a round's work covers ST samples).
//  chunk pass: one lane per (4-edge chunk, sample) into part[];
//  node pass: one lane per (task, sample): the task's partials combined with
//    its aggregation (a mean's 1/n is folded into its response), then
//    v[slot] = act(b + r a); lanes past the round's tasks evaluate the last
//    task again and store nothing.
template <int ST>
__device__ __forceinline__ void warp_round(const BatchArrays &ba, int t0, int t1, int c0, int c1,
                                           int lane, uint32_t mask) {
  const int na = (c1 - c0) * ST;
  for (int it = lane; it < na; it += 32) {
    const int c = c0 + it / ST, s = it % ST;
    sts_f32_a(ba.part + 4u * uint32_t(it), chunk_partial<ST>(ld_chunk(ba, c), ba.v, s));
  }
  __syncwarp();
  const int nt = (t1 - t0) * ST;
  for (int base = 0; base < nt; base += 32) {
    const int it = min(base + lane, nt - 1);
    const int t = t0 + it / ST, s = it % ST;
    const TaskRec tk = ld_task(ba, t);
    const float y = act_lanes(task_act(tk.meta),
                              fmaf(tk.resp, task_aggregate<ST>(tk, ba.part, c0, s), tk.bias), mask);
    if (base + lane < nt) sts_f32_a(ba.v + 4u * uint32_t(task_slot(tk.meta) * ST + s), y);
  }
  __syncwarp();
}

// ---- one sample per genome (the rollout step).  Round r's records (the
// lane's chunk c0 + lane and task t0 + lane, and chunk c0 + lane + 32 / task
// t0 + lane + 32 when the round has more than 32; indices clamped to the
// round, the extra lanes store nothing) are loaded at the start of round
// r - 1, the round-table entries three rounds ahead, so that the L2 latency
// hides under a round.  Rounds beyond 64 chunks or 64 tasks take the rest in
// a loop.  The loop runs two rounds a trip with two record sets, so that no
// record is copied between rounds.
struct RoundRecs {
  uint32_t ra, rb;  // the round's bounds and the next one's
  ChunkRec ca, cb;
  TaskRec ta, tb;
};

__device__ __forceinline__ void load_round(const BatchArrays &ba, uint32_t ra, uint32_t rb,
                                           int lane, RoundRecs &x) {
  const int t0 = int(ra & 0xffffu), t1 = int(rb & 0xffffu), c0 = int(ra >> 16), c1 = int(rb >> 16);
  x.ra = ra;
  x.rb = rb;
  x.ca = ld_chunk(ba, min(c0 + lane, max(c1 - 1, c0)));
  x.ta = ld_task(ba, min(t0 + lane, max(t1 - 1, t0)));
  if (c1 - c0 > 32) x.cb = ld_chunk(ba, min(c0 + lane + 32, c1 - 1));
  if (t1 - t0 > 32) x.tb = ld_task(ba, min(t0 + lane + 32, t1 - 1));
}

// one round from its records `x`; first loads the records of the next round
// (bounds x.rb, rc) into `nx` when there is one (r + 1 < nr); `rq` holds the
// round-table entries of rounds r + 2 and r + 3 (shifted as rounds go)
__device__ __forceinline__ void one_round(const BatchArrays &ba, int r, int nr, int lane,
                                          const RoundRecs &x, RoundRecs &nx, uint32_t (&rq)[2]) {
  const int t0 = int(x.ra & 0xffffu), t1 = int(x.rb & 0xffffu);
  const int c0 = int(x.ra >> 16), c1 = int(x.rb >> 16);
  const int na = c1 - c0, nt = t1 - t0;
  const uint32_t rc = rq[0];
  rq[0] = rq[1];
  rq[1] = r + 4 <= nr ? __ldg(ba.rt + r + 4) : rq[1];
  if (r + 1 < nr) load_round(ba, x.rb, rc, lane, nx);
  const uint32_t part_l = ba.part + 4u * uint32_t(lane);
  // chunk pass
  if (na > 0) {
    const float pa = chunk_partial<1>(x.ca, ba.v, 0);
    if (na > 32) {
      const float pb = chunk_partial<1>(x.cb, ba.v, 0);
      if (lane + 32 < na) sts_f32_a(part_l + 128u, pb);
      for (int it = lane + 64; it < na; it += 32)
        sts_f32_a(ba.part + 4u * uint32_t(it), chunk_partial<1>(ld_chunk(ba, c0 + it), ba.v, 0));
    }
    if (lane < na) sts_f32_a(part_l, pa);
  }
  __syncwarp();
  // node pass: a 32-task pass evaluates only the activation functions its
  // own tasks hold (a warp OR of their activation bits; lanes past the round
  // repeat its last task)
  const int aa = task_act(x.ta.meta);
  const float za = fmaf(x.ta.resp, task_aggregate<1>(x.ta, ba.part, c0, 0), x.ta.bias);
  const uint32_t ma = __reduce_or_sync(0xffffffffu, 1u << aa);
  if (nt > 32) {
    const int ab = task_act(x.tb.meta);
    const float zb = fmaf(x.tb.resp, task_aggregate<1>(x.tb, ba.part, c0, 0), x.tb.bias);
    const uint32_t mb = __reduce_or_sync(0xffffffffu, 1u << ab);
    const float ya = act_lanes(aa, za, ma);
    const float yb = act_lanes(ab, zb, mb);
    if (lane + 32 < nt) sts_f32_a(ba.v + 4u * uint32_t(task_slot(x.tb.meta)), yb);
    sts_f32_a(ba.v + 4u * uint32_t(task_slot(x.ta.meta)), ya);
    // (warp-uniform trip count: act_lanes is called by all 32 lanes)
    for (int base = 64; base < nt; base += 32) {
      const TaskRec tk = ld_task(ba, t0 + min(base + lane, nt - 1));
      const int a = task_act(tk.meta);
      const float y = act_lanes(a, fmaf(tk.resp, task_aggregate<1>(tk, ba.part, c0, 0), tk.bias),
                                __reduce_or_sync(0xffffffffu, 1u << a));
      if (base + lane < nt) sts_f32_a(ba.v + 4u * uint32_t(task_slot(tk.meta)), y);
    }
  } else {
    const float ya = act_lanes(aa, za, ma);
    if (lane < nt) sts_f32_a(ba.v + 4u * uint32_t(task_slot(x.ta.meta)), ya);
  }
  __syncwarp();
}

// all rounds of a batch for one sample; the next batch is claimed when
// round claim_at starts
// the first round's records and the round-table entries of rounds 2 and 3,
// loaded before the batch's staging and input waits
__device__ __forceinline__ void first_round(const BatchArrays &ba, int nr, int lane, RoundRecs &x0,
                                            uint32_t (&rq)[2]) {
  rq[0] = nr >= 2 ? __ldg(ba.rt + 2) : 0u;
  rq[1] = nr >= 3 ? __ldg(ba.rt + 3) : 0u;
  if (nr > 0) load_round(ba, __ldg(ba.rt), __ldg(ba.rt + 1), lane, x0);
}

__device__ __forceinline__ void run_rounds_st1(const BatchArrays &ba, int nr, int lane, int claim_at,
                                               unsigned long long *claim, unsigned long long &old,
                                               bool &claimed, RoundRecs &x0, uint32_t (&rq)[2]) {
  if (nr <= 0) return;
  RoundRecs x1;
  for (int r = 0; r < nr; r += 2) {
    if (r >= claim_at && !claimed) {  // the next batch, a few rounds before this one ends
      if (lane == 0) old = atomicAdd(claim, 1ull);
      claimed = true;
    }
    one_round(ba, r, nr, lane, x0, x1, rq);
    if (r + 1 < nr) one_round(ba, r + 1, nr, lane, x1, x0, rq);
  }
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
constexpr int IN_FLIGHT = 8;  // input loads a lane issues before storing them

// (launch bound: two CTAs of 8 warps per SM, at most 128 registers a thread;
// a 64-register cap spilled the rounds, and above 128 only 12 warps fit)
template <int ST>
//
// pdl (the launch follows a forward of the same batches in its stream, with
// programmatic serialization): the CTAs may start while the previous launch's
// last warps still run, on the SMs it has left; they let the next launch do
// the same at once, stage their first batch's head (batch programs are not
// written by a forward), and wait for the previous grid (griddepcontrol.wait:
// its completion and memory) before reading inputs, claiming batches or
// writing anything.
__global__ void __launch_bounds__(32 * LVL_MAX_WARPS, 2) k_forward_lvl(
    Ws w, const float *__restrict__ inputs, int64_t stride, int S, float *__restrict__ out,
    int warp_bytes, int vals_bytes, int polls, int pdl) {
  if (pdl) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[LVL_MAX_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int I = w.I, O = w.O, G = 1 + I + O;
  const int hcap = lvl_head_cap(I, O);
  unsigned char *head = sm + size_t(wid) * warp_bytes;
  float *v = reinterpret_cast<float *>(head + hcap);
  const uint32_t v_a = sh_addr(v), part_a = sh_addr(head + hcap + vals_bytes);
  const uint32_t mb = uint32_t(__cvta_generic_to_shared(&mbar[wid]));
  const uint32_t head_a = uint32_t(__cvta_generic_to_shared(head));
  const int nbatch = int(w.counters[CTR_NBATCH]);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
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
  // lane walks of the (genome k, input i / output j, sample s) items, item
  // it = (k * I + i) * ST + s for it = lane, lane + 32, ...: ST divides 32,
  // so s = lane % ST throughout and (k, i) advance by 32 / ST items a step
  // (one division per launch instead of one per item)
  constexpr int STEP = 32 / ST;
  const int s_l = lane % ST, r_l = lane / ST;
  const int ki0 = r_l / I, ii0 = r_l % I, dki = STEP / I, dii = STEP % I;
  const int ko0 = r_l / O, jo0 = r_l % O, dko = STEP / O, djo = STEP % O;
  uint32_t parity = 0;
  // Batches: warp w starts with batch w; each warp claims its next batch
  // (a few rounds before the current one ends, so the atomic's latency hides
  // under the last rounds) from a 64-bit epoch counter that the transform
  // zeroes.  Every launch makes exactly nbatch claims (one per batch
  // processed: the successful ones plus one failed claim per warp that had a
  // first batch), so claim index = counter mod nbatch and nothing is reset at
  // the end.
  unsigned long long *claim = reinterpret_cast<unsigned long long *>(w.counters + CTR_LVL_ITEM);
  bool broken = false;  // a drain wait gave up: the buffer may still be written
  int b = blockIdx.x * nw + wid;
  auto next_batch = [&](unsigned long long old) {
    const int n = lane == 0 ? nwarps + int(old % (unsigned long long)nbatch) : 0;
    return __shfl_sync(0xffffffffu, n, 0);
  };
  while (b < nbatch) {
    unsigned long long old = 0;
    bool claimed = false;
    if (broken) {  // keep the claim count: NaN the batch without staging it
      if (lane == 0) old = atomicAdd(claim, 1ull);
      nan_batch_outputs(w, b, S, out, lane);
      __syncwarp();
      b = next_batch(old);
      continue;
    }
    const BatchLoc loc = w.lvl_loc[b];
    const unsigned char *src = w.lvl_arena + loc.off;
    if (lane == 0) {
      // the previous batch's reads of the head buffer are ordered before the copy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb),
                   "r"(loc.head)
                   : "memory");
      bulk_g2s(head_a, src, loc.head, mb);
    }
    // the round table's first entries and the batch's counts come from global
    // memory while the head is in flight
    const BatchHead hg = *reinterpret_cast<const BatchHead *>(src);
    const BatchArrays ba{reinterpret_cast<const uint32_t *>(src + hg.off_round),
                         reinterpret_cast<const uint4 *>(src + hg.off_task),
                         reinterpret_cast<const uint2 *>(src + hg.off_eslot),
                         reinterpret_cast<const uint4 *>(src + hg.off_ew), part_a, v_a};
    // (one sample per genome: the first round's records load during the waits)
    RoundRecs x0;
    uint32_t rq[2];
    if constexpr (ST == 1) first_round(ba, hg.n_rounds, lane, x0, rq);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(mb, parity, polls));
    if (pdl) {  // (once: the first batch; later ones come after it)
      asm volatile("griddepcontrol.wait;" ::: "memory");
      pdl = 0;
    }
    if (ok) {
      const int *gio = reinterpret_cast<const int *>(head + hg.off_gio);
      if (lane < 2 * ST) v[lane] = lane < ST ? 0.0f : 1.0f;  // the constant slots 0 and 1
      for (int s0 = 0; s0 < S; s0 += ST) {
        // the lane's items in groups of IN_FLIGHT: all of a group's loads are
        // issued before its stores, so their L2 latencies overlap
        const int n_in = hg.n_genomes * I * ST;
        for (int it = lane, k = ki0, i = ii0; it < n_in;) {
          float xv[IN_FLIGHT];
          int sl[IN_FLIGHT];
#pragma unroll
          for (int u = 0; u < IN_FLIGHT; ++u) {
            sl[u] = -1;
            xv[u] = 0.0f;
            if (it < n_in) {
              const int gs = s0 + s_l;
              sl[u] = gio[k * G + 1 + i];
              if (sl[u] >= 0 && gs < S)
                xv[u] = __ldg(inputs + size_t(gio[k * G]) * stride + size_t(gs) * I + i);
            }
            it += 32;
            k += dki;
            i += dii;
            if (i >= I) { i -= I; ++k; }
          }
#pragma unroll
          for (int u = 0; u < IN_FLIGHT; ++u)
            if (sl[u] >= 0) v[sl[u] * ST + s_l] = xv[u];
        }
        __syncwarp();
        if constexpr (ST == 1) {
          run_rounds_st1(ba, hg.n_rounds, lane, max(hg.n_rounds - 3, 0), claim, old, claimed,
                         x0, rq);
        } else {
          for (int r = 0; r < hg.n_rounds; ++r) {
            const uint32_t r0 = __ldg(ba.rt + r), r1 = __ldg(ba.rt + r + 1);
            warp_round<ST>(ba, int(r0 & 0xffffu), int(r1 & 0xffffu), int(r0 >> 16),
                           int(r1 >> 16), lane, hg.act_mask);
          }
        }
        for (int it = lane, k = ko0, j = jo0; it < hg.n_genomes * O * ST; it += 32) {
          const int gs = s0 + s_l;
          if (gs < S) {
            const int slot = gio[k * G + 1 + I + j];
            out[(size_t(gio[k * G]) * S + gs) * O + j] = slot < 0 ? qnan() : v[slot * ST + s_l];
          }
          k += dko;
          j += djo;
          if (j >= O) { j -= O; ++k; }
        }
        __syncwarp();
      }
    } else {
      // the staging wait gave up: report it, let the copy land (bounded)
      // before the buffer is reused, and NaN this batch's outputs
      if (lane == 0) atomicOr(w.counters + CTR_ERR, ERR_TMA_TIMEOUT);
      broken = !__all_sync(0xffffffffu, mbar_wait_bounded(mb, parity, DRAIN_POLLS));
      nan_batch_outputs(w, b, S, out, lane);
      __syncwarp();
    }
    if (!claimed && lane == 0) old = atomicAdd(claim, 1ull);
    parity ^= 1u;
    b = next_batch(old);
  }
}

}  // namespace

int lvl_tile(int S) { return S >= 4 ? 4 : (S >= 2 ? 2 : 1); }

size_t lvl_vals_bytes(const Ws &w, int st_samples) {
  return (sizeof(float) * size_t(w.lvl_slots) * st_samples + 15) & ~size_t(15);
}

size_t lvl_warp_bytes(const Ws &w, int st_samples) {
  // chunk partials of a round, plus 4 so that a clamped index past the round stays inside
  const size_t part = (sizeof(float) * size_t(w.lvl_pcap + 4) * st_samples + 15) & ~size_t(15);
  return (size_t(lvl_head_cap(w.I, w.O)) + lvl_vals_bytes(w, st_samples) + part + 127) &
         ~size_t(127);
}

cudaError_t launch_lvl_build(const Ws &w, int target, int budget_lo, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  const size_t plan_smem = w.P <= PLAN_STAGED ? sizeof(int2) * size_t(w.P) : 0;
  k_lvl_plan<<<1, PLAN_THREADS, plan_smem, st>>>(w, target, budget_lo);
  int slots2 = 1;
  while (slots2 < w.lvl_slots) slots2 <<= 1;
  const size_t smem = 8 * size_t(slots2) + 4 * size_t(w.lvl_slots + 1);
  k_lvl_build<<<w.lvl_max_batches, BLD_THREADS, smem, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_forward_lvl(const Ws &w, const float *inputs, int64_t stride, int S,
                               float *outputs, int warps, int grid, int polls, int pdl,
                               cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const int ST = lvl_tile(S);
  const int wb = int(lvl_warp_bytes(w, ST)), vb = int(lvl_vals_bytes(w, ST));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(32 * warps));
  cfg.dynamicSmemBytes = size_t(wb) * warps;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if (ST == 1)
    return cudaLaunchKernelEx(&cfg, k_forward_lvl<1>, w, inputs, stride, S, outputs, wb, vb, polls,
                              pdl);
  if (ST == 2)
    return cudaLaunchKernelEx(&cfg, k_forward_lvl<2>, w, inputs, stride, S, outputs, wb, vb, polls,
                              pdl);
  return cudaLaunchKernelEx(&cfg, k_forward_lvl<4>, w, inputs, stride, S, outputs, wb, vb, polls,
                            pdl);
}

cudaError_t lvl_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_forward_lvl<1>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_lvl<2>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_lvl<4>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_lvl_build, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_lvl_plan, bytes);
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
