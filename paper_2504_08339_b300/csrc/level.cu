// Level-synchronous batched forward for small sample counts (one or a few
// input vectors per genome, e.g. one observation per rollout step).
//
// With S = 1 a single genome offers only the few independent nodes of one
// layer at a time, so a CTA evaluates a whole BATCH of genomes at once: all
// their layer-r nodes are independent of each other (Sec. 3.3's order only
// requires each node to follow its inputs), so a round evaluates layer-r nodes
// of every genome in the batch.  A round has two fully packed phases: one
// thread per 4-edge chunk of incoming connections (partial sum / product /
// max), then one thread per node (combine the partials, bias, response,
// activation).  Nodes no output depends on are not evaluated at all (this
// form returns only the outputs).  Nodes are sorted by activation so a warp
// runs one activation branch, and by descending in-degree.
//
// Transform time (k_lvl_plan, k_lvl_build): genomes in layer-sorted queue
// order are cut into batches under a byte budget and each batch program is
// written contiguously (see BatchHead in neat_internal.cuh).
// Run time (k_forward_lvl): a persistent CTA claims a batch and stages its
// program into shared memory with two TMA bulk copies (cp.async.bulk with
// mbarrier completion and bounded waits): the head part (genome ids, I/O
// slots, round table) first, so the step's input loads are issued while the
// tasks and edges are still in flight.
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
// batch assignment: weight prefix in layer-sorted queue order (one CTA)
__global__ void __launch_bounds__(1024) k_lvl_plan(Ws w) {
  __shared__ long long wsum[32], psum[32];
  const int P = w.P, T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int I = w.I, O = w.O, budget = w.lvl_budget, sb = lvl_slot_budget(w.N);
  const int per = (P + T - 1) / T;
  const int b0 = min(tid * per, P), e0 = min(b0 + per, P);
  auto pbw = [&](int q, int &pb, int &wt) {
    const GenomeHdr h = w.hdr[w.qlvl[q]];
    const bool ok = h.status == 0u;
    pb = lvl_genome_bytes(h.nlive + I, h.nch, h.L, I, O, ok);  // tasks: the live nodes
    wt = lvl_genome_weight(pb, ok ? h.V : 0, budget, sb);
  };
  long long sw = 0, sp = 0;
  for (int q = b0; q < e0; ++q) {
    int pb, wt;
    pbw(q, pb, wt);
    sw += wt;
    sp += pb;
  }
  long long xw = sw, xp = sp;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long yw = __shfl_up_sync(0xffffffffu, xw, d), yp = __shfl_up_sync(0xffffffffu, xp, d);
    if (lane >= d) { xw += yw; xp += yp; }
  }
  if (lane == 31) { wsum[wid] = xw; psum[wid] = xp; }
  __syncthreads();
  if (wid == 0) {
    long long a = wsum[lane], c = psum[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long ya = __shfl_up_sync(0xffffffffu, a, d), yc = __shfl_up_sync(0xffffffffu, c, d);
      if (lane >= d) { a += ya; c += yc; }
    }
    wsum[lane] = a;
    psum[lane] = c;
  }
  __syncthreads();
  long long cw = (wid > 0 ? wsum[wid - 1] : 0) + xw - sw;
  long long cp = (wid > 0 ? psum[wid - 1] : 0) + xp - sp;
  // batch of the genome just before this thread's chunk
  long long bprev = -1;
  if (b0 > 0 && b0 < e0) {
    int pb, wt;
    pbw(b0 - 1, pb, wt);
    bprev = (cw - wt) / budget;
  }
  for (int q = b0; q < e0; ++q) {
    int pb, wt;
    pbw(q, pb, wt);
    const long long b = cw / budget;
    for (long long bb = bprev + 1; bb <= b; ++bb) w.lvl_first[bb] = q;
    w.lvl_goff[q] = int(cp);
    bprev = b;
    cw += wt;
    cp += pb;
  }
  __syncthreads();
  if (tid == 0) {
    int nb = 0;
    if (P > 0) {
      int pb, wt;
      pbw(P - 1, pb, wt);
      nb = int((wsum[31] - wt) / budget) + 1;
    }
    w.lvl_first[nb] = P;
    w.counters[CTR_NBATCH] = uint32_t(nb);
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
  const int I = w.I, O = w.O;
  const int q0 = w.lvl_first[b], q1 = w.lvl_first[b + 1];
  const int ng = q1 - q0;
  if (tid == 0) s_bad = (ng < 0 || ng > LVL_MAX_GENOMES) ? 1 : 0;
  __syncthreads();
  if (s_bad) return;  // cannot happen by construction of the weights
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
    int s = 0, nr = 0, nt = 0;
    for (int k = 0; k < ng; ++k) {
      g_slot[k] = s;
      s += g_V[k];
      nr = max(nr, g_L[k]);
      nt += g_NL[k];
    }
    g_slot[ng] = s;
    s_nslots = s;
    s_ntasks = nt;
    s_nrounds = nr;
  }
  __syncthreads();
  const int nslots = s_nslots, ntasks = s_ntasks;
  if (nslots > LVL_MAX_SLOTS) return;  // cannot happen by construction of the weights
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
  // rounds: one layer each, split where a layer exceeds LVL_PCAP chunks (a
  // single task never does: a node has fewer than N <= 1024 in-edges)
  if (tid == 0) {
    int R = 0, in = 0, cur = -1;
    for (int j = 0; j < ntasks; ++j) {
      const int lay = int(keys[j] >> 33);
      const int nc = cnt[j + 1] - cnt[j];
      if (j == 0 || lay != cur || in + nc > LVL_PCAP) {
        ++R;
        in = 0;
        cur = lay;
      }
      in += nc;
    }
    s_nrounds = R;
  }
  __syncthreads();
  const int nrounds2 = s_nrounds;
  // program layout: head part (header, gio, round table), then tasks and edges
  const int G = 1 + I + O;
  const int off_gio = int(sizeof(BatchHead));
  const int off_round = (off_gio + 4 * ng * G + 7) & ~7;
  const int off_task = (off_round + int(sizeof(RoundRec)) * (nrounds2 + 1) + 15) & ~15;
  const int off_eslot = off_task + int(sizeof(TaskRec)) * ntasks;
  const int off_ew = (off_eslot + 8 * nchunks + 15) & ~15;
  const int bytes = (off_ew + 16 * nchunks + 15) & ~15;
  unsigned char *base = w.lvl_arena + w.lvl_goff[q0];
  RoundRec *rt = reinterpret_cast<RoundRec *>(base + off_round);
  TaskRec *tasks = reinterpret_cast<TaskRec *>(base + off_task);
  uint16_t *eslot = reinterpret_cast<uint16_t *>(base + off_eslot);
  float *ew = reinterpret_cast<float *>(base + off_ew);
  int *gio = reinterpret_cast<int *>(base + off_gio);
  if (tid == 0) {
    BatchHead hd;
    hd.n_genomes = ng; hd.n_slots = nslots; hd.n_rounds = nrounds2; hd.n_tasks = ntasks;
    hd.n_chunks = nchunks; hd.off_round = off_round; hd.off_task = off_task;
    hd.off_eslot = off_eslot; hd.off_gio = off_gio; hd.prog_bytes = bytes; hd.off_ew = off_ew;
    hd.pad = 0;
    *reinterpret_cast<BatchHead *>(base) = hd;
    BatchLoc loc;
    loc.off = w.lvl_goff[q0];
    loc.bytes = bytes;
    loc.head = off_task;
    loc.pad = 0;
    w.lvl_loc[b] = loc;
    // round table (same walk as above), with the activation groups of each
    // round (tasks of a round are sorted by activation)
    int R = 0, in = 0, cur = -1;
    RoundRec rr;
    int hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    auto close_round = [&](int end) {
      int acc = 0;
      for (int a = 0; a < 8; ++a) {
        rr.act[a] = uint16_t(acc);
        acc += a < 7 ? hist[a] : 0;
      }
      rr.act[7] = uint16_t(end - rr.task);
      rt[R++] = rr;
      for (int a = 0; a < 8; ++a) hist[a] = 0;
    };
    for (int j = 0; j < ntasks; ++j) {
      const int lay = int(keys[j] >> 33);
      const int nc = cnt[j + 1] - cnt[j];
      if (j == 0 || lay != cur || in + nc > LVL_PCAP) {
        if (j > 0) close_round(j);
        rr.task = j;
        rr.chunk = cnt[j];
        in = 0;
        cur = lay;
      }
      in += nc;
      ++hist[int((keys[j] >> 30) & 7u)];
    }
    if (ntasks > 0) close_round(ntasks);
    rr.task = ntasks;
    rr.chunk = nchunks;
    for (int a = 0; a < 8; ++a) rr.act[a] = 0;
    rt[R] = rr;
  }
  // task records and their padded edge chunks
  for (int j = tid; j < ntasks; j += T) {
    const uint64_t key = keys[j];
    const int k = int((key >> 10) & 63u), p = int(key & 1023u);
    const NodeRec n = w.knode[g_noff[k] + p];
    const int c = meta_cnt(n.meta);
    TaskRec t;
    t.bias = n.bias;
    // mean: fold 1/n into the response, so that the round combines partial
    // sums the same way for sum and mean (r (s / n) -> (r / n) s, both
    // rounded once)
    t.resp = (meta_agg(n.meta) == NEAT_AGG_MEAN && c > 0) ? n.resp / float(c) : n.resp;
    t.chunk = uint32_t(cnt[j]);
    t.meta = task_meta(c, meta_act(n.meta), meta_agg(n.meta), g_slot[k] + p);
    tasks[j] = t;
    const EdgeRec *src = w.kedge + g_eoff[k] + n.in_begin;
    const int e0 = 4 * cnt[j], e1 = 4 * cnt[j + 1];
    for (int e = 0; e < e1 - e0; ++e) {
      if (e < c) {
        const EdgeRec er = src[e];
        eslot[e0 + e] = uint16_t(g_slot[k] + int(er.src));
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
// bounded mbarrier wait on a phase parity
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it) {
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
// accesses to them measured ~4 % slower per launch on the partial loads
// alone).  Volatile: never moved across the round's barriers.
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
__device__ __forceinline__ void sts_f32x4(float4 *p, float4 x) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(sh_addr(p)), "f"(x.x), "f"(x.y),
               "f"(x.z), "f"(x.w)
               : "memory");
}

// One round, two fully packed phases.
//  A: one thread per (4-edge chunk, sample): sum, product and max of the
//     chunk's w * v terms (padding slots skipped) into part[].
//  B: warp w takes the tasks of activation types w, w + nwarps, ...; one lane
//     per (task, sample) combines the task's chunk partials with its
//     aggregation, then v[slot] = act(b + r * a) -- one activation branch per
//     warp.
// Node phase of one activation group: lane (task, sample) combines the
// task's 4-edge chunk partials (sum, product, max), applies the aggregation
// (a mean's 1/n is folded into its response) and the activation ACT.
template <int ST, int ACT>
__device__ __forceinline__ void node_group(const TaskRec *__restrict__ tasks, const float4 *part,
                                           float *v, const RoundRec &lo, int g0, int gn,
                                           int lane) {
  for (int it = lane; it < gn; it += 32) {
    const int t = g0 + (ST == 1 ? it : it / ST);
    const int s = ST == 1 ? 0 : it % ST;
    const TaskRec tk = lds_task(tasks + t);
    const int cnt = task_cnt(tk.meta), agg = task_agg(tk.meta);
    const int c0 = int(tk.chunk) - lo.chunk, nc = (cnt + 3) >> 2;
    float sum = 0.0f, prod = 1.0f, mx = qnan();
    // partials four at a time: the loads of a group are in flight together
    for (int k = 0; k < nc; k += 4) {
      float4 p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        p[u] = k + u < nc ? lds_f32x4(part + (c0 + k + u) * ST + s)
                          : make_float4(0.0f, 1.0f, qnan(), 0.0f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sum += p[u].x;
        prod *= p[u].y;
        mx = fmaxf(mx, p[u].z);
      }
    }
    // empty aggregation: 0 for every aggregation
    const float a = nc == 0 ? 0.0f
                  : agg == NEAT_AGG_PRODUCT ? prod
                  : agg == NEAT_AGG_MAX ? mx : sum;
    sts_f32(v + task_slot(tk.meta) * ST + s, act_apply(ACT, fmaf(tk.resp, a, tk.bias)));
  }
}

template <int ST>
__device__ __forceinline__ void run_round(const TaskRec *__restrict__ tasks,
                                          const uint2 *__restrict__ eslot,
                                          const float4 *__restrict__ ew, float4 *part, float *v,
                                          const RoundRec &lo, int hi_chunk) {
  const int na = (hi_chunk - lo.chunk) * ST;
  for (int it = threadIdx.x; it < na; it += blockDim.x) {
    const int c = lo.chunk + (ST == 1 ? it : it / ST);
    const int s = ST == 1 ? 0 : it % ST;
    const uint2 sl = lds_u32x2(eslot + c);
    const float4 w4 = lds_f32x4(ew + c);
    const uint32_t q[4] = {sl.x & 0xffffu, sl.x >> 16, sl.y & 0xffffu, sl.y >> 16};
    const float wq[4] = {w4.x, w4.y, w4.z, w4.w};
    float sum = 0.0f, prod = 1.0f, mx = qnan();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (q[k] != 0xffffu) {
        const float x = lds_f32(v + q[k] * ST + s);
        sum = fmaf(wq[k], x, sum);
        const float tv = wq[k] * x;
        prod *= tv;
        mx = fmaxf(mx, tv);
      }
    }
    sts_f32x4(part + it, make_float4(sum, prod, mx, 0.0f));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int act = warp; act < 7; act += nw) {
    const int g0 = lo.task + lo.act[act], gn = (lo.act[act + 1] - lo.act[act]) * ST;
    if (gn == 0) continue;
    // the activation is a compile-time constant in each group loop
#define NEAT_GROUP(A) node_group<ST, A>(tasks, part, v, lo, g0, gn, lane)
    switch (act) {
      case NEAT_ACT_IDENTITY: NEAT_GROUP(NEAT_ACT_IDENTITY); break;
      case NEAT_ACT_SIGMOID: NEAT_GROUP(NEAT_ACT_SIGMOID); break;
      case NEAT_ACT_TANH: NEAT_GROUP(NEAT_ACT_TANH); break;
      case NEAT_ACT_RELU: NEAT_GROUP(NEAT_ACT_RELU); break;
      case NEAT_ACT_SIN: NEAT_GROUP(NEAT_ACT_SIN); break;
      case NEAT_ACT_GAUSSIAN: NEAT_GROUP(NEAT_ACT_GAUSSIAN); break;
      default: NEAT_GROUP(NEAT_ACT_ABS); break;
    }
#undef NEAT_GROUP
  }
}

template <int ST>
__global__ void __launch_bounds__(256) k_forward_lvl(Ws w, const float *__restrict__ inputs,
                                                     int64_t stride, int S,
                                                     float *__restrict__ out, int prog_cap,
                                                     int vals_bytes) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int s_b;
  const int tid = threadIdx.x;
  const int I = w.I, O = w.O, G = 1 + I + O;
  float *v = reinterpret_cast<float *>(sm + prog_cap);
  float4 *part = reinterpret_cast<float4 *>(sm + prog_cap + vals_bytes);
  const uint32_t mb0 = uint32_t(__cvta_generic_to_shared(&mbar[0]));
  const uint32_t mb1 = uint32_t(__cvta_generic_to_shared(&mbar[1]));
  const uint32_t sm_a = uint32_t(__cvta_generic_to_shared(sm));
  const int nbatch = int(w.counters[CTR_NBATCH]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the step's inputs towards L2, one 128-byte line per thread of the grid
  // (every address inside the inputs): the batches' input loads then hit L2
  if (stride >= 0) {
    const size_t total = size_t(w.P - 1) * size_t(stride) + size_t(S) * I;
    const size_t lines = (total + 31) / 32;
    for (size_t l = size_t(blockIdx.x) * blockDim.x + tid; l < lines;
         l += size_t(gridDim.x) * blockDim.x)
      asm volatile("prefetch.L2 [%0];" ::"l"(inputs + l * 32));
  }
  uint32_t parity = 0;
  // the first batch of each CTA is its own index, later ones are claimed in
  // order of finishing: no contended atomic at the start of the launch
  bool first = true;
  for (;;) {
    if (tid == 0)
      s_b = first ? int(blockIdx.x) : int(gridDim.x + atomicAdd(w.counters + CTR_LVL_ITEM, 1u));
    first = false;
    __syncthreads();
    const int b = s_b;
    if (b >= nbatch) break;
    const BatchLoc loc = w.lvl_loc[b];
    const unsigned char *src = w.lvl_arena + loc.off;
    if (tid == 0) {
      // the head part (up to off_task) and the rest, each on its own mbarrier
      const int head = loc.head;
      // order earlier generic-proxy accesses of the buffer before the copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb0), "r"(head)
                   : "memory");
      bulk_g2s(sm_a, src, head, mb0);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb1),
                   "r"(loc.bytes - head)
                   : "memory");
      bulk_g2s(sm_a + uint32_t(head), src + head, loc.bytes - head, mb1);
    }
    bool ok = mbar_wait_bounded(mb0, parity);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(w.counters + CTR_ERR, ERR_TMA_TIMEOUT);
      mbar_wait_bounded(mb1, parity);  // one more bounded wait for the copy in flight
      break;
    }
    const BatchHead hd = *reinterpret_cast<const BatchHead *>(sm);
    const int *gio = reinterpret_cast<const int *>(sm + hd.off_gio);
    const RoundRec *rt = reinterpret_cast<const RoundRec *>(sm + hd.off_round);
    const TaskRec *tasks = reinterpret_cast<const TaskRec *>(sm + hd.off_task);
    const uint2 *eslot = reinterpret_cast<const uint2 *>(sm + hd.off_eslot);
    const float4 *ew = reinterpret_cast<const float4 *>(sm + hd.off_ew);
    for (int s0 = 0; s0 < S; s0 += ST) {
      // inputs (for the first tile while tasks and edges are still arriving)
      for (int it = tid; it < hd.n_genomes * I * ST; it += blockDim.x) {
        const int s = it % ST, r = it / ST, k = r / I, i = r - k * I;
        const int slot = gio[k * G + 1 + i];
        if (slot < 0) continue;
        const int gs = s0 + s;
        v[slot * ST + s] =
            gs < S ? __ldg(inputs + size_t(gio[k * G]) * stride + size_t(gs) * I + i) : 0.0f;
      }
      if (s0 == 0) {
        ok = mbar_wait_bounded(mb1, parity);
        if (__syncthreads_or(!ok)) {
          ok = false;  // the same outcome on every thread
          if (tid == 0) atomicOr(w.counters + CTR_ERR, ERR_TMA_TIMEOUT);
          break;
        }
      } else {
        __syncthreads();
      }
      for (int r = 0; r < hd.n_rounds; ++r) {
        run_round<ST>(tasks, eslot, ew, part, v, rt[r], rt[r + 1].chunk);
        __syncthreads();
      }
      for (int it = tid; it < hd.n_genomes * O * ST; it += blockDim.x) {
        const int s = it % ST, r = it / ST, k = r / O, j = r - k * O;
        const int gs = s0 + s;
        if (gs >= S) continue;
        const int slot = gio[k * G + 1 + I + j];
        out[(size_t(gio[k * G]) * S + gs) * O + j] = slot < 0 ? qnan() : v[slot * ST + s];
      }
      __syncthreads();
    }
    parity ^= 1u;
    if (!ok) break;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(w.counters + CTR_LVL_DONE, 1u);
    if (t == gridDim.x - 1) {
      atomicExch(w.counters + CTR_LVL_ITEM, 0u);
      atomicExch(w.counters + CTR_LVL_DONE, 0u);
    }
  }
}

size_t prog_cap_bytes(const Ws &w) {
  const int pbmax = lvl_pb_max(w.N, w.C, w.I, w.O);
  return size_t((w.lvl_budget + pbmax + 127) & ~127);
}

size_t vals_bytes(const Ws &w, int st_samples) {
  return (sizeof(float) * size_t(lvl_slot_budget(w.N) + w.N) * st_samples + 15) & ~size_t(15);
}

}  // namespace

int lvl_tile(int S) { return S >= 4 ? 4 : (S >= 2 ? 2 : 1); }

size_t forward_lvl_smem(const Ws &w, int st_samples) {
  return prog_cap_bytes(w) + vals_bytes(w, st_samples) +
         sizeof(float4) * size_t(LVL_PCAP) * st_samples;
}

cudaError_t launch_lvl_build(const Ws &w, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  k_lvl_plan<<<1, 1024, 0, st>>>(w);
  const size_t smem = 8 * size_t(LVL_MAX_SLOTS) + 4 * size_t(LVL_MAX_SLOTS + 1);
  k_lvl_build<<<w.lvl_max_batches, BLD_THREADS, smem, st>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_forward_lvl(const Ws &w, const float *inputs, int64_t stride, int S,
                               float *outputs, int threads, int grid, cudaStream_t st) {
  if (w.P == 0 || S == 0) return cudaSuccess;
  const int ST = lvl_tile(S);
  const size_t smem = forward_lvl_smem(w, ST);
  const int cap = int(prog_cap_bytes(w));
  const int vb = int(vals_bytes(w, ST));
  if (ST == 1)
    k_forward_lvl<1><<<grid, threads, smem, st>>>(w, inputs, stride, S, outputs, cap, vb);
  else if (ST == 2)
    k_forward_lvl<2><<<grid, threads, smem, st>>>(w, inputs, stride, S, outputs, cap, vb);
  else
    k_forward_lvl<4><<<grid, threads, smem, st>>>(w, inputs, stride, S, outputs, cap, vb);
  return cudaGetLastError();
}

cudaError_t lvl_set_smem_limit(int bytes) {
  cudaError_t e = set_dyn_smem_limit(k_forward_lvl<1>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_lvl<2>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_forward_lvl<4>, bytes);
  if (e == cudaSuccess) e = set_dyn_smem_limit(k_lvl_build, bytes);
  return e;
}

int forward_lvl_occupancy(int threads, size_t smem, int st_samples) {
  int n = 0;
  cudaError_t e;
  if (st_samples == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_lvl<1>, threads, smem);
  else if (st_samples == 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_lvl<2>, threads, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_forward_lvl<4>, threads, smem);
  return e == cudaSuccess ? n : 0;
}

}  // namespace neat
