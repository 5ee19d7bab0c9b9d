// Structure check of a plan's transformed population (neat_plan_validate).
//
// Every index a forward, backward or HyperNEAT kernel follows comes either
// from its own loop bounds or from the structures the transform writes: the
// queues, the genome headers, the ragged-packed position programs, the
// compiled programs and the level batch programs.  These kernels check each
// such stored index against the array it addresses (and the counts that bound
// the kernels' loops against their arrays), reading only inside the
// workspace regions whatever the contents, so a corrupted or stale workspace
// is reported instead of being walked.  The kernels of the evaluation path
// are left untouched: their indices are in range whenever these checks pass.
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

struct ValArgs {
  Ws w;
  uint32_t *bits;
  long long nodes_cap, edges_cap;  // knode / kedge records of the packed programs
  long long arena_bytes;
  int feedforward;                 // 1: neat_transform (compiled programs, batches)
  int cpair_cap;
};

__device__ __forceinline__ void flag(const ValArgs &a, uint32_t bit) { atomicOr(a.bits, bit); }

// the status bits a transform sets (any other bit: a corrupt header)
constexpr uint32_t kStatusBits = NEAT_G_CYCLE | NEAT_G_DANGLING_KEY | NEAT_G_DUP_KEY |
                                 NEAT_G_DUP_EDGE | NEAT_G_EDGE_INTO_INPUT | NEAT_G_BAD_ATTR |
                                 NEAT_G_IO_ROW_INVALID;

// queues: every entry a genome id
__global__ void __launch_bounds__(256) k_val_queues(ValArgs a) {
  const int P = a.w.P;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < P; q += gridDim.x * blockDim.x) {
    const int g = a.w.qorder[q];
    bool bad = g < 0 || g >= P;
    if (a.feedforward) {
      const int h = a.w.qlvl[q];
      bad = bad || h < 0 || h >= P;
    }
    if (bad) flag(a, NEAT_BAD_QUEUE);
  }
}

// one warp per genome: header, packed program, input / output positions and
// (feed-forward) the compiled program
__global__ void __launch_bounds__(256) k_val_genomes(ValArgs a) {
  const Ws &w = a.w;
  const int lane = threadIdx.x & 31;
  const int N = w.N, C = w.C, I = w.I, O = w.O;
  for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < w.P;
       g += (gridDim.x * blockDim.x) >> 5) {
    const GenomeHdr h = w.hdr[g];
    if (h.status != 0u) {  // rejected: the kernels walk nothing of it
      if ((h.status & ~kStatusBits) != 0u && lane == 0) flag(a, NEAT_BAD_PACKED);
      continue;
    }
    bool pk = h.V >= I + O && h.V <= N && h.E >= 0 && h.E <= C && h.L >= 0 && h.L <= h.V &&
              h.node_off >= 0 && h.edge_off >= 0 &&
              (long long)h.node_off + h.V <= a.nodes_cap &&
              (long long)h.edge_off + h.E <= a.edges_cap;
    if (pk) {
      for (int p = lane; p < h.V; p += 32) {
        const NodeRec n = w.knode[size_t(h.node_off) + p];
        const int cnt = meta_cnt(n.meta);
        bool ok = meta_act(n.meta) <= NEAT_ACT_ABS && meta_agg(n.meta) <= NEAT_AGG_MEAN &&
                  (long long)n.in_begin + cnt <= h.E;
        if (ok) {
          // sources: earlier positions (feed-forward) or any position (recurrent)
          const uint32_t lim = a.feedforward ? uint32_t(p) : uint32_t(h.V);
          for (int k = 0; k < cnt; ++k)
            ok = ok && w.kedge[size_t(h.edge_off) + n.in_begin + k].src < lim;
        }
        pk = pk && ok;
      }
      for (int i = lane; i < I + O; i += 32) {
        const int pos = w.pio[size_t(g) * (I + O) + i];
        pk = pk && pos >= 0 && pos < h.V;
      }
    }
    if (!__all_sync(0xffffffffu, pk)) {
      if (lane == 0) flag(a, NEAT_BAD_PACKED);
      continue;
    }
    if (!a.feedforward || w.cnode == nullptr) continue;
    // compiled program: rows 0..I-1 inputs, I and I + 1 the constants, node
    // rows after them (at most N + 2 rows in all)
    bool cp = h.nlive >= 0 && h.nlive <= h.V && h.crows >= I + 2 && h.crows <= N + 2 &&
              h.clayers >= 0 && h.clayers <= h.nlive && h.cpairs >= 0 &&
              h.cpairs <= a.cpair_cap;
    if (cp) {
      const CNode *cn = w.cnode + size_t(g) * N;
      const uint4 *pr = w.cpair + size_t(g) * a.cpair_cap;
      const int32_t *cl = w.clay + size_t(g) * (N + 1);
      const uint32_t rows = uint32_t(h.crows);
      for (int c = lane; c < h.nlive; c += 32) {
        const CNode n = cn[c];
        const uint32_t first = n.pairs & ((1u << CN_PAIR_BITS) - 1u), np = n.pairs >> CN_PAIR_BITS;
        cp = cp && first + np <= uint32_t(h.cpairs) &&
             (n.meta & ((1u << CN_ROW_BITS) - 1u)) < rows &&
             ((n.meta >> CN_ROW_BITS) & 7u) <= uint32_t(NEAT_ACT_ABS);
      }
      for (int k = lane; k < h.cpairs; k += 32) {
        const uint4 e = pr[k];
        cp = cp && e.x < rows && e.z < rows;
      }
      for (int k = lane; k <= h.clayers; k += 32) {
        const int v = cl[k], prev = k > 0 ? cl[k - 1] : 0;
        cp = cp && v >= prev && v <= h.nlive && (k < h.clayers || v == h.nlive);
      }
      for (int o = lane; o < O; o += 32) {
        const int r = w.cout[size_t(g) * O + o];
        cp = cp && r >= 0 && uint32_t(r) < rows;
      }
    }
    if (!__all_sync(0xffffffffu, cp) && lane == 0) flag(a, NEAT_BAD_COMPILED);
  }
}

// one warp per level batch: its place in the arena, header, genome table,
// round table, task records and edge slots
__global__ void __launch_bounds__(256) k_val_batches(ValArgs a) {
  const Ws &w = a.w;
  const int lane = threadIdx.x & 31;
  const int I = w.I, O = w.O, G = 1 + I + O, P = w.P;
  const int nb_raw = int(w.counters[CTR_NBATCH]);
  const bool nb_ok = nb_raw >= (P > 0 ? 1 : 0) && nb_raw <= w.lvl_max_batches;
  if (!nb_ok) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flag(a, NEAT_BAD_BATCHES);
    return;
  }
  const int nbatch = nb_raw;
  if (blockIdx.x == 0 && threadIdx.x == 0 &&
      (w.lvl_first[0] != 0 || w.lvl_first[nbatch] != P))
    flag(a, NEAT_BAD_BATCHES);
  const int hcap = lvl_head_cap(I, O);
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbatch;
       b += (gridDim.x * blockDim.x) >> 5) {
    const int q0 = w.lvl_first[b], q1 = w.lvl_first[b + 1];
    const BatchLoc loc = w.lvl_loc[b];
    bool ok = q0 >= 0 && q1 <= P && q1 - q0 >= 1 && q1 - q0 <= LVL_MAX_GENOMES &&
              loc.off >= 0 && (loc.off & 15) == 0 && loc.bytes >= int(sizeof(BatchHead)) &&
              (long long)loc.off + loc.bytes <= a.arena_bytes && (loc.head & 15) == 0 &&
              loc.head <= loc.bytes && loc.head <= hcap;
    BatchHead hd{};
    if (ok) {
      hd = *reinterpret_cast<const BatchHead *>(w.lvl_arena + loc.off);
      const long long nc = hd.n_chunks, nt = hd.n_tasks, nr = hd.n_rounds;
      // (a round holds at least one task: n_rounds <= n_tasks)
      ok = hd.n_genomes == q1 - q0 && hd.n_slots >= LVL_CONST_SLOTS &&
           hd.n_slots <= w.lvl_slots && nt >= 0 && nc >= 0 && nr >= 0 && nr <= nt && nt < 65536 &&
           nc < 65536 && hd.off_gio >= int(sizeof(BatchHead)) &&
           hd.off_gio + 4LL * hd.n_genomes * G <= hd.off_round && hd.off_round == loc.head &&
           hd.off_round + 4 * (nr + 1) <= hd.off_task && (hd.off_task & 15) == 0 &&
           hd.off_task + 16 * nt <= hd.off_eslot && (hd.off_eslot & 7) == 0 &&
           hd.off_eslot + 8 * nc <= hd.off_ew && (hd.off_ew & 15) == 0 &&
           hd.off_ew + 16 * nc <= hd.prog_bytes && hd.prog_bytes <= loc.bytes;
    }
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) flag(a, NEAT_BAD_BATCHES);
      continue;
    }
    const unsigned char *base = w.lvl_arena + loc.off;
    const int *gio = reinterpret_cast<const int *>(base + hd.off_gio);
    const uint32_t *rt = reinterpret_cast<const uint32_t *>(base + hd.off_round);
    const uint4 *tasks = reinterpret_cast<const uint4 *>(base + hd.off_task);
    const uint2 *eslot = reinterpret_cast<const uint2 *>(base + hd.off_eslot);
    const int ns = hd.n_slots;
    // genome table: ids of the batch's queue entries, slots in range or -1
    for (int i = lane; i < hd.n_genomes * G; i += 32) {
      const int k = i / G, f = i - k * G, v = gio[i];
      ok = ok && (f == 0 ? v == w.qlvl[q0 + k] && v >= 0 && v < P : v >= -1 && v < ns);
    }
    // round table: from (0, 0) to (n_tasks, n_chunks), never backwards, at
    // most lvl_pcap chunks a round; each round's tasks take chunks inside it
    const uint32_t last = uint32_t(hd.n_tasks) | (uint32_t(hd.n_chunks) << 16);
    ok = ok && rt[0] == 0u && rt[hd.n_rounds] == last;
    for (int r = 0; r < hd.n_rounds; ++r) {
      const uint32_t ra = rt[r], rb = rt[r + 1];
      const int t0 = int(ra & 0xffffu), t1 = int(rb & 0xffffu);
      const int c0 = int(ra >> 16), c1 = int(rb >> 16);
      if (!(t0 <= t1 && c0 <= c1 && t1 <= hd.n_tasks && c1 <= hd.n_chunks &&
            c1 - c0 <= w.lvl_pcap)) {
        ok = false;
        break;
      }
      for (int t = t0 + lane; t < t1; t += 32) {
        const uint4 q = tasks[t];
        const uint32_t m = q.w;
        const int ch = int(q.z), nch = (task_cnt(m) + 3) >> 2;
        ok = ok && ch >= c0 && ch + nch <= c1 && task_slot(m) >= LVL_CONST_SLOTS &&
             task_slot(m) < ns && task_act(m) <= NEAT_ACT_ABS;
      }
    }
    // edge slots (the first of a chunk carries the aggregation above its 12 bits)
    for (int c = lane; c < hd.n_chunks; c += 32) {
      const uint2 s = eslot[c];
      ok = ok && int(s.x & uint32_t(LVL_MAX_SLOTS - 1)) < ns && int(s.x >> 16) < ns &&
           int(s.y & 0xffffu) < ns && int(s.y >> 16) < ns;
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0) flag(a, NEAT_BAD_BATCHES);
  }
}

}  // namespace

cudaError_t launch_validate(const Ws &w, const Layout &L, int feedforward, uint32_t *bits,
                            int sm_count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess || w.P == 0) return e;
  ValArgs a;
  a.w = w;
  a.bits = bits;
  a.nodes_cap = (long long)w.P * w.N;
  a.edges_cap = (long long)w.P * w.C;
  a.arena_bytes = (long long)L.lvl_arena_bytes;
  a.feedforward = feedforward;
  a.cpair_cap = cpair_cap(w.N, w.C);
  const int blocks = 4 * (sm_count > 0 ? sm_count : 1);
  k_val_queues<<<blocks, 256, 0, st>>>(a);
  k_val_genomes<<<blocks, 256, 0, st>>>(a);
  if (feedforward) k_val_batches<<<blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace neat
