// Transformation stage (TensorNEAT Sec. 3.3): per genome, decode the padded
// rows (Sec. 3.1), check them, sort nodes by key, resolve connection keys,
// run Kahn's algorithm frontier by frontier (ascending key inside a frontier,
// so the order is the unique sort by (layer, key)), and write the order, the
// layer indices and a packed program that replaces the dense C_exp tensor.
//
// One CTA per genome (4 or 8 warps); everything lives in shared memory.  Then
// three small kernels build the size-sorted work queue and the ragged-packed
// copy.
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

constexpr float KEY_LIMIT = 16777216.0f;  // 2^24
// genomes of at most this many valid nodes run Kahn's loop on one warp
constexpr int KAHN_WARP_MAX_V = 256;

__device__ __forceinline__ bool is_int_in(float x, float lo, float hi) {
  return x == x && x >= lo && x < hi && x == floorf(x);
}

// Exclusive scan of a[0..n) in place; returns the total.  All threads call it.
__device__ int block_exclusive_scan(int *a, int n, int *wbuf) {
  const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = (T + 31) >> 5;
  const int per = (n + T - 1) / T;
  const int b = min(tid * per, n), e = min(b + per, n);
  int s = 0;
  for (int i = b; i < e; ++i) s += a[i];
  int x = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wbuf[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? wbuf[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < nw) wbuf[lane] = w;
  }
  __syncthreads();
  int base = (wid > 0 ? wbuf[wid - 1] : 0) + x - s;
  const int total = wbuf[nw - 1];
  for (int i = b; i < e; ++i) {
    int v = a[i];
    a[i] = base;
    base += v;
  }
  __syncthreads();
  return total;
}

// Ascending bitonic sort of a[0..n2), n2 a power of two.
__device__ void bitonic_sort_u64(uint64_t *a, int n2) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < (n2 >> 1); i += blockDim.x) {
        const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
        const int hi = lo + j;
        const uint64_t x = a[lo], y = a[hi];
        const bool up = (lo & k) == 0;
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
        }
      }
      __syncthreads();
    }
}

__host__ __device__ inline int pow2_ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct TSmem {
  // byte offsets into dynamic shared memory
  int sk, ek, key_s, row_of_s, s_of_row, indeg, rem, inbeg, outbeg, outfill, order_s, layer_s,
      pos_of, tmp, ready, outlist, cls, total;
};

__host__ __device__ inline TSmem tsmem_layout(int N, int C) {
  TSmem L;
  const int N2 = pow2_ceil(N), C2 = pow2_ceil(C);
  int off = 0;
  auto take = [&](int bytes) { int o = off; off += (bytes + 15) & ~15; return o; };
  L.sk = take(8 * N2);
  L.ek = take(8 * C2);
  L.key_s = take(4 * N);
  L.row_of_s = take(4 * N);
  L.s_of_row = take(4 * N);
  L.indeg = take(4 * N);
  L.rem = take(4 * N);
  L.inbeg = take(4 * N);
  L.outbeg = take(4 * (N + 1));
  L.outfill = take(4 * N);
  L.order_s = take(4 * N);
  L.layer_s = take(4 * N);
  L.pos_of = take(4 * N);
  L.tmp = take(4 * (N + 1));
  L.ready = take(4 * N);
  L.outlist = take(4 * C);
  L.cls = take(4 * (N + 1));
  L.total = off;
  return L;
}

__global__ void __launch_bounds__(256) k_transform(Ws w, const float *__restrict__ nodes,
                                                   const float *__restrict__ conns,
                                                   int32_t *__restrict__ order,
                                                   int32_t *__restrict__ layer,
                                                   int32_t *__restrict__ n_layers,
                                                   uint32_t *__restrict__ gstatus,
                                                   int recurrent) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int wbuf[33];
  __shared__ unsigned s_status;
  __shared__ int s_V, s_E, s_nch, s_nlive, s_elive, s_crows, s_emit, s_t;

  const int N = w.N, C = w.C, I = w.I, O = w.O;
  const int g = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const TSmem L = tsmem_layout(N, C);
  uint64_t *sk = reinterpret_cast<uint64_t *>(sm + L.sk);
  uint64_t *ek = reinterpret_cast<uint64_t *>(sm + L.ek);
  int *key_s = reinterpret_cast<int *>(sm + L.key_s);
  int *row_of_s = reinterpret_cast<int *>(sm + L.row_of_s);
  int *s_of_row = reinterpret_cast<int *>(sm + L.s_of_row);
  int *indeg = reinterpret_cast<int *>(sm + L.indeg);
  int *rem = reinterpret_cast<int *>(sm + L.rem);
  int *inbeg = reinterpret_cast<int *>(sm + L.inbeg);
  int *outbeg = reinterpret_cast<int *>(sm + L.outbeg);
  int *outfill = reinterpret_cast<int *>(sm + L.outfill);
  int *order_s = reinterpret_cast<int *>(sm + L.order_s);
  int *layer_s = reinterpret_cast<int *>(sm + L.layer_s);
  int *pos_of = reinterpret_cast<int *>(sm + L.pos_of);
  int *tmp = reinterpret_cast<int *>(sm + L.tmp);
  int *ready = reinterpret_cast<int *>(sm + L.ready);
  int *outlist = reinterpret_cast<int *>(sm + L.outlist);

  const float *gn = nodes + size_t(g) * N * 5;
  const float *gc = conns + size_t(g) * C * 4;

  if (tid == 0) { s_status = 0u; s_V = 0; s_E = 0; s_nch = 0; s_nlive = 0; s_elive = 0; }
  __syncthreads();

  // 1. node rows: validity, attribute checks, (key,row) sort keys of the
  // valid rows, gathered at the front (the sort then covers pow2(V) entries)
  unsigned st = 0u;
  for (int i = tid; i < N; i += T) {
    uint64_t key = ~0ull;
    {
      const float k = gn[i * 5 + 0];
      s_of_row[i] = -1;
      if (k == k) {
        uint32_t ku = 0xffffffffu;
        if (is_int_in(k, 0.0f, KEY_LIMIT)) ku = uint32_t(k); else st |= NEAT_G_BAD_ATTR;
        if (i >= I) {
          const float b = gn[i * 5 + 1], r = gn[i * 5 + 2], a = gn[i * 5 + 3], ag = gn[i * 5 + 4];
          if (!is_int_in(a, 0.0f, 7.0f) || !is_int_in(ag, 0.0f, 4.0f) || b != b || r != r)
            st |= NEAT_G_BAD_ATTR;
        }
        key = (uint64_t(ku) << 32) | uint32_t(i);
      } else if (i < I + O) {
        st |= NEAT_G_IO_ROW_INVALID;
      }
    }
    if (key != ~0ull) sk[atomicAdd(&s_V, 1)] = key;
  }
  if (st) atomicOr(&s_status, st);
  __syncthreads();
  const int V = s_V;
  {
    const int v2 = pow2_ceil(max(V, 1));
    for (int i = V + tid; i < v2; i += T) sk[i] = ~0ull;
    __syncthreads();
    bitonic_sort_u64(sk, v2);
  }

  // 2. sorted key table, duplicate keys
  st = 0u;
  for (int s = tid; s < V; s += T) {
    const uint64_t x = sk[s];
    const int row = int(x & 0xffffffffu);
    key_s[s] = int(x >> 32);  // keys < 2^24 (or 0xffffffff for a bad key: genome rejected)
    row_of_s[s] = row;
    s_of_row[row] = s;
    if (s > 0 && (sk[s - 1] >> 32) == (x >> 32)) st |= NEAT_G_DUP_KEY;
    indeg[s] = 0;
    outfill[s] = 0;
    layer_s[s] = -1;
    ready[s] = 0;
  }
  if (st) atomicOr(&s_status, st);
  __syncthreads();

  // 3. connection rows: enabled ones resolved to sorted node indices,
  // gathered at the front (the sort then covers pow2(E) entries)
  st = 0u;
  for (int j = tid; j < C; j += T) {
    uint64_t key = ~0ull;
    {
      const float4 c = reinterpret_cast<const float4 *>(gc)[j];
      const bool valid = (c.x == c.x) && (c.y == c.y);
      const bool enabled = valid && (c.w == c.w) && c.w != 0.0f;
      if (enabled) {
        int src = -1, dst = -1;
        float kk[2] = {c.x, c.y};
        int res[2];
        for (int t = 0; t < 2; ++t) {
          res[t] = -1;
          if (is_int_in(kk[t], 0.0f, KEY_LIMIT)) {
            const int ku = int(kk[t]);
            int lo = 0, hi = V;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (key_s[mid] < ku) lo = mid + 1; else hi = mid;
            }
            if (lo < V && key_s[lo] == ku) res[t] = lo;
          }
        }
        src = res[0];
        dst = res[1];
        if (src < 0 || dst < 0) {
          st |= NEAT_G_DANGLING_KEY;
        } else {
          if (row_of_s[dst] < I) st |= NEAT_G_EDGE_INTO_INPUT;
          if (c.z != c.z) st |= NEAT_G_BAD_ATTR;
          key = (uint64_t(dst) << 40) | (uint64_t(src) << 20) | uint64_t(j);
        }
      }
    }
    if (key != ~0ull) ek[atomicAdd(&s_E, 1)] = key;
  }
  if (st) atomicOr(&s_status, st);
  __syncthreads();
  const int E = s_E;
  {
    const int e2 = pow2_ceil(max(E, 1));
    for (int i = E + tid; i < e2; i += T) ek[i] = ~0ull;
    __syncthreads();
    bitonic_sort_u64(ek, e2);
  }

  // 4. in-degrees, incoming segments, duplicate edges, out-degree counts
  st = 0u;
  for (int i = tid; i < E; i += T) {
    const uint64_t x = ek[i];
    const int dst = int(x >> 40), src = int((x >> 20) & 0xfffffu);
    atomicAdd(&indeg[dst], 1);
    atomicAdd(&outfill[src], 1);
    if (i == 0 || int(ek[i - 1] >> 40) != dst) inbeg[dst] = i;
    if (i > 0 && (ek[i - 1] >> 20) == (x >> 20)) st |= NEAT_G_DUP_EDGE;
  }
  if (st) atomicOr(&s_status, st);
  __syncthreads();
  for (int s = tid; s < V; s += T) outbeg[s] = outfill[s];
  __syncthreads();
  block_exclusive_scan(outbeg, V, wbuf);
  for (int s = tid; s < V; s += T) outfill[s] = 0;
  __syncthreads();
  for (int i = tid; i < E; i += T) {
    const uint64_t x = ek[i];
    const int dst = int(x >> 40), src = int((x >> 20) & 0xfffffu);
    outlist[outbeg[src] + atomicAdd(&outfill[src], 1)] = dst;
  }
  const unsigned status0 = s_status;  // read after the previous barrier
  __syncthreads();

  // 5. Kahn by frontier.  Each round emits every ready node in ascending key
  // (sorted index order = key order), then releases their successors.
  int emitted = 0, t = 0;
  if (recurrent) {
    // recurrent networks need no order: every valid node in ascending key
    // (sorted index order) as one frontier; cycles are legal
    if ((status0 & ~NEAT_G_CYCLE) == 0u) {
      for (int s = tid; s < V; s += T) {
        order_s[s] = s;
        layer_s[s] = 0;
        pos_of[s] = s;
      }
      emitted = V;
      t = V > 0 ? 1 : 0;
    }
  } else if ((status0 & ~NEAT_G_CYCLE) == 0u && V <= KAHN_WARP_MAX_V) {
    // one warp: a frontier is the ready flags of 32-node chunks as ballots,
    // each emitted node's position the popc of the ready bits below it; no
    // CTA barrier inside the loop (the other warps wait at the one after it)
    if (tid < 32) {
      const int lane = tid;
      for (int s = lane; s < V; s += 32) {
        rem[s] = indeg[s];
        ready[s] = indeg[s] == 0;
      }
      __syncwarp();
      const unsigned below = (1u << lane) - 1u;
      for (int round = 0; round <= V; ++round) {  // bounded: each round emits >= 1 node
        int F = 0;
        for (int c = 0; c < V; c += 32) {
          const int s = c + lane;
          const bool r = s < V && ready[s] != 0;
          const unsigned m = __ballot_sync(0xffffffffu, r);
          if (r) {
            const int p = emitted + F + __popc(m & below);
            order_s[p] = s;
            layer_s[s] = t;
            pos_of[s] = p;
            ready[s] = 0;
          }
          F += __popc(m);
        }
        if (F == 0) break;
        __syncwarp();
        for (int p = emitted + lane; p < emitted + F; p += 32) {
          const int s = order_s[p];
          for (int k = outbeg[s]; k < outbeg[s] + outfill[s]; ++k) {
            const int d = outlist[k];
            if (atomicSub(&rem[d], 1) == 1) ready[d] = 1;
          }
        }
        __syncwarp();
        emitted += F;
        ++t;
      }
      if (lane == 0) {
        s_emit = emitted;
        s_t = t;
        if (emitted < V) atomicOr(&s_status, NEAT_G_CYCLE);
      }
    }
    __syncthreads();
    emitted = s_emit;
    t = s_t;
  } else if ((status0 & ~NEAT_G_CYCLE) == 0u) {
    for (int s = tid; s < V; s += T) {
      rem[s] = indeg[s];
      ready[s] = indeg[s] == 0;
    }
    __syncthreads();
    for (int round = 0; round <= V; ++round) {  // bounded: each round emits >= 1 node
      for (int s = tid; s < V; s += T) tmp[s] = ready[s];
      __syncthreads();
      const int F = block_exclusive_scan(tmp, V, wbuf);
      if (F == 0) break;
      for (int s = tid; s < V; s += T)
        if (ready[s]) {
          const int p = emitted + tmp[s];
          order_s[p] = s;
          layer_s[s] = t;
          pos_of[s] = p;
          ready[s] = 0;
        }
      __syncthreads();
      for (int p = emitted + tid; p < emitted + F; p += T) {
        const int s = order_s[p];
        for (int k = outbeg[s]; k < outbeg[s] + outfill[s]; ++k) {
          const int d = outlist[k];
          if (atomicSub(&rem[d], 1) == 1) ready[d] = 1;
        }
      }
      __syncthreads();
      emitted += F;
      ++t;
    }
    if (tid == 0 && emitted < V) atomicOr(&s_status, NEAT_G_CYCLE);
  }
  __syncthreads();
  const unsigned status = s_status;
  const bool no_order = (status & ~NEAT_G_CYCLE) != 0u;

  // 6. order / layer / n_layers / status outputs (order, layer and n_layers
  // are optional in the recurrent mode)
  if (order != nullptr)
    for (int p = tid; p < N; p += T)
      order[size_t(g) * N + p] = (!no_order && p < emitted) ? row_of_s[order_s[p]] : -1;
  if (layer != nullptr)
    for (int r = tid; r < N; r += T) {
      const int s = s_of_row[r];
      layer[size_t(g) * N + r] = (!no_order && s >= 0) ? layer_s[s] : -1;
    }
  if (tid == 0) {
    if (n_layers != nullptr) n_layers[g] = no_order ? 0 : t;
    gstatus[g] = status;
  }

  // 7. padded program (valid genomes only)
  GenomeHdr h;
  h.V = 0; h.E = 0; h.L = 0; h.status = status; h.node_off = 0; h.edge_off = 0;
  h.nlive = 0; h.nch = 0; h.elive = 0; h.crows = 0; h.clayers = 0; h.cpairs = 0;
  if (status == 0u) {
    h.V = V; h.E = E; h.L = t;
    // nodes some output depends on (with pruning on, feed-forward only): the
    // outputs, then frontier by frontier from the last, the sources of every
    // such node; otherwise every node counts
    int *live = ready;     // free after the sort
    int *fstart = outbeg;  // first position of each frontier (N + 1 entries)
    const bool sweep = !recurrent && w.prune;  // else every node counts
    for (int s = tid; s < V; s += T) live[s] = sweep ? 0 : 1;
    __syncthreads();
    if (sweep) {
      for (int p = tid; p < V; p += T)
        if (p == 0 || layer_s[order_s[p]] != layer_s[order_s[p - 1]])
          fstart[layer_s[order_s[p]]] = p;
      if (tid == 0) fstart[t] = V;
      for (int i = tid; i < O; i += T) live[s_of_row[I + i]] = 1;
      __syncthreads();
      for (int l = t - 1; l >= 0; --l) {
        for (int p = fstart[l] + tid; p < fstart[l + 1]; p += T) {
          const int s = order_s[p];
          if (live[s])
            for (int k = inbeg[s]; k < inbeg[s] + indeg[s]; ++k)
              live[int((ek[k] >> 20) & 0xfffffu)] = 1;
        }
        __syncthreads();
      }
    }
    // edge begin per position; 4-edge chunk count of the level-synchronous
    // form, live nodes and their connections
    int my_nch = 0, my_nl = 0, my_el = 0;
    for (int p = tid; p < V; p += T) {
      const int s = order_s[p];
      tmp[p] = indeg[s];
      if (live[s] && row_of_s[s] >= I) {
        my_nch += (indeg[s] + 3) >> 2;
        ++my_nl;
        my_el += indeg[s];
      }
    }
    if (my_nch) atomicAdd(&s_nch, my_nch);
    if (my_nl) atomicAdd(&s_nlive, my_nl);
    if (my_el) atomicAdd(&s_elive, my_el);
    __syncthreads();
    h.nch = s_nch;
    h.nlive = s_nlive;
    h.elive = s_elive;
    block_exclusive_scan(tmp, V, wbuf);
    NodeRec *pn = w.pnode + size_t(g) * N;
    int32_t *prow = w.prow + size_t(g) * N;
    int32_t *play = w.player + size_t(g) * N;
    for (int p = tid; p < N; p += T) {
      NodeRec rec;
      play[p] = p < V ? layer_s[order_s[p]] : -1;
      if (p < V) {
        const int s = order_s[p], row = row_of_s[s];
        const float *nr = gn + row * 5;
        uint32_t meta = uint32_t(indeg[s]) | META_VALID;
        if (row < I) {
          meta |= META_INPUT;
          rec.bias = 0.0f;
          rec.resp = 1.0f;
        } else {
          meta |= (uint32_t(nr[3]) << 16) | (uint32_t(nr[4]) << 20);
          if (!live[s]) meta |= META_DEAD;
          rec.bias = nr[1];
          rec.resp = nr[2];
        }
        rec.in_begin = uint32_t(tmp[p]);
        rec.meta = meta;
        prow[p] = row;
      } else {
        rec.bias = 0.0f; rec.resp = 0.0f; rec.in_begin = 0u; rec.meta = 0u;
        prow[p] = -1;
      }
      pn[p] = rec;
    }
    EdgeRec *pe = w.pedge + size_t(g) * C;
    int32_t *per = w.perow + size_t(g) * C;
    for (int i = tid; i < E; i += T) {
      const uint64_t x = ek[i];
      const int dst = int(x >> 40), src = int((x >> 20) & 0xfffffu), row = int(x & 0xfffffu);
      const int p = pos_of[dst];
      const int idx = tmp[p] + (i - inbeg[dst]);
      EdgeRec er;
      er.src = uint32_t(pos_of[src]);
      er.w = gc[row * 4 + 2];
      pe[idx] = er;
      per[idx] = row;
    }
    int32_t *io = w.pio + size_t(g) * (I + O);
    for (int i = tid; i < I + O; i += T) io[i] = pos_of[s_of_row[i]];

    // 8. compiled program (feed-forward only): value rows by a linear scan
    if (!recurrent && w.cnode != nullptr) {
      int *cidx = tmp;       // compact index of each kept position (free again)
      int *pbeg = outbeg;    // first pair of each kept position
      int *clast = rem;      // last reader (compact index) of each value
      int *crow = outfill;   // value row of each sorted node
      int *cst = reinterpret_cast<int *>(sm + L.sk);  // released rows (sk is free)
      __syncthreads();  // tmp and outbeg are free once step 7 is done with them
      for (int p = tid; p < V; p += T) {
        const int s = order_s[p];
        const bool keep = live[s] && row_of_s[s] >= I;
        cidx[p] = keep ? 1 : 0;
        pbeg[p] = keep ? (indeg[s] + 1) >> 1 : 0;
      }
      for (int s = tid; s < V; s += T) {
        clast[s] = -1;
        crow[s] = -1;
      }
      __syncthreads();
      block_exclusive_scan(cidx, V, wbuf);
      h.cpairs = block_exclusive_scan(pbeg, V, wbuf);
      // the outputs keep their rows; every other value is released at its
      // last reader
      for (int i = tid; i < O; i += T) clast[s_of_row[I + i]] = 0x7fffffff;
      __syncthreads();
      for (int p = tid; p < V; p += T) {
        const int s = order_s[p];
        if (!live[s] || row_of_s[s] < I) continue;
        for (int k = inbeg[s]; k < inbeg[s] + indeg[s]; ++k)
          atomicMax(&clast[int((ek[k] >> 20) & 0xfffffu)], cidx[p]);
      }
      __syncthreads();
      // the values each kept position releases (its sources whose last
      // reader it is; a source feeds a node at most once), gathered in
      // parallel so that the scan itself only moves rows
      int *roff = pos_of;  // free after step 7
      int *rlist = key_s;  // free after step 2
      for (int p = tid; p < V; p += T) {
        const int s = order_s[p];
        int n = 0;
        if (live[s] && row_of_s[s] >= I)
          for (int k = inbeg[s]; k < inbeg[s] + indeg[s]; ++k) {
            const int src = int((ek[k] >> 20) & 0xfffffu);
            n += (clast[src] == cidx[p] && row_of_s[src] >= I) ? 1 : 0;
          }
        roff[p] = n;
      }
      __syncthreads();
      const int nrel = block_exclusive_scan(roff, V, wbuf);
      for (int p = tid; p < V; p += T) {
        const int s = order_s[p];
        if (!live[s] || row_of_s[s] < I) continue;
        int j = roff[p];
        for (int k = inbeg[s]; k < inbeg[s] + indeg[s]; ++k) {
          const int src = int((ek[k] >> 20) & 0xfffffu);
          if (clast[src] == cidx[p] && row_of_s[src] >= I) rlist[j++] = src;
        }
      }
      // Value rows, layer by layer: a layer's k nodes take, in canonical
      // order, the rows on top of the free stack (the i-th node the i-th row
      // from the top), then new rows; the rows its nodes release are pushed
      // (in node order) only after the layer: rows released by a layer become
      // free for later layers only, so the nodes of one layer may run at the
      // same time (the CTA-wide walk), none writing a row another one of them
      // still reads.  Layers are sequential, the nodes of a layer parallel.
      const int nn = h.nlive;
      int *kp = cst + pow2_ceil(N);  // kept position of each compact index (sk's second half)
      int *lstart = reinterpret_cast<int *>(sm + L.cls);  // [t + 1] first compact index >= layer
      __syncthreads();
      for (int i = tid; i < I; i += T) crow[s_of_row[i]] = i;
      for (int p = tid; p < V; p += T) {
        const int s = order_s[p];
        if (live[s] && row_of_s[s] >= I) kp[cidx[p]] = p;
      }
      __syncthreads();
      auto lay_k = [&](int c) { return layer_s[order_s[kp[c]]]; };
      for (int c = tid; c < nn; c += T) {
        const int lc = lay_k(c), lp = c > 0 ? lay_k(c - 1) : -1;
        for (int l = lp + 1; l <= lc; ++l) lstart[l] = c;
        if (c == nn - 1)
          for (int l = lc + 1; l <= t; ++l) lstart[l] = nn;
      }
      if (nn == 0)
        for (int l = tid; l <= t; l += T) lstart[l] = 0;
      __syncthreads();
      int sp = 0, next = I + 2;  // (every thread follows the same counts)
      for (int l = 0; l < t; ++l) {
        const int c0 = lstart[l], c1 = lstart[l + 1], k = c1 - c0;
        if (k == 0) continue;
        for (int c = c0 + tid; c < c1; c += T) {
          const int i = c - c0;
          crow[order_s[kp[c]]] = i < sp ? cst[sp - 1 - i] : next + (i - sp);
        }
        const int spa = max(0, sp - k);
        next += max(0, k - sp);
        const int pl = kp[c1 - 1];
        const int r0 = roff[kp[c0]], r1 = pl + 1 < V ? roff[pl + 1] : nrel;
        __syncthreads();  // the layer's pops are done before its pushes reuse the slots
        for (int j = r0 + tid; j < r1; j += T) cst[spa + (j - r0)] = crow[rlist[j]];
        sp = spa + (r1 - r0);
        __syncthreads();
      }
      if (tid == 0) s_crows = next;
      __syncthreads();
      h.crows = s_crows;
      CNode *cn = w.cnode + size_t(g) * N;
      uint4 *cp = w.cpair + size_t(g) * cpair_cap(N, C);
      for (int p = tid; p < V; p += T) {
        const int s = order_s[p];
        if (!live[s] || row_of_s[s] < I) continue;
        const float *nr = gn + row_of_s[s] * 5;
        const int cnt = indeg[s], act = int(nr[3]), agg = int(nr[4]), np = (cnt + 1) >> 1;
        const int pb = pbeg[p];
        CNode r;
        r.bias = nr[1];
        r.resp = nr[2];
        r.pairs = uint32_t(pb) | (uint32_t(np) << CN_PAIR_BITS);
        r.meta = uint32_t(crow[s]) | (uint32_t(act) << CN_ROW_BITS) |
                 (uint32_t(agg) << (CN_ROW_BITS + 3)) | (uint32_t(cnt & 1) << (CN_ROW_BITS + 5));
        cn[cidx[p]] = r;
        for (int q = 0; q < np; ++q) {
          const uint64_t x0 = ek[inbeg[s] + 2 * q];
          uint4 e;
          e.x = uint32_t(crow[int((x0 >> 20) & 0xfffffu)]);
          e.y = __float_as_uint(gc[int(x0 & 0xfffffu) * 4 + 2]);
          if (2 * q + 1 < cnt) {
            const uint64_t x1 = ek[inbeg[s] + 2 * q + 1];
            e.z = uint32_t(crow[int((x1 >> 20) & 0xfffffu)]);
            e.w = __float_as_uint(gc[int(x1 & 0xfffffu) * 4 + 2]);
          } else if (agg == NEAT_AGG_MAX) {
            e.z = e.x;
            e.w = e.y;
          } else if (agg == NEAT_AGG_PRODUCT) {
            e.z = uint32_t(I + 1);
            e.w = __float_as_uint(1.0f);
          } else {
            e.z = uint32_t(I);
            e.w = 0u;
          }
          cp[pb + q] = e;
        }
      }
      for (int i = tid; i < O; i += T) w.cout[size_t(g) * O + i] = crow[s_of_row[I + i]];
      // first compiled node of each layer that holds any (compact indices
      // follow the canonical order, so a layer's nodes are contiguous)
      __syncthreads();
      if (tid == 0) {
        int32_t *cl = w.clay + size_t(g) * (N + 1);
        int nl = 0;
        for (int l = 0; l < t; ++l)
          if (lstart[l] < lstart[l + 1]) cl[nl++] = lstart[l];
        cl[nl] = nn;
        s_crows = nl;  // (reused: the compiled layer count)
      }
      __syncthreads();
      h.clayers = s_crows;
    }
  }
  if (tid == 0) w.hdr[g] = h;
}

// Work-queue order: genomes by descending cost (ties: lower id first).
// mode 0: cost = E + 2V of the whole genome (sample-parallel forms and the
// backward; measured better than the live part's cost for the compiled walk
// too); mode 1: layers first, then E.
__device__ __forceinline__ uint64_t cost_key(const GenomeHdr &h, int mode, int g) {
  uint32_t cost;
  if (h.status != 0u) cost = 0u;
  else if (mode == 0) cost = uint32_t(h.E + 2 * h.V + 1);
  else cost = (uint32_t(h.L) << 16) | uint32_t(min(h.E, 0xffff));
  return (uint64_t(cost) << 32) | uint64_t(0xffffffffu - uint32_t(g));
}

// Rank of a genome = the number of keys above its own (keys are distinct).  A
// CTA ranks 32 genomes (lane = genome); its 8 warps split every 1024-key tile
// of the population (each thread loads four of its keys, independent loads),
// 128 keys each, and the 8 partial counts are summed: 1/8 of the comparisons
// per thread and few dependent load rounds.
constexpr int RANK_GENOMES = 32, RANK_SPLIT = 8, RANK_TILE = 1024;

__global__ void __launch_bounds__(RANK_GENOMES * RANK_SPLIT) k_rank(Ws w, int mode,
                                                                    int32_t *__restrict__ qout) {
  constexpr int T = RANK_GENOMES * RANK_SPLIT, PER = RANK_TILE / T, SLICE = RANK_TILE / RANK_SPLIT;
  __shared__ uint64_t tile[RANK_TILE];
  __shared__ int part[RANK_SPLIT][RANK_GENOMES];
  const int P = w.P;
  const int gl = threadIdx.x & (RANK_GENOMES - 1), sl = threadIdx.x / RANK_GENOMES;
  const int g = blockIdx.x * RANK_GENOMES + gl;
  const uint64_t kg = g < P ? cost_key(w.hdr[g], mode, g) : 0ull;
  int rank = 0;
  for (int base = 0; base < P; base += RANK_TILE) {
    uint64_t k[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int h = base + j * T + int(threadIdx.x);
      k[j] = h < P ? cost_key(w.hdr[h], mode, h) : 0ull;  // 0: below every key
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) tile[j * T + threadIdx.x] = k[j];
    __syncthreads();
    const uint64_t *t = tile + sl * SLICE;
#pragma unroll 16
    for (int i = 0; i < SLICE; ++i) rank += t[i] > kg;
    __syncthreads();
  }
  part[sl][gl] = rank;
  __syncthreads();
  if (sl == 0 && g < P) {
    int r = 0;
#pragma unroll
    for (int i = 0; i < RANK_SPLIT; ++i) r += part[i][gl];
    qout[r] = g;
  }
}

// Exclusive scans of V and E in queue order -> ragged offsets (one CTA).
__global__ void __launch_bounds__(1024) k_offsets(Ws w) {
  __shared__ int wv[33], we[33];
  __shared__ int nbig;
  const int P = w.P, T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (P + T - 1) / T;
  const int b = min(tid * per, P), e = min(b + per, P);
  if (tid == 0) nbig = 0;
  __syncthreads();
  int sv = 0, se = 0, sb = 0;
  for (int q = b; q < e; ++q) {
    const GenomeHdr h = w.hdr[w.qorder[q]];
    sv += h.V;
    se += h.E;
    // the most expensive genomes (a prefix of the cost-sorted queue) go to
    // whole CTAs in the sample-parallel forward
    sb += (h.status == 0u && sp_cost(h) >= sp_coop_cost(w.prune != 0)) ? 1 : 0;
  }
  if (sb) atomicAdd(&nbig, sb);
  int xv = sv, xe = se;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int yv = __shfl_up_sync(0xffffffffu, xv, d), ye = __shfl_up_sync(0xffffffffu, xe, d);
    if (lane >= d) { xv += yv; xe += ye; }
  }
  if (lane == 31) { wv[wid] = xv; we[wid] = xe; }
  __syncthreads();
  if (wid == 0) {
    int a = wv[lane], c = we[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int ya = __shfl_up_sync(0xffffffffu, a, d), yc = __shfl_up_sync(0xffffffffu, c, d);
      if (lane >= d) { a += ya; c += yc; }
    }
    wv[lane] = a;
    we[lane] = c;
  }
  __syncthreads();
  if (tid == 0) w.counters[CTR_SP_NBIG] = uint32_t(nbig);
  int ov = (wid > 0 ? wv[wid - 1] : 0) + xv - sv;
  int oe = (wid > 0 ? we[wid - 1] : 0) + xe - se;
  for (int q = b; q < e; ++q) {
    const int g = w.qorder[q];
    GenomeHdr h = w.hdr[g];
    h.node_off = ov;
    h.edge_off = oe;
    ov += h.V;
    oe += h.E;
    w.hdr[g] = h;
  }
}

// Copy the padded programs into the ragged-packed arena.
__global__ void __launch_bounds__(128) k_pack(Ws w) {
  const int g = blockIdx.x;
  const GenomeHdr h = w.hdr[g];
  const NodeRec *pn = w.pnode + size_t(g) * w.N;
  const EdgeRec *pe = w.pedge + size_t(g) * w.C;
  const int32_t *per = w.perow + size_t(g) * w.C;
  for (int p = threadIdx.x; p < h.V; p += blockDim.x) w.knode[h.node_off + p] = pn[p];
  for (int i = threadIdx.x; i < h.E; i += blockDim.x) {
    w.kedge[h.edge_off + i] = pe[i];
    w.kerow[h.edge_off + i] = per[i];
  }
}

}  // namespace

cudaError_t launch_transform(const Ws &w, const float *nodes, const float *conns, int32_t *order,
                             int32_t *layer, int32_t *n_layers, uint32_t *gstatus,
                             cudaStream_t st, int recurrent) {
  if (w.P == 0) return cudaSuccess;
  const TSmem L = tsmem_layout(w.N, w.C);
  // 4 warps per genome up to N + C = 1024 (measured on 10,000 genomes of
  // N = 128, C = 512: 525 us against 650 us with 8 warps and 670 us with one
  // warp a genome), 8 warps for larger genomes (1.15 ms against 1.44 ms on
  // 4,000 genomes of N = 1024, C = 4096)
  const int threads = w.N + w.C <= 1024 ? 128 : 256;
  k_transform<<<w.P, threads, L.total, st>>>(w, nodes, conns, order, layer, n_layers, gstatus,
                                             recurrent);
  return cudaGetLastError();
}

cudaError_t launch_queue_build(const Ws &w, int mode, cudaStream_t st) {
  if (w.P == 0) return cudaSuccess;
  (void)mode;
  // size-sorted queue (sample-parallel forms, packing order) and
  // layer-sorted queue (level-synchronous batches)
  const int rank_ctas = (w.P + RANK_GENOMES - 1) / RANK_GENOMES;
  k_rank<<<rank_ctas, RANK_GENOMES * RANK_SPLIT, 0, st>>>(w, 0, w.qorder);
  k_rank<<<rank_ctas, RANK_GENOMES * RANK_SPLIT, 0, st>>>(w, 1, w.qlvl);
  k_offsets<<<1, 1024, 0, st>>>(w);
  k_pack<<<w.P, 128, 0, st>>>(w);
  return cudaGetLastError();
}

}  // namespace neat

namespace neat {
cudaError_t transform_set_smem_limit(int bytes) {
  return set_dyn_smem_limit(k_transform, bytes);
}
size_t transform_smem(int N, int C) { return size_t(tsmem_layout(N, C).total); }
}  // namespace neat
