// Population-wide compatibility distance between genomes, the quantity
// TensorNEAT's Alg. 1 divides the population by (App. A names its disjoint
// and homologous coefficients).  For genomes A and B:
//   delta = node term + connection term, each (c_d D + c_h H) / max(n_A, n_B)
// (0 when both counts are 0).  Node genes: valid node rows keyed by node key;
// connection genes: valid connection rows (enabled or not) keyed by
// (in key, out key), the lowest row of a repeated key counting once.  D
// counts the keys present in exactly one genome; H sums over shared keys
// |b_A - b_B| + |r_A - r_B| + [act differs] + [agg differs] for nodes (0 when
// either row is an input row) and |w_A - w_B| + [enabled differs] for
// connections.  A genome with a status bit other than CYCLE gets NaN.
//
//  k_dist_prep  one CTA per genome: sorts its node genes by key and its
//               connection genes by (in, out, row) in shared memory (bitonic),
//               drops repeated connection keys, writes the sorted gene lists
//               and their key arrays
//  k_dist_hist, k_dist_scan, k_dist_scatter
//               a counting sort of the genomes by connection-gene count, so
//               that the pairs of a warp have genomes of like sizes and their
//               merge loops run about equally long
//  k_distance   one thread per unordered pair (16 x 16 pairs per CTA, tiles
//               on or above the diagonal, genomes taken in that size order):
//               merges the two pairs of sorted key arrays (keys compared as
//               order-preserving integers, so exactly like the float values)
//               and writes both entries of the symmetric matrix
#include <cuda_runtime.h>

#include <cstdint>

#include "neat_internal.cuh"

namespace neat {
namespace {

// node gene: order-preserving key, bias, response, act | agg << 8 | input << 16
struct __align__(16) NodeGene {
  uint32_t key;
  float bias;
  float resp;
  uint32_t meta;
};
// connection gene: order-preserving in / out keys, weight, enabled flag
struct __align__(16) ConnGene {
  uint32_t kin;
  uint32_t kout;
  float w;
  uint32_t en;
};

constexpr uint32_t KEY_END = 0xffffffffu;  // above every finite key's encoding

// float -> uint32 with the same order (finite values; -0 and +0 are equal)
__device__ __forceinline__ uint32_t ord_key(float x) {
  if (x == 0.0f) x = 0.0f;
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ int pow2_ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Exclusive prefix sum of flags[0..n) in place (one CTA), returns the total.
__device__ int cta_scan(int *flags, int n, int *wsum) {
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int per = (n + T - 1) / T, b = min(tid * per, n), e = min(b + per, n);
  int s = 0;
  for (int i = b; i < e; ++i) s += flags[i];
  int x = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int a = lane < (T >> 5) ? wsum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, a, d);
      if (lane >= d) a += y;
    }
    wsum[lane] = a;
  }
  __syncthreads();
  int run = (wid > 0 ? wsum[wid - 1] : 0) + x - s;
  const int total = wsum[(T >> 5) - 1];
  for (int i = b; i < e; ++i) {
    const int f = flags[i];
    flags[i] = run;
    run += f;
  }
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(256) k_dist_prep(const float *__restrict__ nodes,
                                                   const float *__restrict__ conns,
                                                   const uint32_t *__restrict__ gstatus, int N,
                                                   int C, int I, NodeGene *__restrict__ ng,
                                                   ConnGene *__restrict__ cg,
                                                   uint32_t *__restrict__ nkey,
                                                   uint64_t *__restrict__ ckey,
                                                   int4 *__restrict__ counts) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int g = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int N2 = pow2_ceil(N), C2 = pow2_ceil(C);
  uint64_t *nk = reinterpret_cast<uint64_t *>(sm);  // [N2] key << 32 | row
  uint64_t *ck = nk + N2;                           // [C2] in << 32 | out
  uint32_t *cr = reinterpret_cast<uint32_t *>(ck + C2);  // [C2] row
  int *flag = reinterpret_cast<int *>(cr + C2);          // [C2]
  __shared__ int wsum[32];
  __shared__ int s_n;
  const float *gn = nodes + size_t(g) * N * 5;
  const float *gc = conns + size_t(g) * C * 4;
  if (tid == 0) s_n = 0;
  __syncthreads();

  // node genes by key
  int my_n = 0;
  for (int r = tid; r < N2; r += T) {
    const bool valid = r < N && !isnan(gn[r * 5]);
    nk[r] = valid ? (uint64_t(ord_key(gn[r * 5])) << 32) | uint32_t(r) : ~0ull;
    my_n += valid;
  }
  if (my_n) atomicAdd(&s_n, my_n);
  // connection genes by (in, out), ties by row
  for (int r = tid; r < C2; r += T) {
    const bool valid = r < C && !isnan(gc[r * 4]) && !isnan(gc[r * 4 + 1]);
    ck[r] = valid ? (uint64_t(ord_key(gc[r * 4])) << 32) | ord_key(gc[r * 4 + 1]) : ~0ull;
    cr[r] = valid ? uint32_t(r) : 0xffffffffu;
  }
  __syncthreads();
  for (int k = 2; k <= N2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < N2; i += T) {
        const int l = i ^ j;
        if (l > i) {
          const uint64_t x = nk[i], y = nk[l];
          if (((i & k) == 0) == (x > y)) { nk[i] = y; nk[l] = x; }
        }
      }
      __syncthreads();
    }
  for (int k = 2; k <= C2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < C2; i += T) {
        const int l = i ^ j;
        if (l > i) {
          const uint64_t x = ck[i], y = ck[l];
          const uint32_t xr = cr[i], yr = cr[l];
          const bool gt = x > y || (x == y && xr > yr);
          if (((i & k) == 0) == gt) {
            ck[i] = y; ck[l] = x;
            cr[i] = yr; cr[l] = xr;
          }
        }
      }
      __syncthreads();
    }
  const int n = s_n;
  for (int i = tid; i < n; i += T) {
    const int r = int(nk[i] & 0xffffffffu);
    const float *row = gn + r * 5;
    NodeGene q;
    q.key = uint32_t(nk[i] >> 32);
    q.bias = row[1];
    q.resp = row[2];
    // ids of non-input rows (integral and in range unless the genome is bad)
    const uint32_t act = r >= I ? uint32_t(int(row[3]) & 0xff) : 0xffu;
    const uint32_t agg = r >= I ? uint32_t(int(row[4]) & 0xff) : 0xffu;
    q.meta = act | (agg << 8) | (uint32_t(r < I) << 16);
    ng[size_t(g) * N + i] = q;
    nkey[size_t(g) * N + i] = q.key;
  }
  // first row of every (in, out) key
  for (int i = tid; i < C; i += T)
    flag[i] = (cr[i] != 0xffffffffu && (i == 0 || ck[i] != ck[i - 1])) ? 1 : 0;
  __syncthreads();
  // keep = flag before the scan overwrites it
  for (int i = tid; i < C; i += T) cr[i] = flag[i] ? cr[i] : 0xffffffffu;
  __syncthreads();
  const int m = cta_scan(flag, C, wsum);
  for (int i = tid; i < C; i += T) {
    if (cr[i] == 0xffffffffu) continue;
    const float *row = gc + cr[i] * 4;
    ConnGene q;
    q.kin = uint32_t(ck[i] >> 32);
    q.kout = uint32_t(ck[i] & 0xffffffffu);
    q.w = row[2];
    q.en = (!isnan(row[3]) && row[3] != 0.0f) ? 1u : 0u;
    cg[size_t(g) * C + flag[i]] = q;
    ckey[size_t(g) * C + flag[i]] = uint64_t(q.kin) << 32 | q.kout;
  }
  if (tid == 0) {
    const bool bad = gstatus != nullptr && (gstatus[g] & ~uint32_t(NEAT_G_CYCLE)) != 0u;
    counts[g] = make_int4(n, m, bad ? 1 : 0, 0);
  }
}

__device__ __forceinline__ NodeGene ld_ng(const NodeGene *p) {
  const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
  NodeGene q;
  q.key = x.x; q.bias = __uint_as_float(x.y); q.resp = __uint_as_float(x.z); q.meta = x.w;
  return q;
}
__device__ __forceinline__ ConnGene ld_cg(const ConnGene *p) {
  const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
  ConnGene q;
  q.kin = x.x; q.kout = x.y; q.w = __uint_as_float(x.z); q.en = x.w;
  return q;
}

// One thread per pair, 16 x 16 pairs per CTA.  The merges step through the
// genomes' sorted key arrays (node keys 4 B, connection keys 8 B, L1-cached),
// loading only the key of the side that advances; a shared key loads both
// genes' attributes for the homologous term.  The sums run in key order, as
// in the record merge: the same bits, d(a, b) = d(b, a).
// size bucket of a genome: its connection-gene count (0 for a malformed one)
__device__ __forceinline__ int dist_bucket(const int4 c, int C) { return c.z ? 0 : min(c.y, C); }

__global__ void __launch_bounds__(256) k_dist_hist(const int4 *__restrict__ counts, int P, int C,
                                                   int *__restrict__ hist) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < P) atomicAdd(hist + dist_bucket(counts[g], C), 1);
}

// exclusive scan of the C + 1 bucket counts in place (one CTA)
__global__ void __launch_bounds__(1024) k_dist_scan(int *hist, int n) {
  __shared__ int wsum[32];
  cta_scan(hist, n, wsum);
}

// perm[k] = the genome at size rank k (the order inside a bucket is that of
// the atomics; the distances do not depend on it)
__global__ void __launch_bounds__(256) k_dist_scatter(const int4 *__restrict__ counts, int P,
                                                      int C, int *__restrict__ hist,
                                                      int *__restrict__ perm) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < P) perm[atomicAdd(hist + dist_bucket(counts[g], C), 1)] = g;
}

__global__ void __launch_bounds__(256) k_distance(const NodeGene *__restrict__ ng,
                                                  const ConnGene *__restrict__ cg,
                                                  const uint32_t *__restrict__ nkey,
                                                  const uint64_t *__restrict__ ckey,
                                                  const int4 *__restrict__ counts,
                                                  const int *__restrict__ perm, int P, int N,
                                                  int C, float cd, float ch,
                                                  float *__restrict__ dist) {
  // the merge is symmetric in its two genomes (the same keys in the same
  // order, |x - y| = |y - x|): only tiles on or above the diagonal run, and
  // each pair writes both of its entries
  if (blockIdx.y > blockIdx.x) return;
  const int rb = blockIdx.x * 16 + threadIdx.x, ra = blockIdx.y * 16 + threadIdx.y;
  if (ra >= P || rb >= P || rb < ra) return;
  const int a = __ldg(perm + ra), b = __ldg(perm + rb);
  const int4 ca = __ldg(counts + a), cb = __ldg(counts + b);
  float d = qnan();
  if (!ca.z && !cb.z) {
    // nodes
    const uint32_t *A = nkey + size_t(a) * N, *B = nkey + size_t(b) * N;
    const NodeGene *GA = ng + size_t(a) * N, *GB = ng + size_t(b) * N;
    int i = 0, j = 0, D = 0;
    float H = 0.0f;
    uint32_t kx = ca.x > 0 ? __ldg(A) : KEY_END, ky = cb.x > 0 ? __ldg(B) : KEY_END;
    while (kx != KEY_END || ky != KEY_END) {
      if (kx == ky) {
        const NodeGene x = ld_ng(GA + i), y = ld_ng(GB + j);
        if (!((x.meta | y.meta) & 0x10000u))
          H += fabsf(x.bias - y.bias) + fabsf(x.resp - y.resp) +
               float((x.meta & 0xffu) != (y.meta & 0xffu)) +
               float(((x.meta >> 8) & 0xffu) != ((y.meta >> 8) & 0xffu));
        ++i;
        ++j;
        kx = i < ca.x ? __ldg(A + i) : KEY_END;
        ky = j < cb.x ? __ldg(B + j) : KEY_END;
      } else {
        ++D;
        if (kx < ky) {
          ++i;
          kx = i < ca.x ? __ldg(A + i) : KEY_END;
        } else {
          ++j;
          ky = j < cb.x ? __ldg(B + j) : KEY_END;
        }
      }
    }
    const int nmax = max(ca.x, cb.x);
    d = nmax > 0 ? (cd * float(D) + ch * H) / float(nmax) : 0.0f;
    // connections
    const uint64_t *X = ckey + size_t(a) * C, *Y = ckey + size_t(b) * C;
    const ConnGene *CX = cg + size_t(a) * C, *CY = cg + size_t(b) * C;
    i = 0; j = 0; D = 0; H = 0.0f;
    uint64_t qx = ca.y > 0 ? __ldg(X) : ~0ull, qy = cb.y > 0 ? __ldg(Y) : ~0ull;
    while (qx != ~0ull || qy != ~0ull) {
      if (qx == qy) {
        const ConnGene x = ld_cg(CX + i), y = ld_cg(CY + j);
        H += fabsf(x.w - y.w) + float(x.en != y.en);
        ++i;
        ++j;
        qx = i < ca.y ? __ldg(X + i) : ~0ull;
        qy = j < cb.y ? __ldg(Y + j) : ~0ull;
      } else {
        ++D;
        if (qx < qy) {
          ++i;
          qx = i < ca.y ? __ldg(X + i) : ~0ull;
        } else {
          ++j;
          qy = j < cb.y ? __ldg(Y + j) : ~0ull;
        }
      }
    }
    const int mmax = max(ca.y, cb.y);
    if (mmax > 0) d += (cd * float(D) + ch * H) / float(mmax);
  }
  dist[size_t(a) * P + b] = d;
  dist[size_t(b) * P + a] = d;
}

size_t prep_smem(int N, int C) {
  int N2 = 1, C2 = 1;
  while (N2 < N) N2 <<= 1;
  while (C2 < C) C2 <<= 1;
  return size_t(N2) * 8 + size_t(C2) * (8 + 4 + 4);
}

struct DistLayout {
  size_t ng, cg, nkey, ckey, counts, hist, perm, total;
};
DistLayout dist_layout(int P, int N, int C) {
  DistLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) / 256 * 256; return o; };
  L.ng = take(sizeof(NodeGene) * size_t(P) * N);
  L.cg = take(sizeof(ConnGene) * size_t(P) * C);
  L.nkey = take(sizeof(uint32_t) * size_t(P) * N);
  L.ckey = take(sizeof(uint64_t) * size_t(P) * C);
  L.counts = take(sizeof(int4) * size_t(P));
  L.hist = take(sizeof(int) * size_t(C + 1));
  L.perm = take(sizeof(int) * size_t(P));
  L.total = off;
  return L;
}

}  // namespace
}  // namespace neat

extern "C" size_t neat_distance_scratch_bytes(int P, int N, int C) {
  if (P < 0 || N < 1 || N > NEAT_MAX_NODES || C < 1 || C > NEAT_MAX_CONNS) return 0;
  return neat::dist_layout(P, N, C).total;
}

extern "C" neat_status neat_distance(const float *nodes, const float *conns,
                                     const uint32_t *gstatus, int P, int N, int C, int I, int O,
                                     float c_disjoint, float c_homologous, float *dist,
                                     void *scratch, size_t scratch_bytes, cudaStream_t stream) {
  if (P < 0 || N < 1 || N > NEAT_MAX_NODES || C < 1 || C > NEAT_MAX_CONNS || I < 1 || O < 1 ||
      N < I + O)
    return NEAT_ERR_UNSUPPORTED;
  if (P == 0) return NEAT_OK;
  if (int64_t(P) * P > (int64_t(1) << 40)) return NEAT_ERR_UNSUPPORTED;
  if (nodes == nullptr || conns == nullptr || dist == nullptr || scratch == nullptr ||
      (reinterpret_cast<uintptr_t>(nodes) % 4) != 0 || (reinterpret_cast<uintptr_t>(conns) % 4) != 0 ||
      (reinterpret_cast<uintptr_t>(dist) % 4) != 0 ||
      (reinterpret_cast<uintptr_t>(scratch) % 256) != 0 ||
      (gstatus != nullptr && (reinterpret_cast<uintptr_t>(gstatus) % 4) != 0))
    return NEAT_ERR_ARG;
  const neat::DistLayout L = neat::dist_layout(P, N, C);
  if (scratch_bytes < L.total) return NEAT_ERR_WORKSPACE;
  char *base = static_cast<char *>(scratch);
  auto *ng = reinterpret_cast<neat::NodeGene *>(base + L.ng);
  auto *cg = reinterpret_cast<neat::ConnGene *>(base + L.cg);
  auto *nkey = reinterpret_cast<uint32_t *>(base + L.nkey);
  auto *ckey = reinterpret_cast<uint64_t *>(base + L.ckey);
  auto *counts = reinterpret_cast<int4 *>(base + L.counts);
  auto *hist = reinterpret_cast<int *>(base + L.hist);
  auto *perm = reinterpret_cast<int *>(base + L.perm);
  const size_t smem = neat::prep_smem(N, C);
  if (cudaFuncSetAttribute(neat::k_dist_prep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(smem)) != cudaSuccess)
    return NEAT_ERR_UNSUPPORTED;
  neat::k_dist_prep<<<P, 256, smem, stream>>>(nodes, conns, gstatus, N, C, I, ng, cg, nkey, ckey,
                                               counts);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(int) * size_t(C + 1), stream);
  if (e != cudaSuccess) return neat::cuda_error_status(e);
  const unsigned gb = unsigned((P + 255) / 256);
  neat::k_dist_hist<<<gb, 256, 0, stream>>>(counts, P, C, hist);
  neat::k_dist_scan<<<1, 1024, 0, stream>>>(hist, C + 1);
  neat::k_dist_scatter<<<gb, 256, 0, stream>>>(counts, P, C, hist, perm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return neat::cuda_error_status(e);
  const dim3 grid(unsigned((P + 15) / 16), unsigned((P + 15) / 16)), block(16, 16);
  neat::k_distance<<<grid, block, 0, stream>>>(ng, cg, nkey, ckey, counts, perm, P, N, C,
                                               c_disjoint, c_homologous, dist);
  return neat::cuda_error_status(cudaGetLastError());
}
