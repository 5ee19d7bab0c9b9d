/*
 * FP64 CPU oracle for tensorized NEAT network evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  It shares no code, header, table
 * or constant with the CUDA library; only tests, the smoke check and the
 * benchmark's CPU-baseline / reference legs load it.
 *
 * What it follows (TensorNEAT, arXiv 2504.08339):
 *   - Sec. 3.1 "Tensorized Encodings": a node row is (k, attrs...), a
 *     connection row (k_in, k_out, e, attrs...); padding rows are NaN.
 *     Column layout used here: nodes[P,N,5] = (key, bias, response, act, agg),
 *     conns[P,C,4] = (in key, out key, weight, enabled).
 *   - Sec. 3.3 "Tensorized Network Inference", transformation stage: a
 *     topological order N_order of the nodes; the expanded connections C_exp
 *     keep an attribute entry for every enabled connection (e = 1) and mark
 *     disabled ones absent (e = 0).  Here that is a per-node list of enabled
 *     incoming connections.
 *   - Sec. 3.3, calculation stage: v starts undefined, v[input] <- I, then in
 *     N_order each node takes v[k] = f_n(f_c(v | C_exp[:,k]) | node attrs)
 *     with f_c(x | w) = w x and f_n(x | b, agg, act) = act(agg(x) + b);
 *     O = v[output].
 *   - App. B genome interface: input_idx = arange(I), output_idx =
 *     arange(I, I+O) -> inputs are node ROWS 0..I-1, outputs rows I..I+O-1.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1 response: f_n = act(b + r * agg(x)); reduces to the paper's form at r=1.
 *   R2 a row is padding iff a key column is NaN; enabled iff e is not NaN and
 *      e != 0.
 *   R3 keys are arbitrary unique integers in [0, 2^24) resolved by lookup.
 *   R4 topological tie rule: Kahn by frontier, each frontier emitted in
 *      ascending key; the frontier index is the node's layer.
 *   R5 empty aggregation gives 0 for every aggregation (orphan nodes take
 *      act(b)).
 *   R6 activations are the unscaled textbook forms; max aggregation is an
 *      fmax fold (NaN-ignoring).
 *   R7 malformed genomes get status bits; a genome with any bit other than
 *      CYCLE gets no order at all (order/layer -1); a cyclic genome keeps the
 *      order and layers of the nodes Kahn emitted.  A genome with any status
 *      bit produces NaN outputs and zero gradients.
 *   R8 gradients (the paper has none): reverse mode over the same order;
 *      relu'(0) = abs'(0) = 0; a max node passes its gradient to the first
 *      incoming connection (ascending row) that attains the max.
 *   R9 HyperNEAT query: cell c = j*G + i has coordinates
 *      (-1 + 2i/(G-1), -1 + 2j/(G-1)); query (s, d) feeds
 *      (x_s, y_s, x_d, y_d, 1); the stored weight is o if |o| > thresh else 0.
 *   R14 HyperNEAT substrate (the paper names HyperNEAT, Sec. 2 and Sec. 4,
 *      without a substrate): the two-sheet ("sandwich") substrate of the
 *      query's grid, an input sheet and an output sheet of G^2 cells each;
 *      the query's weight w[s][t] connects input cell s to output cell t;
 *      for an input pattern x, y_t = act(sum_s w[s][t] x_s) (no bias), with
 *      the substrate activation act a parameter.
 *   R13 tensorized operations (Sec. 3.2): a list of K operations per genome,
 *      applied in order.  Each is 8 floats (kind, row, v0..v5):
 *        1 add node:  nodes[r] = (v0..v4) at r = the first row whose key is NaN
 *        2 remove node: nodes[row] = NaN (all columns)
 *        3 add connection: conns[r] = (v0..v3) at r = the first row with a
 *          NaN key column
 *        4 remove connection: conns[row] = NaN
 *        5 set node attribute: nodes[row][v0] = v1 (column 1..4)
 *        6 set connection attribute: conns[row][v0] = v1 (column 2..3)
 *        0 (or any other kind): nothing
 *      An operation with no free row, a row out of range or a column out of
 *      range changes nothing and sets bit k (k < 32) of the genome's op status.
 *   R12 compatibility distance (Alg. 1 divides the population by distances;
 *      App. A names the disjoint / homologous coefficients without the
 *      formula): delta(A,B) = node term + connection term, each
 *      (c_d * D + c_h * H) / max(count_A, count_B) (0 when both counts are 0).
 *      Node genes are the valid node rows keyed by node key; connection genes
 *      the valid connection rows (enabled or not) keyed by (in key, out key),
 *      the lowest row of a repeated key counting once.  D counts the keys in
 *      exactly one genome; H sums over shared keys |b_A - b_B| + |r_A - r_B|
 *      + [act differs] + [agg differs] for nodes (0 when either row is an
 *      input row) and |w_A - w_B| + [enabled differs] for connections.  A
 *      genome with a status bit other than CYCLE has NaN distances.
 *   R11 recurrent ("concurrent", Sec. 3.3 names the network type without
 *      its calculation): T synchronous iterations; v^0 = inputs on the input
 *      rows and 0 elsewhere; in iteration t every valid non-input node takes
 *      act(b + r * agg(w * v^{t-1}[src])) while the inputs stay clamped; the
 *      outputs are v^T.  Cycles and self-loops are allowed (no CYCLE bit).
 *
 * All arithmetic is double precision.  The forward can also return a first
 * order bound on the error an fp32 evaluation of the same network may make
 * (unit roundoff 2^-24, any summation order); it is test tolerance machinery.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* activation / aggregation ids carried in node columns 3 and 4 */
#define A_IDENTITY 0
#define A_SIGMOID 1
#define A_TANH 2
#define A_RELU 3
#define A_SIN 4
#define A_GAUSS 5
#define A_ABS 6
#define N_ACTS 7
#define G_SUM 0
#define G_PRODUCT 1
#define G_MAX 2
#define G_MEAN 3
#define N_AGGS 4

/* per-genome status bits */
#define ST_CYCLE 1u
#define ST_DANGLING_KEY 2u
#define ST_DUP_KEY 4u
#define ST_DUP_EDGE 8u
#define ST_EDGE_INTO_INPUT 16u
#define ST_BAD_ATTR 32u
#define ST_IO_ROW_INVALID 64u

#define KEY_LIMIT 16777216.0 /* 2^24 */

typedef struct {
  int N, C, I, O;
  /* nodes, indexed by row */
  int *valid;
  double *key, *bias, *resp;
  int *act, *agg;
  int V;
  /* enabled, resolved connections in ascending row order */
  int ne;
  int *esrc, *edst, *erow; /* src/dst are node rows */
  double *ew;
  /* incoming lists: for node row r, edges in_list[in_beg[r] .. in_beg[r+1]) (indices into e*) */
  int *in_beg, *in_list;
  /* outgoing lists, same layout */
  int *out_beg, *out_list;
  /* valid nodes sorted by (key, row), for key lookup */
  double *skey;
  int *srow;
  uint32_t status;
  /* transform result */
  int nord, nlayers;
  int *order; /* rows in N_order, nord of them */
  int *layer; /* per row, -1 if not emitted */
} genome_t;

static void g_free(genome_t *g) {
  free(g->valid); free(g->key); free(g->bias); free(g->resp); free(g->act); free(g->agg);
  free(g->esrc); free(g->edst); free(g->erow); free(g->ew);
  free(g->in_beg); free(g->in_list); free(g->order); free(g->layer);
  free(g->out_beg); free(g->out_list); free(g->skey); free(g->srow);
  memset(g, 0, sizeof(*g));
}

static int g_alloc(genome_t *g, int N, int C, int I, int O) {
  memset(g, 0, sizeof(*g));
  g->N = N; g->C = C; g->I = I; g->O = O;
  g->valid = calloc((size_t)N + 1, sizeof(int));
  g->key = calloc((size_t)N + 1, sizeof(double));
  g->bias = calloc((size_t)N + 1, sizeof(double));
  g->resp = calloc((size_t)N + 1, sizeof(double));
  g->act = calloc((size_t)N + 1, sizeof(int));
  g->agg = calloc((size_t)N + 1, sizeof(int));
  g->esrc = calloc((size_t)C + 1, sizeof(int));
  g->edst = calloc((size_t)C + 1, sizeof(int));
  g->erow = calloc((size_t)C + 1, sizeof(int));
  g->ew = calloc((size_t)C + 1, sizeof(double));
  g->in_beg = calloc((size_t)N + 2, sizeof(int));
  g->in_list = calloc((size_t)C + 1, sizeof(int));
  g->order = calloc((size_t)N + 1, sizeof(int));
  g->layer = calloc((size_t)N + 1, sizeof(int));
  g->out_beg = calloc((size_t)N + 2, sizeof(int));
  g->out_list = calloc((size_t)C + 1, sizeof(int));
  g->skey = calloc((size_t)N + 1, sizeof(double));
  g->srow = calloc((size_t)N + 1, sizeof(int));
  if (!g->out_beg || !g->out_list || !g->skey || !g->srow || !g->valid || !g->key || !g->bias || !g->resp || !g->act || !g->agg || !g->esrc ||
      !g->edst || !g->erow || !g->ew || !g->in_beg || !g->in_list || !g->order || !g->layer) {
    g_free(g);
    return -1;
  }
  return 0;
}

static int is_int_in(double x, double lo, double hi_excl) {
  return !isnan(x) && x == floor(x) && x >= lo && x < hi_excl;
}

/* row of the valid node with this key (lowest row if several), or -1:
 * binary search in the (key, row)-sorted list of valid nodes */
static int find_row(const genome_t *g, double key) {
  int lo = 0, hi = g->V; /* first index with skey >= key */
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (g->skey[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < g->V && g->skey[lo] == key) ? g->srow[lo] : -1;
}

typedef struct { double a, b; int i; } pair_t;
static int cmp_pair(const void *x, const void *y) {
  const pair_t *p = x, *q = y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return p->i - q->i;
}

/* Sec. 3.1 decoding of one padded genome plus the validity checks (R2, R3, R7). */
static void parse_genome(genome_t *g, const double *nodes, const double *conns) {
  const int N = g->N > 0 ? g->N : 0, C = g->C, I = g->I, O = g->O;
  g->status = 0;
  g->V = 0;
  for (int r = 0; r < N; ++r) {
    const double *row = nodes + (size_t)r * 5;
    double k = row[0];
    g->valid[r] = !isnan(k);
    g->key[r] = k;
    g->bias[r] = row[1];
    g->resp[r] = row[2];
    g->act[r] = -1;
    g->agg[r] = -1;
    if (!g->valid[r]) continue;
    g->V++;
    if (!is_int_in(k, 0.0, KEY_LIMIT)) g->status |= ST_BAD_ATTR;
    if (r >= I) { /* attributes of input rows are never used */
      if (is_int_in(row[3], 0.0, N_ACTS)) g->act[r] = (int)row[3]; else g->status |= ST_BAD_ATTR;
      if (is_int_in(row[4], 0.0, N_AGGS)) g->agg[r] = (int)row[4]; else g->status |= ST_BAD_ATTR;
      if (isnan(row[1]) || isnan(row[2])) g->status |= ST_BAD_ATTR;
    }
  }
  for (int r = 0; r < I + O && r < N; ++r)
    if (!g->valid[r]) g->status |= ST_IO_ROW_INVALID;

  /* duplicate keys: sort (key, row) and look at neighbours */
  {
    pair_t *p = malloc(sizeof(pair_t) * (size_t)(g->V + 1));
    int n = 0;
    for (int r = 0; r < N; ++r)
      if (g->valid[r]) { p[n].a = g->key[r]; p[n].b = 0; p[n].i = r; ++n; }
    qsort(p, (size_t)n, sizeof(pair_t), cmp_pair);
    for (int i = 0; i < n; ++i) { g->skey[i] = p[i].a; g->srow[i] = p[i].i; }
    for (int i = 1; i < n; ++i)
      if (p[i].a == p[i - 1].a) g->status |= ST_DUP_KEY;
    free(p);
  }

  /* enabled connections, in ascending row order (Sec. 3.3: e = 0 rows are absent) */
  g->ne = 0;
  for (int j = 0; j < C; ++j) {
    const double *row = conns + (size_t)j * 4;
    if (isnan(row[0]) || isnan(row[1])) continue;    /* padding row */
    if (isnan(row[3]) || row[3] == 0.0) continue;    /* disabled */
    int s = find_row(g, (double)row[0]);
    int d = find_row(g, (double)row[1]);
    if (s < 0 || d < 0) { g->status |= ST_DANGLING_KEY; continue; }
    if (d < I) g->status |= ST_EDGE_INTO_INPUT;
    if (isnan(row[2])) g->status |= ST_BAD_ATTR;
    g->esrc[g->ne] = s;
    g->edst[g->ne] = d;
    g->erow[g->ne] = j;
    g->ew[g->ne] = row[2];
    g->ne++;
  }
  /* duplicate (src, dst) among enabled connections */
  {
    pair_t *p = malloc(sizeof(pair_t) * (size_t)(g->ne + 1));
    for (int e = 0; e < g->ne; ++e) { p[e].a = g->esrc[e]; p[e].b = g->edst[e]; p[e].i = e; }
    qsort(p, (size_t)g->ne, sizeof(pair_t), cmp_pair);
    for (int e = 1; e < g->ne; ++e)
      if (p[e].a == p[e - 1].a && p[e].b == p[e - 1].b) g->status |= ST_DUP_EDGE;
    free(p);
  }
  /* incoming lists, keeping ascending connection-row order */
  for (int r = 0; r <= N; ++r) g->in_beg[r] = 0;
  for (int e = 0; e < g->ne; ++e) g->in_beg[g->edst[e] + 1]++;
  for (int r = 0; r < N; ++r) g->in_beg[r + 1] += g->in_beg[r];
  {
    int *fill = calloc((size_t)N + 1, sizeof(int));
    for (int e = 0; e < g->ne; ++e) {
      int d = g->edst[e];
      g->in_list[g->in_beg[d] + fill[d]++] = e;
    }
    free(fill);
  }
  /* outgoing lists */
  for (int r = 0; r <= N; ++r) g->out_beg[r] = 0;
  for (int e = 0; e < g->ne; ++e) g->out_beg[g->esrc[e] + 1]++;
  for (int r = 0; r < N; ++r) g->out_beg[r + 1] += g->out_beg[r];
  {
    int *fill = calloc((size_t)N + 1, sizeof(int));
    for (int e = 0; e < g->ne; ++e) {
      int s = g->esrc[e];
      g->out_list[g->out_beg[s] + fill[s]++] = e;
    }
    free(fill);
  }
}

/* Sec. 3.3 transformation: topological order by frontiers (R4). */
static void transform_genome(genome_t *g) {
  const int N = g->N;
  for (int r = 0; r < N; ++r) g->layer[r] = -1;
  g->nord = 0;
  g->nlayers = 0;
  if (g->status & ~ST_CYCLE) return; /* R7: no order for malformed genomes */
  int *indeg = calloc((size_t)N + 1, sizeof(int));
  int *emitted = calloc((size_t)N + 1, sizeof(int));
  int *front = malloc(sizeof(int) * (size_t)(N + 1));
  for (int e = 0; e < g->ne; ++e) indeg[g->edst[e]]++;
  for (int t = 0;; ++t) {
    /* the frontier: valid, not yet emitted, no remaining incoming edge */
    int nf = 0;
    for (int r = 0; r < N; ++r)
      if (g->valid[r] && !emitted[r] && indeg[r] == 0) front[nf++] = r;
    if (nf == 0) break;
    /* ascending key (insertion sort: frontiers are small and this is plain) */
    for (int i = 1; i < nf; ++i) {
      int x = front[i], j = i - 1;
      while (j >= 0 && g->key[front[j]] > g->key[x]) { front[j + 1] = front[j]; --j; }
      front[j + 1] = x;
    }
    for (int i = 0; i < nf; ++i) {
      int r = front[i];
      g->order[g->nord++] = r;
      g->layer[r] = t;
      emitted[r] = 1;
    }
    /* remove the frontier's outgoing edges */
    for (int i = 0; i < nf; ++i)
      for (int k = g->out_beg[front[i]]; k < g->out_beg[front[i] + 1]; ++k)
        indeg[g->edst[g->out_list[k]]]--;
    g->nlayers = t + 1;
  }
  if (g->nord < g->V) g->status |= ST_CYCLE;
  free(indeg);
  free(emitted);
  free(front);
}

static double act_f(int a, double z) {
  switch (a) {
    case A_IDENTITY: return z;
    case A_SIGMOID: /* stable logistic */
      if (z >= 0) return 1.0 / (1.0 + exp(-z));
      else { double e = exp(z); return e / (1.0 + e); }
    case A_TANH: return tanh(z);
    case A_RELU: return z > 0 ? z : 0.0;
    case A_SIN: return sin(z);
    case A_GAUSS: return exp(-z * z);
    case A_ABS: return fabs(z);
  }
  return NAN;
}

/* derivative of the activation at z (R8) */
static double act_d(int a, double z) {
  switch (a) {
    case A_IDENTITY: return 1.0;
    case A_SIGMOID: { double s = act_f(A_SIGMOID, z); return s * (1.0 - s); }
    case A_TANH: { double t = tanh(z); return 1.0 - t * t; }
    case A_RELU: return z > 0 ? 1.0 : 0.0;
    case A_SIN: return cos(z);
    case A_GAUSS: return -2.0 * z * exp(-z * z);
    case A_ABS: return z > 0 ? 1.0 : (z < 0 ? -1.0 : 0.0);
  }
  return NAN;
}

/* largest |act'| over [z - h, z + h], for the fp32 error bound */
static double act_lip(int a, double z, double h) {
  double lo = z - h, hi = z + h;
  double c = (lo > 0) ? lo : (hi < 0 ? hi : 0.0); /* point of [lo,hi] nearest 0 */
  switch (a) {
    case A_IDENTITY: case A_ABS: return 1.0;
    case A_RELU: return hi > 0 ? 1.0 : 0.0;
    case A_SIGMOID: return act_d(A_SIGMOID, c);
    case A_TANH: return act_d(A_TANH, c);
    case A_SIN: return 1.0;
    case A_GAUSS: {
      /* |2x e^{-x^2}| peaks at |x| = 1/sqrt(2) */
      double pk = 1.0 / sqrt(2.0);
      double m = fmax(fabs(act_d(A_GAUSS, lo)), fabs(act_d(A_GAUSS, hi)));
      if ((lo <= pk && pk <= hi) || (lo <= -pk && -pk <= hi)) m = fabs(act_d(A_GAUSS, pk));
      return m;
    }
  }
  return 1.0;
}

#define U32 (1.0 / 16777216.0) /* fp32 unit roundoff 2^-24 */

/* One node of the calculation stage (Sec. 3.3): a = agg over the node's
 * enabled incoming connections (ascending row) of w * vin[src], z = b + r a,
 * v = act(z).  bin / bout (nullable): fp32 error bound of the inputs read and
 * of the result (first order; unit roundoff 2^-24, any summation order). */
static void eval_node(const genome_t *g, int r, const double *vin, const double *bin,
                      double *v_out, double *a_out, double *z_out, double *b_out) {
  const int beg = g->in_beg[r], n = g->in_beg[r + 1] - beg;
  const int want_b = bin != NULL && b_out != NULL;
  double acc = 0.0, sabs = 0.0, eb = 0.0;
  if (n > 0) {
    /* f_c on every incoming enabled connection, then f_agg */
    if (g->agg[r] == G_SUM || g->agg[r] == G_MEAN) {
      acc = 0.0;
      for (int q = 0; q < n; ++q) {
        int e = g->in_list[beg + q];
        double t = g->ew[e] * vin[g->esrc[e]];
        acc += t;
        if (want_b) { sabs += fabs(t); eb += fabs(g->ew[e]) * bin[g->esrc[e]] + U32 * fabs(t); }
      }
      if (want_b) eb += (n * U32 / (1.0 - n * U32)) * sabs;
      if (g->agg[r] == G_MEAN) { acc /= n; if (want_b) eb = eb / n + U32 * fabs(acc); }
    } else if (g->agg[r] == G_PRODUCT) {
      acc = 1.0;
      for (int q = 0; q < n; ++q) {
        int e = g->in_list[beg + q];
        acc *= g->ew[e] * vin[g->esrc[e]];
      }
      if (want_b) {
        /* first order: sum_e beta_e * prod_{f != e} |t_f|, plus 2n roundings */
        for (int q = 0; q < n; ++q) {
          int e = g->in_list[beg + q];
          double others = 1.0;
          for (int q2 = 0; q2 < n; ++q2)
            if (q2 != q) { int f = g->in_list[beg + q2]; others *= fabs(g->ew[f] * vin[g->esrc[f]]); }
          eb += fabs(g->ew[e]) * bin[g->esrc[e]] * others;
        }
        eb += 2.0 * n * U32 * fabs(acc) * 1.01;
      }
    } else { /* G_MAX: fmax fold */
      for (int q = 0; q < n; ++q) {
        int e = g->in_list[beg + q];
        double t = g->ew[e] * vin[g->esrc[e]];
        acc = (q == 0) ? t : fmax(acc, t);
        if (want_b) eb = fmax(eb, fabs(g->ew[e]) * bin[g->esrc[e]] + U32 * fabs(t));
      }
    }
  }
  const double z = g->bias[r] + g->resp[r] * acc;
  const double v = act_f(g->act[r], z);
  *a_out = acc;
  *z_out = z;
  *v_out = v;
  if (want_b) {
    double bz = fabs(g->resp[r]) * eb + U32 * fabs(g->resp[r] * acc) + U32 * fabs(z);
    double lip = act_lip(g->act[r], z, bz);
    double ef = 0.0; /* error of the fp32 activation itself */
    switch (g->act[r]) {
      case A_SIGMOID: case A_TANH: case A_SIN: ef = 8.0 * U32 * fabs(v); break;
      case A_GAUSS: ef = (8.0 + z * z) * 2.0 * U32 * fabs(v); break;
      default: ef = 0.0;
    }
    *b_out = lip * bz + ef + 1e-300;
  }
}

/* Sec. 3.3 calculation for one input vector.  v, a, z are per row; bnd (may be
 * NULL) receives the fp32 error bound per row; in_bnd is the error already in
 * the inputs (0 for exact fp32 inputs). */
static void forward_one(const genome_t *g, const double *x, double in_bnd, double *v, double *a,
                        double *z, double *bnd) {
  const int N = g->N, I = g->I;
  for (int r = 0; r < N; ++r) { v[r] = NAN; a[r] = NAN; z[r] = NAN; if (bnd) bnd[r] = 0; }
  for (int i = 0; i < I; ++i) { v[i] = x[i]; if (bnd) bnd[i] = in_bnd * fabs(x[i]) + (in_bnd > 0 ? in_bnd : 0); }
  for (int p = 0; p < g->nord; ++p) {
    const int r = g->order[p];
    if (r < I) continue;
    eval_node(g, r, v, bnd, &v[r], &a[r], &z[r], bnd ? &bnd[r] : NULL);
  }
}

/* Recurrent ("concurrent") network, synchronous iterations (R11): v^0 is the
 * input vector on rows 0..I-1 and 0 on every other valid row; for t = 1..T
 * every valid non-input row takes eval_node over v^{t-1} (inputs stay
 * clamped); v receives v^T (and bnd its fp32 error bound when non-NULL). */
static void recurrent_one(const genome_t *g, const double *x, int T, double *v, double *bnd) {
  const int N = g->N, I = g->I;
  double *vp = malloc(sizeof(double) * (size_t)N * 4 + 32);
  double *bp = vp + N, *vn = vp + 2 * N, *bn = vp + 3 * N;
  double a, z;
  for (int r = 0; r < N; ++r) { vp[r] = g->valid[r] ? 0.0 : NAN; bp[r] = 0.0; }
  for (int i = 0; i < I; ++i) vp[i] = x[i];
  for (int t = 0; t < T; ++t) {
    for (int r = 0; r < N; ++r) { vn[r] = vp[r]; bn[r] = bp[r]; }
    for (int r = I; r < N; ++r)
      if (g->valid[r]) eval_node(g, r, vp, bnd ? bp : NULL, &vn[r], &a, &z, bnd ? &bn[r] : NULL);
    for (int r = 0; r < N; ++r) { vp[r] = vn[r]; bp[r] = bn[r]; }
  }
  for (int r = 0; r < N; ++r) { v[r] = vp[r]; if (bnd) bnd[r] = bp[r]; }
  free(vp);
}

/* -------------------------------------------------------------------------- */
/* exported entry points                                                       */

/* Transformation stage for P genomes.  order[P,N] (rows, -1 padded),
 * layer[P,N] (-1 for rows not emitted), n_layers[P], status[P]. */
int or_transform(int P, int N, int C, int I, int O, const double *nodes, const double *conns,
                 int32_t *order, int32_t *layer, int32_t *n_layers, uint32_t *status) {
  genome_t g;
  if (P < 0 || N < I + O || C < 0) return -1;
  if (g_alloc(&g, N, C, I, O)) return -2;
  for (int p = 0; p < P; ++p) {
    parse_genome(&g, nodes + (size_t)p * N * 5, conns + (size_t)p * C * 4);
    transform_genome(&g);
    for (int i = 0; i < N; ++i) {
      order[(size_t)p * N + i] = i < g.nord ? g.order[i] : -1;
      layer[(size_t)p * N + i] = g.layer[i];
    }
    n_layers[p] = g.nlayers;
    status[p] = g.status;
  }
  g_free(&g);
  return 0;
}

/* Calculation stage.  inputs: genome p, sample s at inputs[p*in_pop_stride +
 * s*I + i] (stride 0 shares one set).  outputs[P,S,O]; bound (nullable)
 * [P,S,O] fp32 error bound; values (nullable) [P,S,N] node values by row. */
int or_forward(int P, int N, int C, int I, int O, const double *nodes, const double *conns,
               const double *inputs, int64_t in_pop_stride, int S, double *outputs, double *bound,
               double *values) {
  genome_t g;
  if (P < 0 || N < I + O || S < 0) return -1;
  if (g_alloc(&g, N, C, I, O)) return -2;
  double *v = malloc(sizeof(double) * (size_t)N * 4 + 32);
  double *a = v + N, *z = v + 2 * N, *bn = v + 3 * N;
  double *x = malloc(sizeof(double) * (size_t)(I + 1));
  for (int p = 0; p < P; ++p) {
    parse_genome(&g, nodes + (size_t)p * N * 5, conns + (size_t)p * C * 4);
    transform_genome(&g);
    for (int s = 0; s < S; ++s) {
      const double *in = inputs + (size_t)p * (size_t)in_pop_stride + (size_t)s * I;
      double *out = outputs + ((size_t)p * S + s) * O;
      if (g.status) {
        for (int j = 0; j < O; ++j) { out[j] = NAN; if (bound) bound[((size_t)p * S + s) * O + j] = 0; }
        if (values) for (int r = 0; r < N; ++r) values[((size_t)p * S + s) * N + r] = NAN;
        continue;
      }
      for (int i = 0; i < I; ++i) x[i] = in[i];
      forward_one(&g, x, 0.0, v, a, z, bound ? bn : NULL);
      for (int j = 0; j < O; ++j) {
        out[j] = v[I + j];
        if (bound) bound[((size_t)p * S + s) * O + j] = bn[I + j];
      }
      if (values) for (int r = 0; r < N; ++r) values[((size_t)p * S + s) * N + r] = v[r];
    }
  }
  free(v);
  free(x);
  g_free(&g);
  return 0;
}

/* Recurrent calculation (R11) over T synchronous iterations.  No
 * topological order is needed: cycles and self-loops are allowed, and status
 * (nullable) [P] receives every other bit of R7.  outputs [P,S,O] (NaN for a
 * genome with a status bit); bound (nullable) [P,S,O] fp32 error bound. */
int or_forward_recurrent(int P, int N, int C, int I, int O, const double *nodes,
                         const double *conns, const double *inputs, int64_t in_pop_stride, int S,
                         int T, double *outputs, double *bound, uint32_t *status) {
  genome_t g;
  if (P < 0 || N < I + O || S < 0 || T < 0) return -1;
  if (g_alloc(&g, N, C, I, O)) return -2;
  double *v = malloc(sizeof(double) * (size_t)N * 2 + 32);
  double *bn = v + N;
  double *x = malloc(sizeof(double) * (size_t)(I + 1));
  for (int p = 0; p < P; ++p) {
    parse_genome(&g, nodes + (size_t)p * N * 5, conns + (size_t)p * C * 4);
    if (status) status[p] = g.status;
    for (int s = 0; s < S; ++s) {
      const double *in = inputs + (size_t)p * (size_t)in_pop_stride + (size_t)s * I;
      double *out = outputs + ((size_t)p * S + s) * O;
      if (g.status) {
        for (int j = 0; j < O; ++j) { out[j] = NAN; if (bound) bound[((size_t)p * S + s) * O + j] = 0; }
        continue;
      }
      for (int i = 0; i < I; ++i) x[i] = in[i];
      recurrent_one(&g, x, T, v, bound ? bn : NULL);
      for (int j = 0; j < O; ++j) {
        out[j] = v[I + j];
        if (bound) bound[((size_t)p * S + s) * O + j] = bn[I + j];
      }
    }
  }
  free(v);
  free(x);
  g_free(&g);
  return 0;
}

/* HyperNEAT substrate (R14): weights [P, K, K] (input cell, output cell),
 * inputs x at inputs[p * in_pop_stride + s * K + c], outputs [P, S, K];
 * bound (nullable) [P, S, K] first-order fp32 error bound of an evaluation
 * with fp32 products and any summation order (inputs and weights exact). */
int or_substrate(int P, int K, const double *w, const double *inputs, int64_t in_pop_stride,
                 int S, int act, double *out, double *bound) {
  if (P < 0 || K < 1 || S < 0 || act < 0 || act >= N_ACTS) return -1;
  for (int p = 0; p < P; ++p) {
    const double *wp = w + (size_t)p * K * K;
    for (int s = 0; s < S; ++s) {
      const double *x = inputs + (size_t)p * (size_t)in_pop_stride + (size_t)s * K;
      double *y = out + ((size_t)p * S + s) * K;
      for (int t = 0; t < K; ++t) {
        double acc = 0.0, sabs = 0.0;
        for (int c = 0; c < K; ++c) {
          const double term = wp[(size_t)c * K + t] * x[c];
          acc += term;
          sabs += fabs(term);
        }
        y[t] = act_f(act, acc);
        if (bound) {
          const double eb = (K * U32 / (1.0 - K * U32)) * sabs + U32 * sabs;
          double ef = 0.0;
          switch (act) {
            case A_SIGMOID: case A_TANH: case A_SIN: ef = 8.0 * U32 * fabs(y[t]); break;
            case A_GAUSS: ef = (8.0 + acc * acc) * 2.0 * U32 * fabs(y[t]); break;
            default: ef = 0.0;
          }
          bound[((size_t)p * S + s) * K + t] = act_lip(act, acc, eb) * eb + ef + 1e-300;
        }
      }
    }
  }
  return 0;
}

/* Tensorized operations (R13) on every genome, in place: nodes [P,N,5],
 * conns [P,C,4], ops [P,K,8]; op_status [P] receives the failed-op bits. */
int or_apply_ops(int P, int N, int C, double *nodes, double *conns, const double *ops, int K,
                 uint32_t *op_status) {
  if (P < 0 || N < 1 || C < 1 || K < 0) return -1;
  for (int p = 0; p < P; ++p) {
    double *gn = nodes + (size_t)p * N * 5, *gc = conns + (size_t)p * C * 4;
    uint32_t st = 0;
    for (int k = 0; k < K; ++k) {
      const double *op = ops + ((size_t)p * K + k) * 8;
      const double kind = op[0], rowf = op[1];
      int ok = 1;
      if (kind == 1.0 || kind == 3.0) {
        const int cols = kind == 1.0 ? 5 : 4, rows = kind == 1.0 ? N : C;
        double *t = kind == 1.0 ? gn : gc;
        int r = -1;
        for (int i = 0; i < rows && r < 0; ++i) {
          const int pad = kind == 1.0 ? isnan(t[(size_t)i * 5]) : (isnan(t[(size_t)i * 4]) || isnan(t[(size_t)i * 4 + 1]));
          if (pad) r = i;
        }
        if (r < 0) ok = 0;
        else for (int c = 0; c < cols; ++c) t[(size_t)r * cols + c] = op[2 + c];
      } else if (kind == 2.0 || kind == 4.0) {
        const int cols = kind == 2.0 ? 5 : 4, rows = kind == 2.0 ? N : C;
        double *t = kind == 2.0 ? gn : gc;
        if (!(rowf >= 0 && rowf < rows && rowf == floor(rowf))) ok = 0;
        else for (int c = 0; c < cols; ++c) t[(size_t)rowf * cols + c] = NAN;
      } else if (kind == 5.0 || kind == 6.0) {
        const int cols = kind == 5.0 ? 5 : 4, rows = kind == 5.0 ? N : C;
        const int lo = kind == 5.0 ? 1 : 2, hi = cols - 1;
        double *t = kind == 5.0 ? gn : gc;
        const double col = op[2];
        if (!(rowf >= 0 && rowf < rows && rowf == floor(rowf)) ||
            !(col >= lo && col <= hi && col == floor(col)))
          ok = 0;
        else
          t[(size_t)rowf * cols + (size_t)col] = op[3];
      }
      if (!ok && k < 32) st |= 1u << k;
    }
    if (op_status) op_status[p] = st;
  }
  return 0;
}

/* Compatibility distance (R12) for every pair of the P genomes:
 * dist[P, P] (row-major, symmetric, zero diagonal for valid genomes). */
typedef struct {
  int n, m;            /* node genes, connection genes */
  double *nkey, *nb, *nr;
  int *nact, *nagg, *ninput;
  double *cin, *cout, *cw;
  int *cen;
  int bad;             /* status bit other than CYCLE */
} genes_t;

typedef struct { double a, b; int row; } key2_t;
static int cmp_key2(const void *x, const void *y) {
  const key2_t *p = x, *q = y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return p->row - q->row;
}

static void collect_genes(genes_t *G, const genome_t *g, const double *nodes, const double *conns) {
  const int N = g->N, C = g->C, I = g->I;
  G->bad = (g->status & ~ST_CYCLE) != 0;
  /* node genes in ascending key (rows of equal keys cannot occur unless bad) */
  key2_t *t = malloc(sizeof(key2_t) * (size_t)(N + C + 1));
  int n = 0;
  for (int r = 0; r < N; ++r)
    if (g->valid[r]) { t[n].a = g->key[r]; t[n].b = 0; t[n].row = r; ++n; }
  qsort(t, (size_t)n, sizeof(key2_t), cmp_key2);
  G->n = n;
  for (int i = 0; i < n; ++i) {
    const int r = t[i].row;
    G->nkey[i] = g->key[r];
    G->nb[i] = nodes[(size_t)r * 5 + 1];
    G->nr[i] = nodes[(size_t)r * 5 + 2];
    /* ids of non-input rows (integral and in range unless the genome is bad) */
    G->nact[i] = (r >= I && g->act[r] >= 0) ? g->act[r] : -1;
    G->nagg[i] = (r >= I && g->agg[r] >= 0) ? g->agg[r] : -1;
    G->ninput[i] = r < I;
  }
  /* connection genes: valid rows by (in, out, row); the first of a key counts */
  int m = 0;
  for (int j = 0; j < C; ++j) {
    const double *row = conns + (size_t)j * 4;
    if (isnan(row[0]) || isnan(row[1])) continue;
    t[m].a = row[0]; t[m].b = row[1]; t[m].row = j; ++m;
  }
  qsort(t, (size_t)m, sizeof(key2_t), cmp_key2);
  int k = 0;
  for (int i = 0; i < m; ++i) {
    if (k > 0 && t[i].a == G->cin[k - 1] && t[i].b == G->cout[k - 1]) continue;
    const double *row = conns + (size_t)t[i].row * 4;
    G->cin[k] = t[i].a;
    G->cout[k] = t[i].b;
    G->cw[k] = row[2];
    G->cen[k] = !isnan(row[3]) && row[3] != 0.0;
    ++k;
  }
  G->m = k;
  free(t);
}

static double pair_distance(const genes_t *A, const genes_t *B, double cd, double ch) {
  if (A->bad || B->bad) return NAN;
  /* nodes: merge the two key-sorted lists */
  int i = 0, j = 0, D = 0;
  double H = 0.0;
  while (i < A->n || j < B->n) {
    if (j >= B->n || (i < A->n && A->nkey[i] < B->nkey[j])) { ++D; ++i; continue; }
    if (i >= A->n || B->nkey[j] < A->nkey[i]) { ++D; ++j; continue; }
    if (!A->ninput[i] && !B->ninput[j])
      H += fabs(A->nb[i] - B->nb[j]) + fabs(A->nr[i] - B->nr[j]) +
           (A->nact[i] != B->nact[j]) + (A->nagg[i] != B->nagg[j]);
    ++i; ++j;
  }
  const int nmax = A->n > B->n ? A->n : B->n;
  double d = nmax > 0 ? (cd * D + ch * H) / nmax : 0.0;
  /* connections */
  i = 0; j = 0; D = 0; H = 0.0;
  while (i < A->m || j < B->m) {
    int less_a = 0, less_b = 0;
    if (j >= B->m) less_a = 1;
    else if (i >= A->m) less_b = 1;
    else if (A->cin[i] != B->cin[j]) { less_a = A->cin[i] < B->cin[j]; less_b = !less_a; }
    else if (A->cout[i] != B->cout[j]) { less_a = A->cout[i] < B->cout[j]; less_b = !less_a; }
    if (less_a) { ++D; ++i; continue; }
    if (less_b) { ++D; ++j; continue; }
    H += fabs(A->cw[i] - B->cw[j]) + (A->cen[i] != B->cen[j]);
    ++i; ++j;
  }
  const int mmax = A->m > B->m ? A->m : B->m;
  if (mmax > 0) d += (cd * D + ch * H) / mmax;
  return d;
}

int or_distance(int P, int N, int C, int I, int O, const double *nodes, const double *conns,
                double cd, double ch, double *dist) {
  genome_t g;
  if (P < 0 || N < I + O || C < 0) return -1;
  if (g_alloc(&g, N, C, I, O)) return -2;
  genes_t *G = calloc((size_t)P + 1, sizeof(genes_t));
  for (int p = 0; p < P; ++p) {
    genes_t *x = &G[p];
    x->nkey = malloc(sizeof(double) * (size_t)(N + 1)); x->nb = malloc(sizeof(double) * (size_t)(N + 1));
    x->nr = malloc(sizeof(double) * (size_t)(N + 1)); x->nact = malloc(sizeof(int) * (size_t)(N + 1));
    x->nagg = malloc(sizeof(int) * (size_t)(N + 1)); x->ninput = malloc(sizeof(int) * (size_t)(N + 1));
    x->cin = malloc(sizeof(double) * (size_t)(C + 1)); x->cout = malloc(sizeof(double) * (size_t)(C + 1));
    x->cw = malloc(sizeof(double) * (size_t)(C + 1)); x->cen = malloc(sizeof(int) * (size_t)(C + 1));
    parse_genome(&g, nodes + (size_t)p * N * 5, conns + (size_t)p * C * 4);
    collect_genes(x, &g, nodes + (size_t)p * N * 5, conns + (size_t)p * C * 4);
  }
  for (int a = 0; a < P; ++a)
    for (int b = 0; b < P; ++b)
      dist[(size_t)a * P + b] = pair_distance(&G[a], &G[b], cd, ch);
  for (int p = 0; p < P; ++p) {
    genes_t *x = &G[p];
    free(x->nkey); free(x->nb); free(x->nr); free(x->nact); free(x->nagg); free(x->ninput);
    free(x->cin); free(x->cout); free(x->cw); free(x->cen);
  }
  free(G);
  g_free(&g);
  return 0;
}

/* Reverse mode through the calculation stage (R8).  grad_out[P,S,O] is dL/dO.
 * Writes grad_w[P,C] (by connection row; 0 on padding/disabled rows),
 * grad_b[P,N], grad_r[P,N] (by node row; 0 on inputs and padding), and
 * grad_in[P,S,I] (nullable).  Sums over samples. */
int or_backward(int P, int N, int C, int I, int O, const double *nodes, const double *conns,
                const double *inputs, int64_t in_pop_stride, int S, const double *grad_out,
                double *grad_w, double *grad_b, double *grad_r, double *grad_in) {
  genome_t g;
  if (P < 0 || N < I + O || S < 0) return -1;
  if (g_alloc(&g, N, C, I, O)) return -2;
  double *v = malloc(sizeof(double) * (size_t)N * 4 + 32);
  double *a = v + N, *z = v + 2 * N, *dl = v + 3 * N;
  double *x = malloc(sizeof(double) * (size_t)(I + 1));
  double *tv = malloc(sizeof(double) * (size_t)(C + 1));
  double *pre = malloc(sizeof(double) * (size_t)(C + 2));
  double *suf = malloc(sizeof(double) * (size_t)(C + 2));
  for (int p = 0; p < P; ++p) {
    double *gw = grad_w + (size_t)p * C, *gb = grad_b + (size_t)p * N, *gr = grad_r + (size_t)p * N;
    for (int j = 0; j < C; ++j) gw[j] = 0.0;
    for (int r = 0; r < N; ++r) { gb[r] = 0.0; gr[r] = 0.0; }
    parse_genome(&g, nodes + (size_t)p * N * 5, conns + (size_t)p * C * 4);
    transform_genome(&g);
    for (int s = 0; s < S; ++s) {
      double *gi = grad_in ? grad_in + ((size_t)p * S + s) * I : NULL;
      if (g.status) { if (gi) for (int i = 0; i < I; ++i) gi[i] = 0.0; continue; }
      const double *in = inputs + (size_t)p * (size_t)in_pop_stride + (size_t)s * I;
      for (int i = 0; i < I; ++i) x[i] = in[i];
      forward_one(&g, x, 0.0, v, a, z, NULL);
      for (int r = 0; r < N; ++r) dl[r] = 0.0;
      for (int j = 0; j < O; ++j) dl[I + j] += grad_out[((size_t)p * S + s) * O + j];
      for (int q = g.nord - 1; q >= 0; --q) {
        const int r = g.order[q];
        if (r < I) continue;
        const double u = dl[r] * act_d(g.act[r], z[r]); /* dL/dz */
        gb[r] += u;
        gr[r] += u * a[r];
        const double da = u * g.resp[r];                  /* dL/d agg */
        const int beg = g.in_beg[r], n = g.in_beg[r + 1] - beg;
        if (n == 0) continue;
        for (int k = 0; k < n; ++k) {
          int e = g.in_list[beg + k];
          tv[k] = g.ew[e] * v[g.esrc[e]];
        }
        int argmax = 0;
        if (g.agg[r] == G_PRODUCT) {
          pre[0] = 1.0;
          for (int k = 0; k < n; ++k) pre[k + 1] = pre[k] * tv[k];
          suf[n] = 1.0;
          for (int k = n - 1; k >= 0; --k) suf[k] = suf[k + 1] * tv[k];
        } else if (g.agg[r] == G_MAX) {
          for (int k = 1; k < n; ++k)
            if (tv[k] > tv[argmax] || isnan(tv[argmax])) argmax = k;
        }
        for (int k = 0; k < n; ++k) {
          int e = g.in_list[beg + k];
          double dt; /* d agg / d t_k */
          switch (g.agg[r]) {
            case G_SUM: dt = 1.0; break;
            case G_MEAN: dt = 1.0 / n; break;
            case G_PRODUCT: dt = pre[k] * suf[k + 1]; break;
            default: dt = (k == argmax) ? 1.0 : 0.0; break;
          }
          const double dtk = da * dt;
          gw[g.erow[e]] += dtk * v[g.esrc[e]];
          dl[g.esrc[e]] += dtk * g.ew[e];
        }
      }
      if (gi) for (int i = 0; i < I; ++i) gi[i] = dl[i];
    }
  }
  free(v); free(x); free(tv); free(pre); free(suf);
  g_free(&g);
  return 0;
}

/* HyperNEAT substrate query (R9).  Evaluates each CPPN on (x_s, y_s, x_d,
 * y_d, 1) for the queries listed in qidx (flat index s * G^2 + d, nq of them,
 * the same list for every genome), or for all G^4 queries when qidx is NULL.
 * out[P, nq] thresholded weights, raw (nullable) the unthresholded output,
 * bound (nullable) the fp32 error bound of raw (coordinates computed in fp32). */
int or_hyperneat(int P, int N, int C, const double *nodes, const double *conns, int G,
                 double thresh, const int64_t *qidx, int64_t nq, double *out, double *raw,
                 double *bound) {
  const int I = 5, O = 1;
  genome_t g;
  if (P < 0 || N < I + O || G < 2) return -1;
  const int64_t G2 = (int64_t)G * G;
  const int64_t total = qidx ? nq : G2 * G2;
  if (g_alloc(&g, N, C, I, O)) return -2;
  double *v = malloc(sizeof(double) * (size_t)N * 4 + 32);
  double *a = v + N, *z = v + 2 * N, *bn = v + 3 * N;
  double x[5];
  for (int p = 0; p < P; ++p) {
    parse_genome(&g, nodes + (size_t)p * N * 5, conns + (size_t)p * C * 4);
    transform_genome(&g);
    for (int64_t q = 0; q < total; ++q) {
      const int64_t flat = qidx ? qidx[q] : q;
      const int64_t sc = flat / G2, dc = flat % G2;
      const size_t o = (size_t)p * (size_t)total + (size_t)q;
      if (g.status) { out[o] = NAN; if (raw) raw[o] = NAN; if (bound) bound[o] = 0; continue; }
      x[0] = -1.0 + 2.0 * (double)(sc % G) / (G - 1);
      x[1] = -1.0 + 2.0 * (double)(sc / G) / (G - 1);
      x[2] = -1.0 + 2.0 * (double)(dc % G) / (G - 1);
      x[3] = -1.0 + 2.0 * (double)(dc / G) / (G - 1);
      x[4] = 1.0;
      forward_one(&g, x, bound ? 4.0 * U32 : 0.0, v, a, z, bound ? bn : NULL);
      const double o0 = v[I];
      out[o] = fabs(o0) > thresh ? o0 : 0.0;
      if (raw) raw[o] = o0;
      if (bound) bound[o] = bn[I];
    }
  }
  free(v);
  g_free(&g);
  return 0;
}
