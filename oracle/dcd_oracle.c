/*
 * dcd_oracle.c -- plain sequential CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Follows, in order:
 *   Sec. III-A   notation: e_{i->C}, a_C, d_w(i), m_t; Eq. (1) modularity
 *   Sec. III-B   Algorithm 1: local-move iterations, Q-based convergence,
 *                graph compaction, repeat
 *   Sec. III-D   incremental approach: t = 1 static; t > 1 inherit C_{t-1},
 *                R_t = DeltaScreening(G_t, Delta_t), R_t used at level 0 only
 *   Sec. III-E   Algorithm 2 (Delta-screening)
 * Readings where the paper is silent (tie-breaks, tau, the synchronous
 * schedule, the singleton-swap guard, the deletion rule) are stated at the
 * function that takes them.  No blocking, fusion or reordering: each
 * quantity is recomputed from its definition where the definition is cheap
 * enough for test-sized graphs.
 */
#include "dcd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

struct orc_graph {
  int64_t n;
  int64_t* row_ptr; /* n + 1 */
  int32_t* col;     /* nnz, ascending within each row */
  int64_t* w;       /* nnz, > 0 */
};

/* ------------------------------------------------------------------ */
/* graphs                                                              */
/* ------------------------------------------------------------------ */

static orc_graph* graph_alloc(int64_t n, int64_t nnz) {
  orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
  if (!g) return NULL;
  g->n = n;
  g->row_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->col = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  g->w = (int64_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
  if (!g->row_ptr || !g->col || !g->w) {
    free(g->row_ptr); free(g->col); free(g->w); free(g);
    return NULL;
  }
  return g;
}

void orc_graph_free(orc_graph* g) {
  if (!g) return;
  free(g->row_ptr); free(g->col); free(g->w); free(g);
}

int64_t orc_graph_n(const orc_graph* g) { return g->n; }
int64_t orc_graph_nnz(const orc_graph* g) { return g->row_ptr[g->n]; }

orc_graph* orc_graph_new(int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const int64_t* w) {
  int64_t nnz = row_ptr ? row_ptr[n] : 0;
  orc_graph* g = graph_alloc(n, nnz);
  if (!g) return NULL;
  if (row_ptr) {
    memcpy(g->row_ptr, row_ptr, (size_t)(n + 1) * sizeof(int64_t));
    memcpy(g->col, col, (size_t)nnz * sizeof(int32_t));
    memcpy(g->w, w, (size_t)nnz * sizeof(int64_t));
  }
  return g;
}

void orc_graph_copy(const orc_graph* g, int64_t* row_ptr, int32_t* col, int64_t* w) {
  int64_t nnz = g->row_ptr[g->n];
  if (row_ptr) memcpy(row_ptr, g->row_ptr, (size_t)(g->n + 1) * sizeof(int64_t));
  if (col) memcpy(col, g->col, (size_t)nnz * sizeof(int32_t));
  if (w) memcpy(w, g->w, (size_t)nnz * sizeof(int64_t));
}

/* An ordered pair (u,v) with weight w: one directed CSR entry. */
typedef struct { int32_t u, v; int64_t w; } triple;

static int cmp_triple(const void* pa, const void* pb) {
  const triple* a = (const triple*)pa;
  const triple* b = (const triple*)pb;
  if (a->u != b->u) return a->u < b->u ? -1 : 1;
  if (a->v != b->v) return a->v < b->v ? -1 : 1;
  return 0;
}

/* Sort ordered pairs, add up the weights of equal pairs, drop pairs whose
 * total weight is 0, and lay the result out as CSR. */
static orc_graph* graph_from_triples(int64_t n, triple* t, int64_t m) {
  if (m > 0) qsort(t, (size_t)m, sizeof(triple), cmp_triple);
  int64_t k = 0;
  for (int64_t i = 0; i < m;) {
    int64_t j = i;
    int64_t sum = 0;
    while (j < m && t[j].u == t[i].u && t[j].v == t[i].v) sum += t[j++].w;
    if (sum != 0) { t[k] = t[i]; t[k].w = sum; k++; }
    i = j;
  }
  orc_graph* g = graph_alloc(n, k);
  if (!g) return NULL;
  for (int64_t i = 0; i < k; i++) {
    g->row_ptr[t[i].u + 1]++;
    g->col[i] = t[i].v;
    g->w[i] = t[i].w;
  }
  for (int64_t u = 0; u < n; u++) g->row_ptr[u + 1] += g->row_ptr[u];
  return g;
}

/* Position of entry (u,v) in g, or -1. */
static int64_t find_entry(const orc_graph* g, int32_t u, int32_t v) {
  int64_t lo = g->row_ptr[u], hi = g->row_ptr[u + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (g->col[mid] < v) lo = mid + 1; else hi = mid;
  }
  return (lo < g->row_ptr[u + 1] && g->col[lo] == v) ? lo : -1;
}

/* Sec. III-A: the graph is undirected and each change is stored as the two
 * ordered pairs (i,j) and (j,i) (Sec. III-E).  Edge deletions are outside the
 * paper (it assumes edges only grow, Sec. III-A; deletions are future work,
 * Sec. V); the reading taken here: all deletes of the batch act first and
 * remove the whole edge, then every insert adds its weight (a new edge or a
 * larger multiplicity). */
orc_graph* orc_apply(const orc_graph* g, const int32_t* ins, int64_t n_ins,
                     const int32_t* del, int64_t n_del, uint8_t* del_present,
                     int* err) {
  int64_t n = g->n;
  *err = ORC_OK;
  for (int64_t i = 0; i < n_ins; i++) {
    int32_t u = ins[3 * i], v = ins[3 * i + 1], w = ins[3 * i + 2];
    if (u < 0 || v < 0 || u >= n || v >= n || u == v || w <= 0) { *err = ORC_EINVAL; return NULL; }
  }
  for (int64_t i = 0; i < n_del; i++) {
    int32_t u = del[2 * i], v = del[2 * i + 1];
    if (u < 0 || v < 0 || u >= n || v >= n || u == v) { *err = ORC_EINVAL; return NULL; }
  }
  int64_t nnz = g->row_ptr[n];
  int64_t m = nnz + 2 * n_ins;
  triple* t = (triple*)malloc((size_t)(m > 0 ? m : 1) * sizeof(triple));
  if (!t) { *err = ORC_ENOMEM; return NULL; }
  for (int64_t u = 0; u < n; u++)
    for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; e++) {
      t[e].u = (int32_t)u; t[e].v = g->col[e]; t[e].w = g->w[e];
    }
  for (int64_t i = 0; i < n_del; i++) {
    int32_t u = del[2 * i], v = del[2 * i + 1];
    int64_t e1 = find_entry(g, u, v), e2 = find_entry(g, v, u);
    if (del_present) del_present[i] = (uint8_t)(e1 >= 0);
    if (e1 >= 0) t[e1].w = 0;
    if (e2 >= 0) t[e2].w = 0;
  }
  for (int64_t i = 0; i < n_ins; i++) {
    int32_t u = ins[3 * i], v = ins[3 * i + 1], w = ins[3 * i + 2];
    t[nnz + 2 * i].u = u; t[nnz + 2 * i].v = v; t[nnz + 2 * i].w = w;
    t[nnz + 2 * i + 1].u = v; t[nnz + 2 * i + 1].v = u; t[nnz + 2 * i + 1].w = w;
  }
  orc_graph* out = graph_from_triples(n, t, m);
  free(t);
  if (!out) { *err = ORC_ENOMEM; return NULL; }
  /* Level-0 weights are int32 in the library; the oracle flags the same limit. */
  for (int64_t e = 0; e < out->row_ptr[n]; e++)
    if (out->w[e] > INT32_MAX) { orc_graph_free(out); *err = ORC_EOVERFLOW; return NULL; }
  return out;
}

/* ------------------------------------------------------------------ */
/* Sec. III-A quantities                                               */
/* ------------------------------------------------------------------ */

/* d_w(v) = sum of weights of the entries of row v (a coarse self-loop is
 * stored once, with the internal directed weight, so it counts once). */
static void weighted_degrees(const orc_graph* g, int64_t* k, int64_t* m2) {
  int64_t s = 0;
  for (int64_t u = 0; u < g->n; u++) {
    int64_t d = 0;
    for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; e++) d += g->w[e];
    k[u] = d;
    s += d;
  }
  *m2 = s;
}

/* a_C = sum of d_w over the members of C, and |C|, indexed by label. */
static void community_sums(int64_t n, const int32_t* labels, const int64_t* k,
                           int64_t* a, int64_t* size) {
  for (int64_t c = 0; c < n; c++) { a[c] = 0; if (size) size[c] = 0; }
  for (int64_t v = 0; v < n; v++) {
    a[labels[v]] += k[v];
    if (size) size[labels[v]] += 1;
  }
}

/* Eq. (1) scaled by m2^2:  N = m2 * sum_i e_{i->C(i)} - sum_C a_C^2, where
 * sum_i e_{i->C(i)} runs over ordered pairs (each undirected intra-community
 * edge twice; a coarse self-loop entry once).  Q = N / m2^2. */
static i128 modularity_N(const orc_graph* g, const int32_t* labels, int64_t* m2_out) {
  int64_t n = g->n;
  int64_t* k = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* a = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t m2;
  weighted_degrees(g, k, &m2);
  community_sums(n, labels, k, a, NULL);
  i128 in = 0;
  for (int64_t u = 0; u < n; u++)
    for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; e++)
      if (labels[g->col[e]] == labels[u]) in += g->w[e];
  i128 sq = 0;
  for (int64_t c = 0; c < n; c++) sq += (i128)a[c] * (i128)a[c];
  free(k); free(a);
  *m2_out = m2;
  return (i128)m2 * in - sq;
}

/* Round-to-nearest conversions of the exact integers, then one division. */
static double q_from(i128 N, int64_t m2) {
  if (m2 == 0) return 0.0;
  return (double)N / ((double)m2 * (double)m2);
}

double orc_modularity(const orc_graph* g, const int32_t* labels, int64_t* m2,
                      int64_t* n_lo, int64_t* n_hi) {
  int64_t mm;
  i128 N = modularity_N(g, labels, &mm);
  if (m2) *m2 = mm;
  if (n_lo) *n_lo = (int64_t)(uint64_t)N;
  if (n_hi) *n_hi = (int64_t)(N >> 64);
  return q_from(N, mm);
}

/* e_{v->D} excluding v's own self-loop (Sec. III-A). */
static int64_t edge_weight_to(const orc_graph* g, const int32_t* labels, int32_t v, int32_t D) {
  int64_t s = 0;
  for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++)
    if (g->col[e] != v && labels[g->col[e]] == D) s += g->w[e];
  return s;
}

/* Gain of moving v from C = labels[v] to D (Sec. III-A; cf. the expanded
 * form in the proof of Lemma 3.2, Appendix A):
 *   S = m2 (e_{v->D} - e_{v->C\v}) - k_v (a_D - (a_C - k_v)),
 * which is (2m)^2 times the paper's Delta Q_{v->D}, and half the change of N. */
static i128 gain_S(int64_t m2, int64_t kv, int64_t eD, int64_t eC, int64_t aD, int64_t aC) {
  return (i128)m2 * (i128)(eD - eC) - (i128)kv * (i128)(aD - (aC - kv));
}

void orc_gain(const orc_graph* g, const int32_t* labels, int32_t v, int32_t D,
              int64_t* s_lo, int64_t* s_hi) {
  i128 S = 0;
  if (labels[v] != D) {
    int64_t n = g->n, m2;
    int64_t* k = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* a = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    weighted_degrees(g, k, &m2);
    community_sums(n, labels, k, a, NULL);
    int32_t C = labels[v];
    S = gain_S(m2, k[v], edge_weight_to(g, labels, v, D), edge_weight_to(g, labels, v, C),
               a[D], a[C]);
    free(k); free(a);
  }
  *s_lo = (int64_t)(uint64_t)S;
  *s_hi = (int64_t)(S >> 64);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1, inner loop                                             */
/* ------------------------------------------------------------------ */

typedef struct { int32_t label; int64_t w; } lw;

static int cmp_lw(const void* pa, const void* pb) {
  const lw* a = (const lw*)pa;
  const lw* b = (const lw*)pb;
  return (a->label > b->label) - (a->label < b->label);
}

/* The greedy choice of Algorithm 1 for one vertex (Sec. III-B, Louvain rule
 * C(v) <- argmax_{C(j), j in Gamma(v) u {v}} Delta Q), read from a fixed
 * snapshot (labels, a, size):
 *   - candidates: labels of neighbours u != v other than C = labels[v];
 *   - best = largest S, ties to the smallest label; staying (S = 0) wins ties;
 *   - singleton-swap guard (the minimum-label rule of Lu, Halappanavar and
 *     Kalyanaraman, the parallel Louvain heuristics the paper cites for its
 *     notation): a singleton does not move into another singleton with a
 *     larger label.
 * Returns the chosen label, or C. */
static int32_t best_move(const orc_graph* g, const int32_t* labels, const int64_t* k,
                         const int64_t* a, const int64_t* size, int64_t m2, int32_t v,
                         lw* buf) {
  int32_t C = labels[v];
  int64_t cnt = 0;
  for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
    if (g->col[e] == v) continue;
    buf[cnt].label = labels[g->col[e]];
    buf[cnt].w = g->w[e];
    cnt++;
  }
  if (cnt == 0) return C;
  qsort(buf, (size_t)cnt, sizeof(lw), cmp_lw);
  int64_t eC = 0;
  for (int64_t i = 0; i < cnt; i++) if (buf[i].label == C) eC += buf[i].w;
  int32_t best = C;
  i128 bestS = 0;
  for (int64_t i = 0; i < cnt;) {
    int32_t D = buf[i].label;
    int64_t eD = 0;
    int64_t j = i;
    while (j < cnt && buf[j].label == D) eD += buf[j++].w;
    i = j;
    if (D == C) continue;
    i128 S = gain_S(m2, k[v], eD, eC, a[D], a[C]);
    if (S > bestS) { bestS = S; best = D; } /* ascending D: strict > keeps the smallest */
  }
  if (best != C && size[C] == 1 && size[best] == 1 && best > C) return C;
  return best;
}

int64_t orc_local_move_pass(const orc_graph* g, const int32_t* labels,
                            const uint8_t* active, int32_t* out) {
  int64_t n = g->n, m2, maxdeg = 1;
  int64_t* k = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* a = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* size = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  weighted_degrees(g, k, &m2);
  community_sums(n, labels, k, a, size);
  for (int64_t u = 0; u < n; u++)
    if (g->row_ptr[u + 1] - g->row_ptr[u] > maxdeg) maxdeg = g->row_ptr[u + 1] - g->row_ptr[u];
  lw* buf = (lw*)malloc((size_t)maxdeg * sizeof(lw));
  int64_t moves = 0;
  for (int64_t v = 0; v < n; v++) {
    out[v] = labels[v];
    if (active && !active[v]) continue;
    out[v] = best_move(g, labels, k, a, size, m2, (int32_t)v, buf);
    if (out[v] != labels[v]) moves++;
  }
  free(buf); free(k); free(a); free(size);
  return moves;
}

/* x * 10^6 <= y  (y >= 0)  <=>  x <= floor(y / 10^6): the exact form of
 * "gain below tau = 1e-6 of |Q|" (tau is not given in the paper, Sec. III-B). */
static int below_tau(i128 gain, i128 base) {
  i128 y = base < 0 ? -base : base;
  return gain <= y / ORC_TAU_INV;
}

/* Inner loop of Algorithm 1 on one level, synchronous: every pass reads the
 * labels of the previous pass and all proposals are applied together.  Stops
 * when no vertex moves, when the pass gained at most 1e-6 of |Q| (a loss
 * included; the state is kept), or after max_iters passes. */
int64_t orc_run_level(const orc_graph* g, int32_t* labels, const uint8_t* active,
                      int64_t max_iters, int64_t* moves_out, int64_t* edges_out) {
  int64_t n = g->n, m2, iters = 0, moves = 0, edges = 0, act_deg = 0;
  int32_t* next = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  for (int64_t v = 0; v < n; v++)
    if (!active || active[v]) act_deg += g->row_ptr[v + 1] - g->row_ptr[v];
  i128 N_old = modularity_N(g, labels, &m2);
  while (iters < max_iters) {
    int64_t mv = orc_local_move_pass(g, labels, active, next);
    iters++;
    edges += act_deg;
    if (mv == 0) break;
    moves += mv;
    memcpy(labels, next, (size_t)n * sizeof(int32_t));
    i128 N_new = modularity_N(g, labels, &m2);
    if (below_tau(N_new - N_old, N_old)) break;
    N_old = N_new;
  }
  free(next);
  if (moves_out) *moves_out = moves;
  if (edges_out) *edges_out = edges;
  return iters;
}

/* ------------------------------------------------------------------ */
/* Graph compaction (Algorithm 1, "perform graph compaction")          */
/* ------------------------------------------------------------------ */

/* Communities become vertices: coarse id = rank of the label among the labels
 * in use, ascending.  Every fine entry (u,v,w) adds w to coarse entry
 * (c(u), c(v)); intra-community entries therefore land on the coarse self-loop,
 * which carries the internal directed weight, so d_w and m2 are preserved. */
orc_graph* orc_coarsen(const orc_graph* g, const int32_t* labels, int32_t* cid_of_v) {
  int64_t n = g->n;
  int32_t* rank = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  uint8_t* used = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int64_t v = 0; v < n; v++) used[labels[v]] = 1;
  int32_t nc = 0;
  for (int64_t c = 0; c < n; c++) rank[c] = used[c] ? nc++ : -1;
  int64_t nnz = g->row_ptr[n];
  triple* t = (triple*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(triple));
  for (int64_t u = 0; u < n; u++)
    for (int64_t e = g->row_ptr[u]; e < g->row_ptr[u + 1]; e++) {
      t[e].u = rank[labels[u]];
      t[e].v = rank[labels[g->col[e]]];
      t[e].w = g->w[e];
    }
  orc_graph* cg = graph_from_triples(nc, t, nnz);
  if (cid_of_v)
    for (int64_t v = 0; v < n; v++) cid_of_v[v] = rank[labels[v]];
  free(t); free(rank); free(used);
  return cg;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 (Delta-screening) and the deletion rule                 */
/* ------------------------------------------------------------------ */

typedef struct { int32_t i, j; } opair;

static int cmp_opair(const void* pa, const void* pb) {
  const opair* a = (const opair*)pa;
  const opair* b = (const opair*)pb;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  return (a->j > b->j) - (a->j < b->j);
}

/* Mark v and every neighbour of v in g. */
static void mark_closed_nbhd(const orc_graph* g, int32_t v, uint8_t* mark) {
  mark[v] = 1;
  for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) mark[g->col[e]] = 1;
}

/* Algorithm 2 on G_t with the labels C_{t-1}:
 *   the inserted edges as ordered pairs (i,j) and (j,i), sorted by source;
 *   per source i: j* = argmax over sinks j of S(i -> C_{t-1}(j)) (S = 0 when
 *   C_{t-1}(j) = C_{t-1}(i)); ties to the smaller C_{t-1}(j), then the smaller
 *   j (the paper fixes no tie rule);  gain1 = S(i -> C(j*)),
 *   gain2 = S(j* -> C(i));  if gain1 >= gain2 and gain1 > 0, add
 *   {i, j*} u Gamma(i) u C_{t-1}(j*) to R_t.  Gains are evaluated on G_t
 *   (m_t, degrees and community sums after the batch; the appendix proofs use
 *   m_t).  Screening changes no label (Sec. III-E).
 * Deletions are outside the paper (Sec. V lists them as future work).  Rule
 * taken here, for each ordered deleted pair (i,j) whose edge was in G_{t-1}:
 *   if C(i) = C(j): add i, j and Gamma_{G_t}(i) (i's tie to its community
 *   weakens, the mirror of Lemma 3.1);  otherwise add i and j. */
int orc_screen(const orc_graph* g_prev, const orc_graph* g_t, const int32_t* L,
               const int32_t* ins, int64_t n_ins, const int32_t* del, int64_t n_del,
               uint8_t* r_out) {
  int64_t n = g_t->n, m2;
  int64_t* k = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* a = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  uint8_t* mark = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  uint8_t* flag = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  opair* p = (opair*)malloc((size_t)(2 * n_ins > 0 ? 2 * n_ins : 1) * sizeof(opair));
  weighted_degrees(g_t, k, &m2);
  community_sums(n, L, k, a, NULL);

  for (int64_t x = 0; x < n_ins; x++) {
    p[2 * x].i = ins[3 * x]; p[2 * x].j = ins[3 * x + 1];
    p[2 * x + 1].i = ins[3 * x + 1]; p[2 * x + 1].j = ins[3 * x];
  }
  if (n_ins > 0) qsort(p, (size_t)(2 * n_ins), sizeof(opair), cmp_opair);

  for (int64_t s = 0; s < 2 * n_ins;) {
    int32_t i = p[s].i;
    int64_t e_end = s;
    while (e_end < 2 * n_ins && p[e_end].i == i) e_end++;
    int32_t jstar = -1;
    i128 g1 = 0;
    for (int64_t x = s; x < e_end; x++) {
      int32_t j = p[x].j;
      int32_t D = L[j];
      i128 S = 0;
      if (D != L[i])
        S = gain_S(m2, k[i], edge_weight_to(g_t, L, i, D), edge_weight_to(g_t, L, i, L[i]),
                   a[D], a[L[i]]);
      int better;
      if (jstar < 0) better = 1;
      else if (S != g1) better = S > g1;
      else if (D != L[jstar]) better = D < L[jstar];
      else better = j < jstar;
      if (better) { jstar = j; g1 = S; }
    }
    i128 g2 = 0;
    if (L[jstar] != L[i])
      g2 = gain_S(m2, k[jstar], edge_weight_to(g_t, L, jstar, L[i]),
                  edge_weight_to(g_t, L, jstar, L[jstar]), a[L[i]], a[L[jstar]]);
    if (g1 >= g2 && g1 > 0) {
      mark_closed_nbhd(g_t, i, mark);
      mark[jstar] = 1;
      flag[L[jstar]] = 1;
    }
    s = e_end;
  }

  for (int64_t x = 0; x < n_del; x++) {
    int32_t u = del[2 * x], v = del[2 * x + 1];
    if (find_entry(g_prev, u, v) < 0) continue; /* absent edge: no-op */
    for (int side = 0; side < 2; side++) {
      int32_t i = side ? v : u, j = side ? u : v;
      if (L[i] == L[j]) mark_closed_nbhd(g_t, i, mark);
      mark[i] = 1;
      mark[j] = 1;
    }
  }

  for (int64_t v = 0; v < n; v++) r_out[v] = (uint8_t)(mark[v] | flag[L[v]]);
  free(k); free(a); free(mark); free(flag); free(p);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1, outer loop                                             */
/* ------------------------------------------------------------------ */

/* Levels: run the inner loop; stop when no community merged two vertices
 * (nothing to compact), or when a level >= 1 gained at most 1e-6 of |Q|
 * ("no longer an appreciable modularity gain between successive levels",
 * Sec. III-B), or at 64 levels; otherwise compact and continue on the coarse
 * graph, every coarse vertex active and a singleton.  The level-0 active set
 * is R_t (Sec. III-D, step 2c: R_t is used at the first level only).
 * Output labels are canonical: the smallest member vertex id. */
int orc_louvain(const orc_graph* g0, const int32_t* init, const uint8_t* active0,
                int32_t* out, orc_stats* st) {
  int64_t n0 = g0->n;
  int32_t* comp = (int32_t*)malloc((size_t)(n0 > 0 ? n0 : 1) * sizeof(int32_t));
  int32_t* L = (int32_t*)malloc((size_t)(n0 > 0 ? n0 : 1) * sizeof(int32_t));
  for (int64_t v = 0; v < n0; v++) { comp[v] = (int32_t)v; L[v] = init[v]; }
  const orc_graph* g = g0;
  orc_graph* owned = NULL;
  const uint8_t* active = active0;
  int64_t m2;
  i128 N_start = modularity_N(g, L, &m2);
  i128 N_end = N_start;
  int64_t level = 0, iters_total = 0, iters0 = 0, moves_total = 0, edges_total = 0;
  for (;;) {
    int64_t moves = 0, edges = 0;
    int64_t it = orc_run_level(g, L, active, ORC_MAX_ITERS, &moves, &edges);
    iters_total += it;
    if (level == 0) iters0 = it;
    moves_total += moves;
    edges_total += edges;
    N_end = modularity_N(g, L, &m2);
    int64_t nv = g->n;
    uint8_t* used = (uint8_t*)calloc((size_t)(nv > 0 ? nv : 1), 1);
    int64_t nc = 0;
    for (int64_t v = 0; v < nv; v++) if (!used[L[v]]) { used[L[v]] = 1; nc++; }
    free(used);
    level++;
    if (nc == nv) break;
    if (level >= 2 && below_tau(N_end - N_start, N_start)) break;
    if (level >= ORC_MAX_LEVELS) break;
    int32_t* cid = (int32_t*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(int32_t));
    orc_graph* cg = orc_coarsen(g, L, cid);
    for (int64_t v = 0; v < n0; v++) comp[v] = cid[comp[v]];
    free(cid);
    if (owned) orc_graph_free(owned);
    owned = cg;
    g = cg;
    free(L);
    L = (int32_t*)malloc((size_t)(g->n > 0 ? g->n : 1) * sizeof(int32_t));
    for (int64_t v = 0; v < g->n; v++) L[v] = (int32_t)v;
    active = NULL;
    N_start = N_end;
  }
  /* compose: community of original v is the final-level label of its coarse vertex */
  int64_t nf = g->n;
  int32_t* minid = (int32_t*)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(int32_t));
  for (int64_t c = 0; c < nf; c++) minid[c] = INT32_MAX;
  for (int64_t v = 0; v < n0; v++) {
    int32_t c = L[comp[v]];
    if ((int32_t)v < minid[c]) minid[c] = (int32_t)v;
  }
  int64_t ncomm = 0;
  for (int64_t v = 0; v < n0; v++) {
    out[v] = minid[L[comp[v]]];
    if (out[v] == (int32_t)v) ncomm++;
  }
  if (st) {
    i128 N = modularity_N(g0, out, &m2);
    st->n = n0;
    st->nnz = g0->row_ptr[n0];
    st->m2 = m2;
    st->levels = level;
    st->iters_total = iters_total;
    st->iters_level0 = iters0;
    st->moves_total = moves_total;
    st->edges_scanned = edges_total;
    st->communities = ncomm;
    st->n_lo = (int64_t)(uint64_t)N;
    st->n_hi = (int64_t)(N >> 64);
    st->q = q_from(N, m2);
  }
  free(minid); free(comp); free(L);
  if (owned) orc_graph_free(owned);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Smart local moving (the paper's second host method, dSLM-Delta-s)   */
/* ------------------------------------------------------------------ */

/* The paper applies Delta-screening to SLM (Waltman and van Eck's smart
 * local moving) as well as to Louvain and defers to SLM's own definition.
 * Restated here in the synchronous, exact-integer form of the Louvain code
 * above, with these readings:
 *   - a local-move pass also offers every vertex an empty community (SLM's
 *     local moving does); vertex v's empty community is label n + v, chosen
 *     only when its gain is larger than every neighbouring community's; after
 *     each pass every community is renamed to its smallest member id;
 *   - passes alternate direction: an even pass moves vertices only to
 *     smaller labels, an odd pass only to larger ones (the empty community
 *     counts as larger).  SLM's coarse levels start from whole communities,
 *     and two communities that both prefer each other would otherwise swap
 *     their members in every synchronous pass; one direction per pass lets
 *     them merge, and replaces the singleton-swap guard of the Louvain code;
 *   - a level stops after a down-and-up cycle of two passes that moved
 *     nothing or gained at most 1e-6 of |Q|, or after 500 passes;
 *   - refinement: each community is split by local moving from singletons
 *     restricted to the edges inside it, with the gains of the whole graph
 *     (k_v and 2m of the graph, a over the sub-communities), so it optimises
 *     the same modularity; it moves nothing between communities and runs over
 *     every vertex;
 *   - aggregation: sub-communities become vertices (rank of the sub label),
 *     each starting in the community that holds it (named by its smallest
 *     coarse member); the run stops when every sub-community is a single
 *     vertex, when a level >= 1 gained at most 1e-6 of |Q|, or at 64 levels;
 *   - Delta-screening: R_t restricts the local moving of level 0 only. */

/* The SLM choice for one vertex from a snapshot.  parent (NULL = none)
 * restricts the candidates to neighbours in v's parent community; up (0 or 1)
 * is the pass direction: only labels below C, or only above (empty included). */
static int32_t slm_best_move(const orc_graph* g, const int32_t* labels, const int32_t* parent,
                             const int64_t* k, const int64_t* a, const int64_t* size, int64_t m2,
                             int32_t v, int up, lw* buf) {
  int32_t C = labels[v];
  int64_t cnt = 0;
  for (int64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; e++) {
    int32_t u = g->col[e];
    if (u == v || (parent && parent[u] != parent[v])) continue;
    buf[cnt].label = labels[u];
    buf[cnt].w = g->w[e];
    cnt++;
  }
  qsort(buf, (size_t)cnt, sizeof(lw), cmp_lw);
  int64_t eC = 0;
  for (int64_t i = 0; i < cnt; i++) if (buf[i].label == C) eC += buf[i].w;
  int32_t best = C;
  i128 bestS = 0;
  for (int64_t i = 0; i < cnt;) {
    int32_t D = buf[i].label;
    int64_t eD = 0;
    int64_t j = i;
    while (j < cnt && buf[j].label == D) eD += buf[j++].w;
    i = j;
    if (D == C || (up ? D < C : D > C)) continue;
    i128 S = gain_S(m2, k[v], eD, eC, a[D], a[C]);
    if (S > bestS) { bestS = S; best = D; }
  }
  if (up && size[C] > 1) {
    i128 S0 = gain_S(m2, k[v], 0, eC, 0, a[C]);  /* into an empty community */
    if (S0 > bestS) return (int32_t)(g->n + v);
  }
  return best;
}

/* Every community named by its smallest member (labels in [0, 2n) in, [0, n) out). */
static void canonical(int64_t n, int32_t* labels, int32_t* minid /* 2n scratch */) {
  for (int64_t c = 0; c < 2 * n; c++) minid[c] = INT32_MAX;
  for (int64_t v = 0; v < n; v++)
    if ((int32_t)v < minid[labels[v]]) minid[labels[v]] = (int32_t)v;
  for (int64_t v = 0; v < n; v++) labels[v] = minid[labels[v]];
}

/* One synchronous SLM pass; labels canonical on entry and exit.  Returns movers. */
static int64_t slm_pass(const orc_graph* g, int32_t* labels, const int32_t* parent,
                        const uint8_t* active, int up, const int64_t* k, int64_t m2, lw* buf,
                        int32_t* next, int32_t* scratch) {
  int64_t n = g->n, moves = 0;
  int64_t* a = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* size = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  community_sums(n, labels, k, a, size);
  for (int64_t v = 0; v < n; v++) {
    next[v] = labels[v];
    if (active && !active[v]) continue;
    next[v] = slm_best_move(g, labels, parent, k, a, size, m2, (int32_t)v, up, buf);
    if (next[v] != labels[v]) moves++;
  }
  memcpy(labels, next, (size_t)n * sizeof(int32_t));
  canonical(n, labels, scratch);
  free(a); free(size);
  return moves;
}

/* Passes to convergence: down-and-up cycles until a cycle moves nothing or
 * gains at most 1e-6 of |Q| of the partition being moved, or 500 passes.
 * Returns the number of passes. */
static int64_t slm_level(const orc_graph* g, int32_t* labels, const int32_t* parent,
                         const uint8_t* active, int64_t* moves_out, int64_t* edges_out) {
  int64_t n = g->n, m2, iters = 0, moves = 0, edges = 0, act_deg = 0, maxdeg = 1;
  int64_t* k = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int32_t* next = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t* scratch = (int32_t*)malloc((size_t)(n > 0 ? 2 * n : 2) * sizeof(int32_t));
  weighted_degrees(g, k, &m2);
  for (int64_t v = 0; v < n; v++) {
    int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
    if (d > maxdeg) maxdeg = d;
    if (!active || active[v]) act_deg += d;
  }
  lw* buf = (lw*)malloc((size_t)maxdeg * sizeof(lw));
  i128 N_old = modularity_N(g, labels, &m2);
  int64_t cycle_moves = 0;
  while (iters < ORC_MAX_ITERS) {
    const int up = (int)(iters & 1);
    int64_t mv = slm_pass(g, labels, parent, active, up, k, m2, buf, next, scratch);
    iters++;
    edges += act_deg;
    moves += mv;
    cycle_moves += mv;
    if (!up) continue;
    if (cycle_moves == 0) break;
    cycle_moves = 0;
    i128 N_new = modularity_N(g, labels, &m2);
    if (below_tau(N_new - N_old, N_old)) break;
    N_old = N_new;
  }
  free(buf); free(k); free(next); free(scratch);
  if (moves_out) *moves_out = moves;
  if (edges_out) *edges_out = edges;
  return iters;
}

int64_t orc_slm_refine(const orc_graph* g, const int32_t* parent, int32_t* sub, int64_t* moves) {
  for (int64_t v = 0; v < g->n; v++) sub[v] = (int32_t)v;
  return slm_level(g, sub, parent, NULL, moves, NULL);
}

int64_t orc_slm_level(const orc_graph* g, int32_t* labels, const uint8_t* active, int64_t* moves) {
  int32_t* scratch = (int32_t*)malloc((size_t)(g->n > 0 ? 2 * g->n : 2) * sizeof(int32_t));
  canonical(g->n, labels, scratch);
  free(scratch);
  return slm_level(g, labels, NULL, active, moves, NULL);
}

int orc_slm(const orc_graph* g0, const int32_t* init, const uint8_t* active0, int32_t* out,
            orc_stats* st) {
  int64_t n0 = g0->n;
  int32_t* comp = (int32_t*)malloc((size_t)(n0 > 0 ? n0 : 1) * sizeof(int32_t));
  int32_t* L = (int32_t*)malloc((size_t)(n0 > 0 ? n0 : 1) * sizeof(int32_t));
  int32_t* scratch = (int32_t*)malloc((size_t)(n0 > 0 ? 2 * n0 : 2) * sizeof(int32_t));
  for (int64_t v = 0; v < n0; v++) { comp[v] = (int32_t)v; L[v] = init[v]; }
  canonical(n0, L, scratch);
  free(scratch);
  const orc_graph* g = g0;
  orc_graph* owned = NULL;
  const uint8_t* active = active0;
  int64_t m2;
  i128 N_start = modularity_N(g, L, &m2);
  int64_t level = 0, iters_total = 0, iters0 = 0, moves_total = 0, edges_total = 0;
  int64_t refine_iters = 0, refine_moves = 0;
  for (;;) {
    int64_t moves = 0, edges = 0;
    int64_t it = slm_level(g, L, NULL, active, &moves, &edges);
    iters_total += it;
    if (level == 0) iters0 = it;
    moves_total += moves;
    edges_total += edges;
    i128 N_end = modularity_N(g, L, &m2);
    int64_t nv = g->n;
    int32_t* sub = (int32_t*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(int32_t));
    int64_t rmoves = 0;
    refine_iters += orc_slm_refine(g, L, sub, &rmoves);
    refine_moves += rmoves;
    int64_t ns = 0;
    for (int64_t v = 0; v < nv; v++) if (sub[v] == (int32_t)v) ns++;  /* canonical: one min member each */
    level++;
    int stop = ns == nv || (level >= 2 && below_tau(N_end - N_start, N_start)) || level >= ORC_MAX_LEVELS;
    if (stop) { free(sub); break; }
    int32_t* cid = (int32_t*)malloc((size_t)(nv > 0 ? nv : 1) * sizeof(int32_t));
    orc_graph* cg = orc_coarsen(g, sub, cid);
    for (int64_t v = 0; v < n0; v++) comp[v] = cid[comp[v]];
    /* coarse start: the community holding the sub-community, named by its
     * smallest coarse member (the sub-community of the community's smallest
     * fine member, since coarse ids rank the sub labels) */
    int32_t* Lc = (int32_t*)malloc((size_t)(cg->n > 0 ? cg->n : 1) * sizeof(int32_t));
    for (int64_t v = 0; v < nv; v++) Lc[cid[v]] = cid[L[v]];
    free(cid); free(sub);
    if (owned) orc_graph_free(owned);
    owned = cg;
    g = cg;
    free(L);
    L = Lc;
    active = NULL;
    N_start = N_end;
  }
  int64_t nf = g->n;
  int32_t* minid = (int32_t*)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(int32_t));
  for (int64_t c = 0; c < nf; c++) minid[c] = INT32_MAX;
  for (int64_t v = 0; v < n0; v++) {
    int32_t c = L[comp[v]];
    if ((int32_t)v < minid[c]) minid[c] = (int32_t)v;
  }
  int64_t ncomm = 0;
  for (int64_t v = 0; v < n0; v++) {
    out[v] = minid[L[comp[v]]];
    if (out[v] == (int32_t)v) ncomm++;
  }
  if (st) {
    i128 N = modularity_N(g0, out, &m2);
    st->n = n0;
    st->nnz = g0->row_ptr[n0];
    st->m2 = m2;
    st->levels = level;
    st->iters_total = iters_total;
    st->iters_level0 = iters0;
    st->moves_total = moves_total;
    st->edges_scanned = edges_total;
    st->communities = ncomm;
    st->n_lo = (int64_t)(uint64_t)N;
    st->n_hi = (int64_t)(N >> 64);
    st->q = q_from(N, m2);
    st->refine_iters = refine_iters;
    st->refine_moves = refine_moves;
  }
  free(minid); free(comp); free(L);
  if (owned) orc_graph_free(owned);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Incremental driver (Sec. III-D)                                     */
/* ------------------------------------------------------------------ */

struct orc_ctx {
  int64_t n;
  int64_t t;          /* time steps computed so far */
  orc_graph* g;       /* G_{t} after the last update */
  int32_t* labels;    /* C_t, canonical */
  uint8_t* rset;      /* R_t of the last update */
  int32_t* ins; int64_t n_ins, cap_ins;
  int32_t* del; int64_t n_del, cap_del;
};

orc_ctx* orc_create(int64_t n) {
  if (n <= 0 || n > INT32_MAX) return NULL;
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  c->n = n;
  c->g = graph_alloc(n, 0);
  c->labels = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  c->rset = (uint8_t*)calloc((size_t)n, 1);
  for (int64_t v = 0; v < n; v++) c->labels[v] = (int32_t)v;
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  orc_graph_free(c->g);
  free(c->labels); free(c->rset); free(c->ins); free(c->del); free(c);
}

/* Batches staged before one update concatenate into one Delta_t. */
int orc_apply_batch(orc_ctx* c, const int32_t* ins, int64_t n_ins, const int32_t* del,
                    int64_t n_del) {
  for (int64_t i = 0; i < n_ins; i++) {
    int32_t u = ins[3 * i], v = ins[3 * i + 1], w = ins[3 * i + 2];
    if (u < 0 || v < 0 || u >= c->n || v >= c->n || u == v || w <= 0) return ORC_EINVAL;
  }
  for (int64_t i = 0; i < n_del; i++) {
    int32_t u = del[2 * i], v = del[2 * i + 1];
    if (u < 0 || v < 0 || u >= c->n || v >= c->n || u == v) return ORC_EINVAL;
  }
  if (c->n_ins + n_ins > c->cap_ins) {
    int64_t cap = 2 * (c->n_ins + n_ins);
    c->ins = (int32_t*)realloc(c->ins, (size_t)cap * 3 * sizeof(int32_t));
    c->cap_ins = cap;
  }
  if (c->n_del + n_del > c->cap_del) {
    int64_t cap = 2 * (c->n_del + n_del);
    c->del = (int32_t*)realloc(c->del, (size_t)cap * 2 * sizeof(int32_t));
    c->cap_del = cap;
  }
  if (n_ins) memcpy(c->ins + 3 * c->n_ins, ins, (size_t)n_ins * 3 * sizeof(int32_t));
  if (n_del) memcpy(c->del + 2 * c->n_del, del, (size_t)n_del * 2 * sizeof(int32_t));
  c->n_ins += n_ins;
  c->n_del += n_del;
  return ORC_OK;
}

/* Step 1 (t = 1): Static(G_1).  Step 2 (t > 1): (a) every vertex keeps its
 * label C_{t-1}(i) (the vertex set is fixed, so an isolated vertex is its own
 * singleton community); (b) R_t = Delta-screening(G_t, Delta_t) in DELTA
 * mode, V_t in BASE mode (dLouvain-base, Sec. III-D), the caller's set in
 * GIVEN_R mode; (c) the multi-level run with R_t at level 0.  STATIC runs
 * Static(G_t) from scratch (the naive approach, Sec. III-C). */
int orc_update(orc_ctx* c, int mode, const uint8_t* r_given, int32_t* labels_out,
               double* q_out, orc_stats* st) {
  return orc_update_alg(c, ORC_LOUVAIN, mode, r_given, labels_out, q_out, st);
}

int orc_update_alg(orc_ctx* c, int alg, int mode, const uint8_t* r_given, int32_t* labels_out,
                   double* q_out, orc_stats* st) {
  if (alg != ORC_LOUVAIN && alg != ORC_SLM) return ORC_EINVAL;
  int err;
  int64_t n = c->n;
  orc_graph* gt = orc_apply(c->g, c->ins, c->n_ins, c->del, c->n_del, NULL, &err);
  if (!gt) return err;
  int32_t* init = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int first = (c->t == 0);
  if (first || mode == ORC_STATIC) {
    for (int64_t v = 0; v < n; v++) { init[v] = (int32_t)v; c->rset[v] = 1; }
  } else {
    memcpy(init, c->labels, (size_t)n * sizeof(int32_t));
    if (mode == ORC_BASE) memset(c->rset, 1, (size_t)n);
    else if (mode == ORC_GIVEN_R) memcpy(c->rset, r_given, (size_t)n);
    else orc_screen(c->g, gt, c->labels, c->ins, c->n_ins, c->del, c->n_del, c->rset);
  }
  orc_stats s;
  memset(&s, 0, sizeof(s));
  if (alg == ORC_SLM) orc_slm(gt, init, c->rset, c->labels, &s);
  else orc_louvain(gt, init, c->rset, c->labels, &s);
  free(init);
  int64_t r = 0;
  for (int64_t v = 0; v < n; v++) r += c->rset[v];
  c->t += 1;
  s.t = c->t;
  s.r_size = r;
  orc_graph_free(c->g);
  c->g = gt;
  c->n_ins = c->n_del = 0;
  if (labels_out) memcpy(labels_out, c->labels, (size_t)n * sizeof(int32_t));
  if (q_out) *q_out = s.q;
  if (st) *st = s;
  return ORC_OK;
}

int orc_get_rset(const orc_ctx* c, uint8_t* r_out) {
  memcpy(r_out, c->rset, (size_t)c->n);
  return ORC_OK;
}

const orc_graph* orc_ctx_graph(const orc_ctx* c) { return c->g; }

/* A deep copy of the whole context: G_t, C_t, R_t, t and any staged batch.
 * Test and timing infrastructure only (a timed step can start again from one
 * saved state); it computes nothing. */
orc_ctx* orc_clone(const orc_ctx* c) {
  if (!c) return NULL;
  orc_ctx* d = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  if (!d) return NULL;
  d->n = c->n;
  d->t = c->t;
  d->g = orc_graph_new(c->n, c->g->row_ptr, c->g->col, c->g->w);
  d->labels = (int32_t*)malloc((size_t)c->n * sizeof(int32_t));
  d->rset = (uint8_t*)malloc((size_t)c->n);
  if (!d->g || !d->labels || !d->rset) {
    orc_destroy(d);
    return NULL;
  }
  memcpy(d->labels, c->labels, (size_t)c->n * sizeof(int32_t));
  memcpy(d->rset, c->rset, (size_t)c->n);
  if (c->n_ins) {
    d->ins = (int32_t*)malloc((size_t)c->n_ins * 3 * sizeof(int32_t));
    memcpy(d->ins, c->ins, (size_t)c->n_ins * 3 * sizeof(int32_t));
    d->n_ins = d->cap_ins = c->n_ins;
  }
  if (c->n_del) {
    d->del = (int32_t*)malloc((size_t)c->n_del * 2 * sizeof(int32_t));
    memcpy(d->del, c->del, (size_t)c->n_del * 2 * sizeof(int32_t));
    d->n_del = d->cap_del = c->n_del;
  }
  return d;
}

int orc_set_labels(orc_ctx* c, const int32_t* labels) {
  for (int64_t v = 0; v < c->n; v++)
    if (labels[v] < 0 || labels[v] >= c->n) return ORC_EINVAL;
  memcpy(c->labels, labels, (size_t)c->n * sizeof(int32_t));
  if (c->t == 0) c->t = 1;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Learned-screen features (not in the paper)                          */
/* ------------------------------------------------------------------ */

/* Pool = R_t of Delta-screening, every vertex with a batch change, and the
 * G_t-neighbours of those.  For each pool vertex of positive degree, under
 * labels L (= C_{t-1}) on G_t, twelve float32 features (row v of X):
 *   log1p(deg), log1p(d_w), log1p(#inserted sinks), log1p(#deleted present
 *   sinks), inserted weight / d_w (at most 1), e_{v->C\v}/d_w, e_{v->D*}/d_w,
 *   S(v->D*)/(d_w 2m), a_C/2m, a_{D*}/2m, log1p(|C|), [v in R_t];
 * D* = the other neighbouring community of largest S (ties: smaller label).
 * pool_out[v] = 1 for the rows written. */
int orc_screen_features(const orc_graph* g_prev, const orc_graph* g_t, const int32_t* L, const int32_t* ins,
                        int64_t n_ins, const int32_t* del, int64_t n_del, const uint8_t* rds, uint8_t* pool_out,
                        float* X) {
  int64_t n = g_t->n, m2;
  int64_t* k = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* a = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* size = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  uint8_t* touched = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  weighted_degrees(g_t, k, &m2);
  community_sums(n, L, k, a, size);
  for (int64_t x = 0; x < n_ins; x++) { touched[ins[3 * x]] = 1; touched[ins[3 * x + 1]] = 1; }
  for (int64_t x = 0; x < n_del; x++) { touched[del[2 * x]] = 1; touched[del[2 * x + 1]] = 1; }
  for (int64_t v = 0; v < n; v++) pool_out[v] = rds[v] | touched[v];
  for (int64_t v = 0; v < n; v++)
    if (touched[v])
      for (int64_t e = g_t->row_ptr[v]; e < g_t->row_ptr[v + 1]; e++) pool_out[g_t->col[e]] = 1;
  /* distinct insert sinks, their summed weight, and distinct deleted sinks
   * whose edge was in G_{t-1}, per source (both orientations) */
  int64_t* nins = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t* ndel = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int64_t* wins = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  {
    opair* p = (opair*)malloc((size_t)(2 * n_ins > 0 ? 2 * n_ins : 1) * sizeof(opair));
    for (int64_t x = 0; x < n_ins; x++) {
      p[2 * x].i = ins[3 * x]; p[2 * x].j = ins[3 * x + 1];
      p[2 * x + 1].i = ins[3 * x + 1]; p[2 * x + 1].j = ins[3 * x];
      wins[ins[3 * x]] += ins[3 * x + 2];
      wins[ins[3 * x + 1]] += ins[3 * x + 2];
    }
    if (n_ins) qsort(p, (size_t)(2 * n_ins), sizeof(opair), cmp_opair);
    for (int64_t x = 0; x < 2 * n_ins; x++)
      if (x == 0 || p[x].i != p[x - 1].i || p[x].j != p[x - 1].j) nins[p[x].i]++;
    free(p);
    p = (opair*)malloc((size_t)(2 * n_del > 0 ? 2 * n_del : 1) * sizeof(opair));
    int64_t m = 0;
    for (int64_t x = 0; x < n_del; x++) {
      if (find_entry(g_prev, del[2 * x], del[2 * x + 1]) < 0) continue;
      p[m].i = del[2 * x]; p[m].j = del[2 * x + 1]; m++;
      p[m].i = del[2 * x + 1]; p[m].j = del[2 * x]; m++;
    }
    if (m) qsort(p, (size_t)m, sizeof(opair), cmp_opair);
    for (int64_t x = 0; x < m; x++)
      if (x == 0 || p[x].i != p[x - 1].i || p[x].j != p[x - 1].j) ndel[p[x].i]++;
    free(p);
  }
  int64_t maxdeg = 1;
  for (int64_t v = 0; v < n; v++)
    if (g_t->row_ptr[v + 1] - g_t->row_ptr[v] > maxdeg) maxdeg = g_t->row_ptr[v + 1] - g_t->row_ptr[v];
  lw* buf = (lw*)malloc((size_t)maxdeg * sizeof(lw));
  for (int64_t v = 0; v < n; v++) {
    int64_t deg = g_t->row_ptr[v + 1] - g_t->row_ptr[v];
    if (!pool_out[v] || deg == 0) { pool_out[v] = 0; continue; }
    int32_t C = L[v];
    int64_t cnt = 0;
    for (int64_t e = g_t->row_ptr[v]; e < g_t->row_ptr[v + 1]; e++) {
      if (g_t->col[e] == v) continue;
      buf[cnt].label = L[g_t->col[e]];
      buf[cnt].w = g_t->w[e];
      cnt++;
    }
    if (cnt) qsort(buf, (size_t)cnt, sizeof(lw), cmp_lw);
    int64_t eC = 0;
    for (int64_t i = 0; i < cnt; i++) if (buf[i].label == C) eC += buf[i].w;
    int32_t D = -1;
    int64_t eD = 0;
    i128 SD = 0;
    for (int64_t i = 0; i < cnt;) {
      int32_t lab = buf[i].label;
      int64_t s = 0;
      int64_t j = i;
      while (j < cnt && buf[j].label == lab) s += buf[j++].w;
      i = j;
      if (lab == C) continue;
      i128 S = gain_S(m2, k[v], s, eC, a[lab], a[C]);
      if (D < 0 || S > SD) { D = lab; eD = s; SD = S; }
    }
    float* x = X + v * 12;
    float fk = (float)k[v], fm = (float)m2;
    x[0] = log1pf((float)deg);
    x[1] = log1pf(fk);
    x[2] = log1pf((float)nins[v]);
    x[3] = log1pf((float)ndel[v]);
    x[4] = k[v] > 0 ? fminf((float)wins[v] / fk, 1.f) : 0.f;
    x[5] = k[v] > 0 ? (float)eC / fk : 0.f;
    x[6] = k[v] > 0 ? (float)eD / fk : 0.f;
    x[7] = (k[v] > 0 && m2 > 0 && D >= 0) ? (float)((double)SD / ((double)k[v] * (double)m2)) : 0.f;
    x[8] = m2 > 0 ? (float)a[C] / fm : 0.f;
    x[9] = (m2 > 0 && D >= 0) ? (float)a[D] / fm : 0.f;
    x[10] = log1pf((float)size[C]);
    x[11] = rds[v] ? 1.f : 0.f;
  }
  free(buf); free(k); free(a); free(size); free(touched); free(nins); free(ndel); free(wins);
  return ORC_OK;
}
