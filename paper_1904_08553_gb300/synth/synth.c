/*
 * synth.c -- seeded synthetic temporal graph streams.
 *
 * Input generators only: this file holds none of the community-detection
 * arithmetic.  It serves the CUDA library's tests and benchmark and the CPU
 * oracle's tests alike, and produces, per time step, a list of inserted edges
 * (u, v, w) and a list of deleted edges (u, v).
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), one stream per generator
 * seeded by the caller.  Bounded integers use the multiply-shift map of
 * Lemire (2019); reals are the top 53 bits scaled to [0,1).
 *
 * Workload shapes stand in for the paper's inputs (Sec. IV-A, Table I):
 *   temporal SBM        -- the MIT Graph Challenge streaming block models
 *   LFR-style power law -- sx-stackoverflow (2.6M vertices, 63M temporal edges)
 *   R-MAT               -- a large skewed graph
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- RNG ---------------- */

typedef struct { uint64_t s; } rng;

static inline uint64_t rnext(rng* r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline double runif(rng* r) { return (double)(rnext(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline uint64_t rbelow(rng* r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)rnext(r) * (unsigned __int128)n) >> 64);
}

/* ---------------- edge set: dense list + open-addressing index ---------------- */

typedef struct {
  uint64_t* items;  /* dense list of keys (min << 32 | max) */
  int64_t count, cap_items;
  uint64_t* hk;     /* table keys, EMPTY = ~0 */
  int64_t* hv;      /* index into items */
  int64_t hcap;     /* power of two */
} edgeset;

#define ES_EMPTY (~(uint64_t)0)

static inline uint64_t ekey(int32_t u, int32_t v) {
  uint32_t a = (uint32_t)(u < v ? u : v), b = (uint32_t)(u < v ? v : u);
  return ((uint64_t)a << 32) | b;
}
static inline uint64_t hmix(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL;
  return x ^ (x >> 33);
}

static int es_init(edgeset* s, int64_t expect) {
  memset(s, 0, sizeof(*s));
  int64_t cap = 16;
  while (cap < 2 * expect + 16) cap <<= 1;
  s->hcap = cap;
  s->hk = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
  s->hv = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
  s->cap_items = expect + 16;
  s->items = (uint64_t*)malloc((size_t)s->cap_items * sizeof(uint64_t));
  if (!s->hk || !s->hv || !s->items) return -1;
  for (int64_t i = 0; i < cap; i++) s->hk[i] = ES_EMPTY;
  return 0;
}
static void es_free(edgeset* s) { free(s->items); free(s->hk); free(s->hv); }

static int64_t es_find_slot(const edgeset* s, uint64_t k) {
  int64_t m = s->hcap - 1, i = (int64_t)(hmix(k) & (uint64_t)m);
  while (s->hk[i] != ES_EMPTY && s->hk[i] != k) i = (i + 1) & m;
  return i;
}
static int es_has(const edgeset* s, uint64_t k) { return s->hk[es_find_slot(s, k)] == k; }

static void es_grow(edgeset* s) {
  int64_t old = s->hcap;
  uint64_t* ok = s->hk;
  int64_t* ov = s->hv;
  s->hcap = old * 2;
  s->hk = (uint64_t*)malloc((size_t)s->hcap * sizeof(uint64_t));
  s->hv = (int64_t*)malloc((size_t)s->hcap * sizeof(int64_t));
  for (int64_t i = 0; i < s->hcap; i++) s->hk[i] = ES_EMPTY;
  for (int64_t i = 0; i < old; i++)
    if (ok[i] != ES_EMPTY) {
      int64_t j = es_find_slot(s, ok[i]);
      s->hk[j] = ok[i]; s->hv[j] = ov[i];
    }
  free(ok); free(ov);
}

/* Returns 1 if newly added. */
static int es_add(edgeset* s, uint64_t k) {
  int64_t i = es_find_slot(s, k);
  if (s->hk[i] == k) return 0;
  if (s->count == s->cap_items) {
    s->cap_items *= 2;
    s->items = (uint64_t*)realloc(s->items, (size_t)s->cap_items * sizeof(uint64_t));
  }
  s->hk[i] = k; s->hv[i] = s->count;
  s->items[s->count++] = k;
  if (2 * s->count > s->hcap) es_grow(s);
  return 1;
}

/* Remove by key (swap-with-last in the dense list, backward-shift delete). */
static void es_remove(edgeset* s, uint64_t k) {
  int64_t m = s->hcap - 1;
  int64_t i = es_find_slot(s, k);
  if (s->hk[i] != k) return;
  int64_t pos = s->hv[i];
  uint64_t last = s->items[s->count - 1];
  s->items[pos] = last;
  s->count--;
  if (last != k) s->hv[es_find_slot(s, last)] = pos;
  int64_t j = i;
  for (;;) {
    j = (j + 1) & m;
    if (s->hk[j] == ES_EMPTY) break;
    int64_t h = (int64_t)(hmix(s->hk[j]) & (uint64_t)m);
    /* move entry j into the hole i when its home h does not lie in (i, j] */
    int inrange = (i <= j) ? (h > i && h <= j) : (h > i || h <= j);
    if (!inrange) { s->hk[i] = s->hk[j]; s->hv[i] = s->hv[j]; i = j; }
  }
  s->hk[i] = ES_EMPTY;
}

/* ---------------- stream container ---------------- */

typedef struct {
  int64_t n;
  int32_t steps;
  int32_t* ins; int64_t n_ins, cap_ins;   /* triples */
  int32_t* del; int64_t n_del, cap_del;   /* pairs */
  int64_t* ins_off; int64_t* del_off;     /* steps + 1 */
  int32_t* planted;                       /* planted community at the last step */
} dcdsyn_stream;

static void st_push_ins(dcdsyn_stream* s, int32_t u, int32_t v, int32_t w) {
  if (s->n_ins == s->cap_ins) {
    s->cap_ins = s->cap_ins ? 2 * s->cap_ins : 1024;
    s->ins = (int32_t*)realloc(s->ins, (size_t)s->cap_ins * 3 * sizeof(int32_t));
  }
  int32_t* p = s->ins + 3 * s->n_ins++;
  p[0] = u; p[1] = v; p[2] = w;
}
static void st_push_del(dcdsyn_stream* s, int32_t u, int32_t v) {
  if (s->n_del == s->cap_del) {
    s->cap_del = s->cap_del ? 2 * s->cap_del : 1024;
    s->del = (int32_t*)realloc(s->del, (size_t)s->cap_del * 2 * sizeof(int32_t));
  }
  int32_t* p = s->del + 2 * s->n_del++;
  p[0] = u; p[1] = v;
}
static dcdsyn_stream* st_new(int64_t n, int32_t steps) {
  dcdsyn_stream* s = (dcdsyn_stream*)calloc(1, sizeof(dcdsyn_stream));
  s->n = n; s->steps = steps;
  s->ins_off = (int64_t*)calloc((size_t)steps + 1, sizeof(int64_t));
  s->del_off = (int64_t*)calloc((size_t)steps + 1, sizeof(int64_t));
  s->planted = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  return s;
}
static void st_close_step(dcdsyn_stream* s, int32_t t) {
  s->ins_off[t + 1] = s->n_ins;
  s->del_off[t + 1] = s->n_del;
}

void dcdsyn_free(dcdsyn_stream* s) {
  if (!s) return;
  free(s->ins); free(s->del); free(s->ins_off); free(s->del_off); free(s->planted); free(s);
}
int64_t dcdsyn_n(const dcdsyn_stream* s) { return s->n; }
int32_t dcdsyn_steps(const dcdsyn_stream* s) { return s->steps; }
int64_t dcdsyn_n_ins(const dcdsyn_stream* s, int32_t t) { return s->ins_off[t + 1] - s->ins_off[t]; }
int64_t dcdsyn_n_del(const dcdsyn_stream* s, int32_t t) { return s->del_off[t + 1] - s->del_off[t]; }
void dcdsyn_copy_ins(const dcdsyn_stream* s, int32_t t, int32_t* out) {
  memcpy(out, s->ins + 3 * s->ins_off[t], (size_t)dcdsyn_n_ins(s, t) * 3 * sizeof(int32_t));
}
void dcdsyn_copy_del(const dcdsyn_stream* s, int32_t t, int32_t* out) {
  memcpy(out, s->del + 2 * s->del_off[t], (size_t)dcdsyn_n_del(s, t) * 2 * sizeof(int32_t));
}
void dcdsyn_copy_planted(const dcdsyn_stream* s, int32_t* out) {
  memcpy(out, s->planted, (size_t)s->n * sizeof(int32_t));
}

static void shuffle_i32(rng* r, int32_t* a, int64_t n) {
  for (int64_t i = n - 1; i > 0; i--) {
    int64_t j = (int64_t)rbelow(r, (uint64_t)i + 1);
    int32_t t = a[i]; a[i] = a[j]; a[j] = t;
  }
}

/* Delete `count` distinct edges chosen uniformly from the current set. */
static void delete_uniform(rng* r, edgeset* es, dcdsyn_stream* s, int64_t count) {
  if (count > es->count) count = es->count;
  for (int64_t x = 0; x < count; x++) {
    int64_t idx = (int64_t)rbelow(r, (uint64_t)es->count);
    uint64_t k = es->items[idx];
    st_push_del(s, (int32_t)(k >> 32), (int32_t)(k & 0xffffffffu));
    es_remove(es, k);
  }
}

/* ---------------- temporal stochastic block model ---------------- */

/* Vertices get blocks from the sizes list through a seeded permutation.
 * Step 1 inserts exactly m_intra distinct uniform intra-block pairs and
 * m_inter distinct uniform inter-block pairs.  Each later step first deletes
 * del_count (or del_frac of the current edges) distinct edges chosen
 * uniformly, then inserts ins_count (or ins_frac of the current edges) pairs
 * absent from the previous graph, a fraction intra_frac of them intra-block.
 * All weights are 1. */
dcdsyn_stream* dcdsyn_sbm(uint64_t seed, int64_t n, int64_t nblocks, const int64_t* sizes,
                          int64_t m_intra, int64_t m_inter, int32_t steps, int64_t ins_count,
                          double ins_frac, int64_t del_count, double del_frac,
                          double intra_frac) {
  rng r = {seed};
  int64_t tot = 0;
  for (int64_t b = 0; b < nblocks; b++) tot += sizes[b];
  if (tot != n || n <= 1 || steps < 1) return NULL;
  dcdsyn_stream* s = st_new(n, steps);
  int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  for (int64_t v = 0; v < n; v++) perm[v] = (int32_t)v;
  shuffle_i32(&r, perm, n);
  /* members[block_off[b] .. block_off[b+1]) are the vertices of block b */
  int64_t* boff = (int64_t*)malloc((size_t)(nblocks + 1) * sizeof(int64_t));
  double* pcum = (double*)malloc((size_t)nblocks * sizeof(double));
  boff[0] = 0;
  for (int64_t b = 0; b < nblocks; b++) boff[b + 1] = boff[b] + sizes[b];
  int32_t* block = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  for (int64_t b = 0; b < nblocks; b++)
    for (int64_t x = boff[b]; x < boff[b + 1]; x++) block[perm[x]] = (int32_t)b;
  double acc = 0;
  for (int64_t b = 0; b < nblocks; b++) {
    acc += (double)sizes[b] * (double)(sizes[b] - 1) * 0.5;
    pcum[b] = acc;
  }
  memcpy(s->planted, block, (size_t)n * sizeof(int32_t));

  int64_t expect = m_intra + m_inter + 16;
  if (ins_count > 0) expect += (int64_t)steps * ins_count;
  else expect = (int64_t)((double)expect * pow(1.0 + ins_frac, steps)) + 16;
  edgeset es;
  es_init(&es, expect);
  edgeset prev; /* edges of G_{t-1} at the start of a step */
  memset(&prev, 0, sizeof(prev));

  for (int32_t t = 0; t < steps; t++) {
    int64_t want_intra, want_inter;
    if (t == 0) {
      want_intra = m_intra; want_inter = m_inter;
    } else {
      int64_t dc = del_count > 0 ? del_count : (int64_t)llround(del_frac * (double)es.count);
      int64_t ic = ins_count > 0 ? ins_count : (int64_t)llround(ins_frac * (double)es.count);
      /* absent from G_{t-1}: remember G_{t-1} before deleting */
      es_free(&prev);
      es_init(&prev, es.count + 16);
      for (int64_t x = 0; x < es.count; x++) es_add(&prev, es.items[x]);
      delete_uniform(&r, &es, s, dc);
      want_intra = (int64_t)llround(intra_frac * (double)ic);
      want_inter = ic - want_intra;
    }
    int64_t got = 0, guard = 0;
    while (got < want_intra && guard < 1000 * (want_intra + 10)) {
      guard++;
      double x = runif(&r) * acc;
      int64_t lo = 0, hi = nblocks - 1;
      while (lo < hi) { int64_t mid = (lo + hi) / 2; if (pcum[mid] > x) hi = mid; else lo = mid + 1; }
      int64_t sz = sizes[lo];
      if (sz < 2) continue;
      int32_t u = perm[boff[lo] + (int64_t)rbelow(&r, (uint64_t)sz)];
      int32_t v = perm[boff[lo] + (int64_t)rbelow(&r, (uint64_t)sz)];
      if (u == v) continue;
      uint64_t k = ekey(u, v);
      if (t > 0 && es_has(&prev, k)) continue;
      if (!es_add(&es, k)) continue;
      st_push_ins(s, u, v, 1);
      got++;
    }
    got = 0; guard = 0;
    while (got < want_inter && guard < 1000 * (want_inter + 10)) {
      guard++;
      int32_t u = (int32_t)rbelow(&r, (uint64_t)n);
      int32_t v = (int32_t)rbelow(&r, (uint64_t)n);
      if (u == v || block[u] == block[v]) continue;
      uint64_t k = ekey(u, v);
      if (t > 0 && es_has(&prev, k)) continue;
      if (!es_add(&es, k)) continue;
      st_push_ins(s, u, v, 1);
      got++;
    }
    st_close_step(s, t);
  }
  es_free(&es);
  es_free(&prev);
  free(perm); free(boff); free(pcum); free(block);
  return s;
}

/* ---------------- LFR-style power-law temporal graph ---------------- */

/* Continuous power law p(x) ~ x^-g on [a, b] by inverse transform. */
static double powlaw(rng* r, double a, double b, double g) {
  double e = 1.0 - g, u = runif(r);
  return pow(pow(a, e) + u * (pow(b, e) - pow(a, e)), 1.0 / e);
}

/* Vose alias table over weights p[0..m). */
typedef struct { double* prob; int32_t* alias; int64_t m; } alias_t;

static void alias_build(alias_t* t, const double* p, int64_t m, int32_t* wl, int32_t* wh,
                        double* sc) {
  double sum = 0;
  for (int64_t i = 0; i < m; i++) sum += p[i];
  int64_t nl = 0, nh = 0;
  for (int64_t i = 0; i < m; i++) {
    sc[i] = p[i] * (double)m / sum;
    if (sc[i] < 1.0) wl[nl++] = (int32_t)i; else wh[nh++] = (int32_t)i;
  }
  while (nl && nh) {
    int32_t l = wl[--nl], h = wh[nh - 1];
    t->prob[l] = sc[l]; t->alias[l] = h;
    sc[h] = (sc[h] + sc[l]) - 1.0;
    if (sc[h] < 1.0) { nh--; wl[nl++] = h; }
  }
  while (nh) { int32_t h = wh[--nh]; t->prob[h] = 1.0; t->alias[h] = h; }
  while (nl) { int32_t l = wl[--nl]; t->prob[l] = 1.0; t->alias[l] = l; }
}
static inline int64_t alias_draw(rng* r, const double* prob, const int32_t* alias, int64_t m) {
  int64_t i = (int64_t)rbelow(r, (uint64_t)m);
  return runif(r) < prob[i] ? i : alias[i];
}

/* n vertices with degree propensities ~ power law (exponent g_deg on
 * [kmin, kmax]); planted communities with sizes ~ power law (exponent g_com
 * on [smin, smax]) filled to n, vertices assigned at random.  n_events edge
 * events, each with a uniform time step in 1..steps.  An event draws u with
 * probability proportional to its propensity, then v the same way inside u's
 * current planted community with probability 1 - mu, else over all vertices
 * (redrawn when v == u); every event inserts (u, v, 1), so repeats accumulate
 * weight.  At the start of every step after the first, a fraction drift of
 * the vertices moves to another planted community chosen by size, and a
 * fraction del_frac of the previous graph's distinct edges is deleted. */
dcdsyn_stream* dcdsyn_lfr(uint64_t seed, int64_t n, double g_deg, double kmin, double kmax,
                          double g_com, double smin, double smax, double mu, int64_t n_events,
                          int32_t steps, double drift, double del_frac) {
  if (n < 2 || steps < 1) return NULL;
  rng r = {seed};
  dcdsyn_stream* s = st_new(n, steps);
  double* kp = (double*)malloc((size_t)n * sizeof(double));
  for (int64_t v = 0; v < n; v++) kp[v] = powlaw(&r, kmin, kmax, g_deg);
  /* community sizes */
  int64_t ncap = 1024, nc = 0, tot = 0;
  int64_t* csz = (int64_t*)malloc((size_t)ncap * sizeof(int64_t));
  while (tot < n) {
    int64_t x = (int64_t)powlaw(&r, smin, smax, g_com);
    if (x < 1) x = 1;
    if (tot + x > n) x = n - tot;
    if (nc == ncap) { ncap *= 2; csz = (int64_t*)realloc(csz, (size_t)ncap * sizeof(int64_t)); }
    csz[nc++] = x;
    tot += x;
  }
  if (nc > 1 && csz[nc - 1] < (int64_t)smin) { csz[nc - 2] += csz[nc - 1]; nc--; }
  int32_t* comm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  for (int64_t v = 0; v < n; v++) perm[v] = (int32_t)v;
  shuffle_i32(&r, perm, n);
  {
    int64_t x = 0;
    for (int64_t c = 0; c < nc; c++)
      for (int64_t y = 0; y < csz[c]; y++) comm[perm[x++]] = (int32_t)c;
  }
  /* per-step event counts: a uniform step per event */
  int64_t* cnt = (int64_t*)calloc((size_t)steps, sizeof(int64_t));
  for (int64_t e = 0; e < n_events; e++) cnt[rbelow(&r, (uint64_t)steps)]++;

  alias_t glob = {(double*)malloc((size_t)n * sizeof(double)),
                  (int32_t*)malloc((size_t)n * sizeof(int32_t)), n};
  int32_t* wl = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* wh = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  double* sc = (double*)malloc((size_t)n * sizeof(double));
  alias_build(&glob, kp, n, wl, wh, sc);
  /* per-community alias tables over members sorted by community */
  int64_t* coff = (int64_t*)malloc((size_t)(nc + 1) * sizeof(int64_t));
  int32_t* mem = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  double* mp = (double*)malloc((size_t)n * sizeof(double));
  double* cprob = (double*)malloc((size_t)n * sizeof(double));
  int32_t* calias = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  double* sizew = (double*)malloc((size_t)nc * sizeof(double));
  alias_t ctab = {(double*)malloc((size_t)nc * sizeof(double)),
                  (int32_t*)malloc((size_t)nc * sizeof(int32_t)), nc};

  edgeset es;
  es_init(&es, n_events / 2 + 16);
  for (int32_t t = 0; t < steps; t++) {
    if (t > 0) {
      /* drift: move a fraction of the vertices to another community by size */
      int64_t* cs = (int64_t*)calloc((size_t)nc, sizeof(int64_t));
      for (int64_t v = 0; v < n; v++) cs[comm[v]]++;
      for (int64_t c = 0; c < nc; c++) sizew[c] = (double)cs[c];
      free(cs);
      alias_build(&ctab, sizew, nc, wl, wh, sc);
      for (int64_t v = 0; v < n; v++) {
        if (runif(&r) >= drift) continue;
        if (nc < 2) continue;
        for (int tries = 0; tries < 64; tries++) {
          int32_t c = (int32_t)alias_draw(&r, ctab.prob, ctab.alias, nc);
          if (c != comm[v]) { comm[v] = c; break; }
        }
      }
      /* delete a fraction of G_{t-1}'s distinct edges (Bernoulli per edge) */
      int64_t m0 = es.count;
      uint64_t* pick = (uint64_t*)malloc((size_t)(m0 > 0 ? m0 : 1) * sizeof(uint64_t));
      int64_t np = 0;
      for (int64_t x = 0; x < m0; x++)
        if (runif(&r) < del_frac) pick[np++] = es.items[x];
      for (int64_t x = 0; x < np; x++) {
        st_push_del(s, (int32_t)(pick[x] >> 32), (int32_t)(pick[x] & 0xffffffffu));
        es_remove(&es, pick[x]);
      }
      free(pick);
    }
    /* community member lists and alias tables for this step */
    for (int64_t c = 0; c <= nc; c++) coff[c] = 0;
    for (int64_t v = 0; v < n; v++) coff[comm[v] + 1]++;
    for (int64_t c = 0; c < nc; c++) coff[c + 1] += coff[c];
    {
      int64_t* fill = (int64_t*)malloc((size_t)nc * sizeof(int64_t));
      for (int64_t c = 0; c < nc; c++) fill[c] = coff[c];
      for (int64_t v = 0; v < n; v++) mem[fill[comm[v]]++] = (int32_t)v;
      free(fill);
    }
    for (int64_t x = 0; x < n; x++) mp[x] = kp[mem[x]];
    for (int64_t c = 0; c < nc; c++) {
      int64_t m = coff[c + 1] - coff[c];
      if (m <= 0) continue;
      alias_t sub = {cprob + coff[c], calias + coff[c], m};
      alias_build(&sub, mp + coff[c], m, wl, wh, sc);
    }
    for (int64_t e = 0; e < cnt[t]; e++) {
      int32_t u = (int32_t)alias_draw(&r, glob.prob, glob.alias, n);
      int32_t v = u;
      int intra = runif(&r) >= mu;
      int32_t c = comm[u];
      int64_t m = coff[c + 1] - coff[c];
      for (int tries = 0; tries < 64 && v == u; tries++) {
        if (intra && m > 1)
          v = mem[coff[c] + alias_draw(&r, cprob + coff[c], calias + coff[c], m)];
        else
          v = (int32_t)alias_draw(&r, glob.prob, glob.alias, n);
      }
      if (v == u) v = (int32_t)((u + 1) % n);
      st_push_ins(s, u, v, 1);
      es_add(&es, ekey(u, v));
    }
    st_close_step(s, t);
  }
  memcpy(s->planted, comm, (size_t)n * sizeof(int32_t));
  es_free(&es);
  free(kp); free(csz); free(comm); free(perm); free(cnt);
  free(glob.prob); free(glob.alias); free(wl); free(wh); free(sc);
  free(coff); free(mem); free(mp); free(cprob); free(calias); free(sizew);
  free(ctab.prob); free(ctab.alias);
  return s;
}

/* ---------------- R-MAT ---------------- */

/* One R-MAT sample on 2^scale vertices (Chakrabarti, Zhan & Faloutsos 2004). */
static void rmat_pair(rng* r, int32_t scale, double a, double b, double c, int32_t* u,
                      int32_t* v) {
  uint32_t x = 0, y = 0;
  for (int32_t l = 0; l < scale; l++) {
    double p = runif(r);
    x <<= 1; y <<= 1;
    if (p < a) {
    } else if (p < a + b) {
      y |= 1;
    } else if (p < a + b + c) {
      x |= 1;
    } else {
      x |= 1; y |= 1;
    }
  }
  *u = (int32_t)x; *v = (int32_t)y;
}

/* Step 1: edge_factor * 2^scale samples, weights uniform in 1..wmax, self
 * loops dropped, ids relabelled by a seeded permutation; duplicates stay in
 * the insert list (their weights add up).  Each later step first deletes
 * del_frac of the current distinct edges (uniform), then inserts ins_frac of
 * the current distinct-edge count as fresh samples. */
dcdsyn_stream* dcdsyn_rmat(uint64_t seed, int32_t scale, int64_t edge_factor, double a, double b,
                           double c, int32_t wmax, int32_t steps, double ins_frac,
                           double del_frac) {
  if (scale < 1 || scale > 30 || steps < 1) return NULL;
  rng r = {seed};
  int64_t n = (int64_t)1 << scale;
  dcdsyn_stream* s = st_new(n, steps);
  int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  for (int64_t v = 0; v < n; v++) perm[v] = (int32_t)v;
  shuffle_i32(&r, perm, n);
  int64_t m0 = edge_factor * n;
  edgeset es;
  es_init(&es, m0 + 16);
  for (int32_t t = 0; t < steps; t++) {
    int64_t want = m0;
    if (t > 0) {
      int64_t dc = (int64_t)llround(del_frac * (double)es.count);
      want = (int64_t)llround(ins_frac * (double)es.count);
      delete_uniform(&r, &es, s, dc);
    }
    for (int64_t e = 0; e < want; e++) {
      int32_t u, v;
      rmat_pair(&r, scale, a, b, c, &u, &v);
      int32_t w = 1 + (int32_t)rbelow(&r, (uint64_t)wmax);
      if (u == v) continue;
      u = perm[u]; v = perm[v];
      st_push_ins(s, u, v, w);
      es_add(&es, ekey(u, v));
    }
    st_close_step(s, t);
  }
  es_free(&es);
  free(perm);
  return s;
}

/* ---------------- batched SBM parameters ---------------- */

/* Per-graph parameters of a batch of independent temporal SBMs:
 * n_g = round(exp(U[ln nmin, ln nmax])), community sizes uniform in
 * [smin, smax] filled to n_g (a remainder below smin joins the last block),
 * mean degree uniform in [dmin, dmax].  sizes_out receives the block sizes of
 * all graphs back to back (capacity sizes_cap); nblocks_out[g] their count. */
int64_t dcdsyn_batch_params(uint64_t seed, int32_t G, double nmin, double nmax, int64_t smin,
                            int64_t smax, double dmin, double dmax, int64_t* n_out,
                            double* deg_out, int64_t* nblocks_out, int64_t* sizes_out,
                            int64_t sizes_cap) {
  rng r = {seed};
  int64_t used = 0;
  for (int32_t g = 0; g < G; g++) {
    double x = log(nmin) + runif(&r) * (log(nmax) - log(nmin));
    int64_t n = (int64_t)llround(exp(x));
    n_out[g] = n;
    deg_out[g] = dmin + runif(&r) * (dmax - dmin);
    int64_t tot = 0, nb = 0;
    while (tot < n) {
      int64_t sz = smin + (int64_t)rbelow(&r, (uint64_t)(smax - smin + 1));
      if (tot + sz > n) sz = n - tot;
      if (sz < smin && nb > 0) {
        sizes_out[used - 1] += sz;
      } else {
        if (used >= sizes_cap) return -1;
        sizes_out[used++] = sz;
        nb++;
      }
      tot += sz;
    }
    nblocks_out[g] = nb;
  }
  return used;
}
