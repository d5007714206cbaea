/*
 * dcd_oracle.h -- plain sequential CPU oracle for incremental dynamic
 * community detection with Delta-screening (Zarayeneh & Kalyanaraman,
 * "A Fast and Efficient Incremental Approach toward Dynamic Community
 * Detection", arXiv 1904.08553).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg link it.
 * It shares no code with the CUDA library.
 *
 * Every floating-point-free decision is taken on exact integers:
 *   m2   = 2m = sum of weighted degrees                      (Sec. III-A)
 *   N    = m2 * in - sum_C a_C^2,   Q = N / m2^2             (Eq. 1)
 *   S    = m2 (e_{v,D} - e_{v,C\v}) - k_v (a_D - (a_C - k_v))  (gain, Sec. III-A;
 *          the paper's Delta Q_{v->D} equals S / m2^2)
 * Weights are int64 throughout the oracle; products use 128-bit integers.
 */
#ifndef DCD_ORACLE_H
#define DCD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_STATIC = 0, ORC_BASE = 1, ORC_DELTA = 2, ORC_GIVEN_R = 3 };
enum { ORC_LOUVAIN = 0, ORC_SLM = 1 }; /* the host method of the multi-level run */

enum {
  ORC_OK = 0,
  ORC_EINVAL = -1,
  ORC_ENOMEM = -2,
  ORC_EOVERFLOW = -5
};

#define ORC_MAX_ITERS 500
#define ORC_MAX_LEVELS 64
#define ORC_TAU_INV 1000000 /* relative gain threshold 1e-6 */

typedef struct orc_graph orc_graph;
typedef struct orc_ctx orc_ctx;

typedef struct {
  int64_t t;              /* time step just computed (1-based)            */
  int64_t n;              /* |V_t|                                        */
  int64_t nnz;            /* directed CSR entries of G_t                  */
  int64_t m2;             /* 2 m_t                                        */
  int64_t r_size;         /* |R_t| (vertices active at level 0)           */
  int64_t levels;         /* levels run                                   */
  int64_t iters_total;    /* local-move passes over all levels            */
  int64_t iters_level0;   /* local-move passes at level 0                 */
  int64_t moves_total;    /* applied single-vertex moves                  */
  int64_t edges_scanned;  /* sum over passes of sum of active degrees     */
  int64_t communities;    /* |C_t|                                        */
  int64_t n_lo, n_hi;     /* N as a 128-bit integer (two's complement)    */
  double q;               /* modularity Q_t                               */
  int64_t refine_iters;   /* SLM: refinement passes over all levels       */
  int64_t refine_moves;   /* SLM: moves applied by the refinements        */
} orc_stats;

/* ---- graphs (CSR: int64 row_ptr[n+1], int32 col[nnz] sorted, int64 w) ---- */
orc_graph* orc_graph_new(int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const int64_t* w);
void orc_graph_free(orc_graph* g);
int64_t orc_graph_n(const orc_graph* g);
int64_t orc_graph_nnz(const orc_graph* g);
void orc_graph_copy(const orc_graph* g, int64_t* row_ptr, int32_t* col, int64_t* w);

/* G_t = G_{t-1} with deletes applied first, then inserts adding weight.
 * ins is n_ins triples (u,v,w); del is n_del pairs (u,v).  del_present
 * (may be NULL) receives 1 for each delete whose edge existed in g. */
orc_graph* orc_apply(const orc_graph* g, const int32_t* ins, int64_t n_ins,
                     const int32_t* del, int64_t n_del, uint8_t* del_present,
                     int* err);

/* Modularity of a partition (labels in [0,n)): returns Q, writes m2 and N. */
double orc_modularity(const orc_graph* g, const int32_t* labels, int64_t* m2,
                      int64_t* n_lo, int64_t* n_hi);

/* Gain S(v -> D) under labels (0 when D == labels[v]); 128-bit result. */
void orc_gain(const orc_graph* g, const int32_t* labels, int32_t v, int32_t D,
              int64_t* s_lo, int64_t* s_hi);

/* One synchronous local-move pass: proposals for active vertices (active may
 * be NULL = all).  out[v] = new label.  Returns the number of movers. */
int64_t orc_local_move_pass(const orc_graph* g, const int32_t* labels,
                            const uint8_t* active, int32_t* out);

/* One level of local-move passes to convergence; labels updated in place.
 * Returns the number of passes. */
int64_t orc_run_level(const orc_graph* g, int32_t* labels, const uint8_t* active,
                      int64_t max_iters, int64_t* moves, int64_t* edges);

/* Graph compaction: coarse vertex of fine vertex v is cid_of_v[v]. */
orc_graph* orc_coarsen(const orc_graph* g, const int32_t* labels, int32_t* cid_of_v);

/* Delta-screening (Algorithm 2 for inserts, plus the deletion rule):
 * g_prev = G_{t-1}, g_t = G_t, labels0 = C_{t-1}.  r_out[v] in {0,1}. */
int orc_screen(const orc_graph* g_prev, const orc_graph* g_t, const int32_t* labels0,
               const int32_t* ins, int64_t n_ins, const int32_t* del, int64_t n_del,
               uint8_t* r_out);

/* Multi-level Louvain (Algorithm 1) from level-0 labels init and level-0
 * active set (NULL = all).  out = canonical labels (min member id). */
int orc_louvain(const orc_graph* g, const int32_t* init, const uint8_t* active,
                int32_t* out, orc_stats* st);

/* Smart local moving, the paper's second host method (dSLM-Delta-s), with the
 * readings stated in dcd_oracle.c.  orc_slm: multi-level SLM from init with
 * the level-0 active set (NULL = all); out = canonical labels.
 * orc_slm_refine: the refinement of one level (sub-communities of each
 * parent community, canonical).  orc_slm_level: SLM local moving of one level
 * (labels made canonical first, updated in place).  Both return passes. */
int orc_slm(const orc_graph* g, const int32_t* init, const uint8_t* active, int32_t* out,
            orc_stats* st);
int64_t orc_slm_refine(const orc_graph* g, const int32_t* parent, int32_t* sub, int64_t* moves);
int64_t orc_slm_level(const orc_graph* g, int32_t* labels, const uint8_t* active, int64_t* moves);

/* Learned-screen pool and features (not in the paper): see dcd_oracle.c. */
int orc_screen_features(const orc_graph* g_prev, const orc_graph* g_t, const int32_t* labels, const int32_t* ins,
                        int64_t n_ins, const int32_t* del, int64_t n_del, const uint8_t* rds, uint8_t* pool_out,
                        float* X);

/* ---- stateful incremental driver (Sec. III-D) ---- */
orc_ctx* orc_create(int64_t n);
void orc_destroy(orc_ctx* c);
int orc_apply_batch(orc_ctx* c, const int32_t* ins, int64_t n_ins, const int32_t* del,
                    int64_t n_del);
/* mode: ORC_STATIC, ORC_BASE, ORC_DELTA, ORC_GIVEN_R (r_given used as R_t).
 * The first update of a context is always static (step 1 of Sec. III-D). */
int orc_update(orc_ctx* c, int mode, const uint8_t* r_given, int32_t* labels_out,
               double* q_out, orc_stats* st);
/* As orc_update with the host method alg (ORC_LOUVAIN or ORC_SLM). */
int orc_update_alg(orc_ctx* c, int alg, int mode, const uint8_t* r_given, int32_t* labels_out,
                   double* q_out, orc_stats* st);
int orc_get_rset(const orc_ctx* c, uint8_t* r_out);
const orc_graph* orc_ctx_graph(const orc_ctx* c);
int orc_set_labels(orc_ctx* c, const int32_t* labels);
/* Deep copy of a context (G_t, C_t, R_t, t, staged batch): test and timing
 * infrastructure, no arithmetic. */
orc_ctx* orc_clone(const orc_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
