/*
 * apex_oracle.c -- FP64 CPU oracle for APEX exhaustive enumeration.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg load this library. It shares no code, header, table or helper with the
 * CUDA path (paper_2510_24380_b300/), and the CUDA path never calls it.
 *
 * What it computes, in the paper's plain (unfactorized) order:
 *   library   D = reactions t -> R-group slots j -> synthons s          (Sec. 3.2, App. A.1)
 *   compound  chi = (t, s_1..s_n), one synthon per slot                 (Sec. 3.2 multi-index)
 *   global id off_t + mixed radix of (s_1..s_n), slot 1 most significant
 *   embedding g(chi) = sum_j u_{t,j,s_j}                                (Eq. factorizer)
 *   outputs   o = head(g): z_l = W_l a_{l-1} + b_l, a_l = act(z_l) on all but the last
 *             layer. A one-layer identity head is Eq. surrogate exactly; deeper heads are
 *             the dense heads of the benchmark workloads.
 *   objective f0 = sum_j w_j o_j, maximized                             (Eq. orig_topk)
 *   feasible  <=> lower_i <= o_{p_i} <= upper_i for every constraint i (inclusive)
 *   result    the first min(k, |feasible|) compounds under (f0 desc, id asc)
 *             (Eq. apex_topk; the lexicographic (c, f0) queue of Sec. 3.3 followed by
 *             removal of c < 0 keeps exactly this set -- a test checks that equivalence).
 * Everything is double precision; embeddings and weights are widened from float32.
 *
 * Pins (tests/test_oracle_pins.py): compound count vs the paper's worked example and vs the
 * number of compounds visited; the cost model vs the worked numbers of Sec. 3.3; identity
 * activation collapsing the head to one affine map; activation values at closed-form points;
 * a linear head reducing to Eq. apex (top-k of the X+Y sums, full sort); brute force on tiny
 * libraries; 1-slot reactions as a plain sort; permutation invariance; monotonicity in k;
 * the lexicographic-queue equivalence; id decode round trips; the associative embeddings
 * u = K_r v_s (Eq. assoc_embeds) against identity keys, basis values and linearity.
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_ACT_IDENTITY 0
#define ORC_ACT_RELU 1
#define ORC_ACT_SILU 2

typedef struct {
  int32_t n_reactions;
  const int32_t *n_slots;     /* [n_reactions] */
  const int64_t *slot_sizes;  /* [sum n_slots], reaction-major */
  int32_t d;
  const float *U;             /* [sum slot_sizes, d], rows reaction -> slot -> synthon */
  int32_t n_layers;
  const int32_t *dims;        /* [n_layers + 1], dims[0] == d */
  const float *const *W;      /* W[l]: [dims[l+1], dims[l]] row-major */
  const float *const *b;      /* b[l]: [dims[l+1]] */
  int32_t activation;
} orc_library;

typedef struct {
  int32_t n_weights;
  const double *weights;      /* objective = sum_{j < n_weights} weights[j] * o[j] */
  int32_t n_constraints;
  const int32_t *output_index;
  const double *lower;
  const double *upper;
  int64_t k;
  int32_t n_subset;           /* 0 = every reaction */
  const int32_t *subset;
} orc_query;

/* ------------------------------------------------------------------ prepared tables */
typedef struct {
  const orc_library *L;
  int64_t *slot_first;  /* [T+1] index of the first slot of reaction t */
  int64_t *row_first;   /* [S+1] first U row of slot s (flattened) */
  int64_t *id_first;    /* [T+1] first global id of reaction t */
  double **Wt;          /* Wt[l][k * dims[l+1] + i] = W[l][i][k]  (transposed, widened) */
  double **bd;
  int32_t max_width;
} prep;

static void prep_free(prep *P) {
  free(P->slot_first);
  free(P->row_first);
  free(P->id_first);
  if (P->Wt)
    for (int l = 0; l < P->L->n_layers; ++l) free(P->Wt[l]);
  if (P->bd)
    for (int l = 0; l < P->L->n_layers; ++l) free(P->bd[l]);
  free(P->Wt);
  free(P->bd);
}

/* number of compounds of reaction t: product of its slot sizes (App. A.1); -1 on overflow */
static int64_t reaction_count(const orc_library *L, const int64_t *slot_first, int t) {
  __int128 n = 1;
  for (int64_t s = slot_first[t]; s < slot_first[t + 1]; ++s) {
    n *= L->slot_sizes[s];
    if (n > (__int128)INT64_MAX) return -1;
  }
  return (int64_t)n;
}

static int prep_init(prep *P, const orc_library *L, int with_weights) {
  memset(P, 0, sizeof(*P));
  P->L = L;
  int T = L->n_reactions;
  if (T < 1) return -1;
  P->slot_first = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
  P->id_first = (int64_t *)calloc((size_t)T + 1, sizeof(int64_t));
  if (!P->slot_first || !P->id_first) return -1;
  for (int t = 0; t < T; ++t) {
    if (L->n_slots[t] < 1 || L->n_slots[t] > 64) return -1;
    P->slot_first[t + 1] = P->slot_first[t] + L->n_slots[t];
  }
  int64_t S = P->slot_first[T];
  P->row_first = (int64_t *)calloc((size_t)S + 1, sizeof(int64_t));
  if (!P->row_first) return -1;
  for (int64_t s = 0; s < S; ++s) {
    if (L->slot_sizes[s] < 1) return -1;
    P->row_first[s + 1] = P->row_first[s] + L->slot_sizes[s];
  }
  for (int t = 0; t < T; ++t) {
    int64_t n = reaction_count(L, P->slot_first, t);
    if (n < 0 || P->id_first[t] > INT64_MAX - n) return -1;
    P->id_first[t + 1] = P->id_first[t] + n;
  }
  if (!with_weights) return 0;
  if (L->n_layers < 1 || L->dims[0] != L->d) return -1;
  P->Wt = (double **)calloc((size_t)L->n_layers, sizeof(double *));
  P->bd = (double **)calloc((size_t)L->n_layers, sizeof(double *));
  if (!P->Wt || !P->bd) return -1;
  P->max_width = L->d;
  for (int l = 0; l < L->n_layers; ++l) {
    int in = L->dims[l], out = L->dims[l + 1];
    if (in < 1 || out < 1) return -1;
    if (out > P->max_width) P->max_width = out;
    P->Wt[l] = (double *)malloc(sizeof(double) * (size_t)in * out);
    P->bd[l] = (double *)malloc(sizeof(double) * (size_t)out);
    if (!P->Wt[l] || !P->bd[l]) return -1;
    for (int i = 0; i < out; ++i) {
      P->bd[l][i] = (double)L->b[l][i];
      for (int k = 0; k < in; ++k) P->Wt[l][(size_t)k * out + i] = (double)L->W[l][(size_t)i * in + k];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ head (FP64) */
static double act(int a, double z) {
  if (a == ORC_ACT_RELU) return z > 0.0 ? z : 0.0;
  if (a == ORC_ACT_SILU) return z / (1.0 + exp(-z)); /* SiLU(z) = z * sigmoid(z) */
  return z;
}

/* o = head(g); buf0/buf1 hold max_width doubles each */
static void head_eval(const prep *P, const double *g, double *buf0, double *buf1, double *o) {
  const orc_library *L = P->L;
  const double *x = g;
  for (int l = 0; l < L->n_layers; ++l) {
    int in = L->dims[l], out = L->dims[l + 1];
    double *y = (l == L->n_layers - 1) ? o : ((l % 2 == 0) ? buf0 : buf1);
    const double *Wt = P->Wt[l];
    for (int i = 0; i < out; ++i) y[i] = P->bd[l][i];
    for (int k = 0; k < in; ++k) { /* y_i += W_ik x_k, k in increasing order for every i */
      const double xk = x[k];
      const double *col = Wt + (size_t)k * out;
      for (int i = 0; i < out; ++i) y[i] += col[i] * xk;
    }
    if (l < L->n_layers - 1)
      for (int i = 0; i < out; ++i) y[i] = act(L->activation, y[i]);
    x = y;
  }
}

/* g = sum_j u_{t,j,s_j} in slot order (Eq. factorizer) */
static void embed(const prep *P, int t, const int64_t *s, double *g) {
  const orc_library *L = P->L;
  int d = L->d;
  for (int c = 0; c < d; ++c) g[c] = 0.0;
  for (int64_t j = 0; j < L->n_slots[t]; ++j) {
    int64_t row = P->row_first[P->slot_first[t] + j] + s[j];
    const float *u = L->U + (size_t)row * d;
    for (int c = 0; c < d; ++c) g[c] += (double)u[c];
  }
}

/* global id -> (t, s_1..s_n); slot 1 is the most significant digit */
static int decode(const prep *P, int64_t id, int *t_out, int64_t *s) {
  const orc_library *L = P->L;
  int T = L->n_reactions;
  if (id < 0 || id >= P->id_first[T]) return -1;
  int lo = 0, hi = T - 1;
  while (lo < hi) { /* last t with id_first[t] <= id */
    int mid = (lo + hi + 1) / 2;
    if (P->id_first[mid] <= id) lo = mid; else hi = mid - 1;
  }
  int t = lo;
  int64_t rem = id - P->id_first[t];
  int n = L->n_slots[t];
  for (int j = n - 1; j >= 0; --j) {
    int64_t nj = L->slot_sizes[P->slot_first[t] + j];
    s[j] = rem % nj;
    rem /= nj;
  }
  *t_out = t;
  return 0;
}

/* ------------------------------------------------------------------ public: shape */
int64_t orc_count(const orc_library *L) {
  prep P;
  int64_t n = -1;
  if (prep_init(&P, L, 0) == 0) n = P.id_first[L->n_reactions];
  prep_free(&P);
  return n;
}

/* Linear-probe cost model of Sec. 3.3: caching |S| d-float32 embeddings costs |S|*d*4 bytes;
 * one task's contributions v_{r,s} = w^T u_{r,s} cost (2d - 1) flops each, 2|S|d - |S| in all;
 * a compound of an n-slot reaction then costs n flops (n - 1 additions and the bias). */
int orc_linear_cost(int32_t n_reactions, const int32_t *n_slots, const int64_t *slot_sizes, int32_t d,
                    double *cache_bytes, double *precompute_flops, double *total_flops, int64_t *n_compounds) {
  orc_library L;
  memset(&L, 0, sizeof(L));
  L.n_reactions = n_reactions;
  L.n_slots = n_slots;
  L.slot_sizes = slot_sizes;
  L.d = d;
  prep P;
  if (prep_init(&P, &L, 0) != 0) { prep_free(&P); return -1; }
  double S = 0.0, flops = 0.0;
  for (int64_t s = 0; s < P.slot_first[n_reactions]; ++s) S += (double)slot_sizes[s];
  for (int t = 0; t < n_reactions; ++t)
    flops += (double)(P.id_first[t + 1] - P.id_first[t]) * (double)n_slots[t];
  *cache_bytes = S * (double)d * 4.0;
  *precompute_flops = 2.0 * S * (double)d - S;
  *total_flops = flops;
  *n_compounds = P.id_first[n_reactions];
  prep_free(&P);
  return 0;
}

/* Associative embeddings of Eq. assoc_embeds: u_{r,s} = K_r v_s for every synthon row of every
 * R-group slot r (slots in library order, rows slot-major). K: [n_slots_total x d x d_u], each
 * K_r row-major (d rows of d_u); V: [rows x d_u]; U: [rows x d]. Every product is formed in
 * double precision, K and V widened from float32, summed over the d_u terms in order. */
int orc_assoc(int64_t n_slots_total, const int64_t *slot_sizes, int32_t d, int32_t d_u, const float *K,
              const float *V, double *U) {
  if (n_slots_total < 0 || d < 1 || d_u < 1) return -1;
  int64_t row = 0;
  for (int64_t r = 0; r < n_slots_total; ++r) {
    const float *Kr = K + (size_t)r * d * d_u;
    for (int64_t s = 0; s < slot_sizes[r]; ++s, ++row) {
      const float *v = V + (size_t)row * d_u;
      for (int32_t i = 0; i < d; ++i) {
        double acc = 0.0;
        for (int32_t j = 0; j < d_u; ++j) acc += (double)Kr[(size_t)i * d_u + j] * (double)v[j];
        U[(size_t)row * d + i] = acc;
      }
    }
  }
  return 0;
}

int orc_decode(const orc_library *L, int64_t n, const int64_t *ids, int32_t *t_out, int64_t *s_out,
               int32_t max_slots) {
  prep P;
  if (prep_init(&P, L, 0) != 0) { prep_free(&P); return -1; }
  int rc = 0;
  int64_t s[64];
  for (int64_t i = 0; i < n && rc == 0; ++i) {
    int t;
    if (decode(&P, ids[i], &t, s) != 0) { rc = -2; break; }
    if (L->n_slots[t] > max_slots) { rc = -3; break; }
    t_out[i] = t;
    for (int j = 0; j < max_slots; ++j) s_out[i * max_slots + j] = j < L->n_slots[t] ? s[j] : -1;
  }
  prep_free(&P);
  return rc;
}

/* ------------------------------------------------------------------ public: head */
int orc_head(const orc_library *L, int64_t n, const double *g, double *out) {
  prep P;
  if (prep_init(&P, L, 1) != 0) { prep_free(&P); return -1; }
  double *b0 = (double *)malloc(sizeof(double) * P.max_width);
  double *b1 = (double *)malloc(sizeof(double) * P.max_width);
  int nout = L->dims[L->n_layers];
  for (int64_t i = 0; i < n; ++i) head_eval(&P, g + (size_t)i * L->d, b0, b1, out + (size_t)i * nout);
  free(b0);
  free(b1);
  prep_free(&P);
  return 0;
}

/* ------------------------------------------------------------------ threads */
typedef struct {
  const prep *P;
  const int64_t *ids;
  double *out;
  int64_t n;
  atomic_llong *next;
  int rc;
} score_job;

static void *score_worker(void *arg) {
  score_job *J = (score_job *)arg;
  const orc_library *L = J->P->L;
  int nout = L->dims[L->n_layers];
  double *g = (double *)malloc(sizeof(double) * L->d);
  double *b0 = (double *)malloc(sizeof(double) * J->P->max_width);
  double *b1 = (double *)malloc(sizeof(double) * J->P->max_width);
  int64_t s[64];
  for (;;) {
    int64_t i0 = atomic_fetch_add(J->next, 256);
    if (i0 >= J->n) break;
    int64_t i1 = i0 + 256 < J->n ? i0 + 256 : J->n;
    for (int64_t i = i0; i < i1; ++i) {
      int t;
      if (decode(J->P, J->ids[i], &t, s) != 0) { J->rc = -2; continue; }
      embed(J->P, t, s, g);
      head_eval(J->P, g, b0, b1, J->out + (size_t)i * nout);
    }
  }
  free(g);
  free(b0);
  free(b1);
  return NULL;
}

static int resolve_threads(int32_t n_threads) {
  if (n_threads > 0) return n_threads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

int orc_score_ids(const orc_library *L, int64_t n, const int64_t *ids, double *out, int32_t n_threads) {
  prep P;
  if (prep_init(&P, L, 1) != 0) { prep_free(&P); return -1; }
  int nt = resolve_threads(n_threads);
  atomic_llong next = 0;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
  score_job *jobs = (score_job *)calloc((size_t)nt, sizeof(score_job));
  for (int i = 0; i < nt; ++i) {
    jobs[i] = (score_job){&P, ids, out, n, &next, 0};
    pthread_create(&th[i], NULL, score_worker, &jobs[i]);
  }
  int rc = 0;
  for (int i = 0; i < nt; ++i) {
    pthread_join(th[i], NULL);
    if (jobs[i].rc) rc = jobs[i].rc;
  }
  free(th);
  free(jobs);
  prep_free(&P);
  return rc;
}

/* ------------------------------------------------------------------ top-k */
typedef struct {
  double f;
  int64_t id;
} entry;

/* a ranks before b: higher objective first, then smaller global id */
static int better(const entry *a, const entry *b) { return a->f > b->f || (a->f == b->f && a->id < b->id); }

/* bounded heap whose root is the entry every other entry ranks before */
typedef struct {
  entry *e;
  int64_t n, cap;
} heap;

static void heap_push(heap *H, entry x) {
  if (H->cap == 0) return;
  if (H->n < H->cap) {
    int64_t i = H->n++;
    while (i > 0) {
      int64_t p = (i - 1) / 2;
      if (!better(&H->e[p], &x)) break; /* parent already ranks after x: x stays below it */
      H->e[i] = H->e[p];
      i = p;
    }
    H->e[i] = x;
    return;
  }
  if (!better(&x, &H->e[0])) return;
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, w = i;
    const entry *cur = &x;
    if (l < H->n && better(cur, &H->e[l])) { w = l; cur = &H->e[l]; }
    if (r < H->n && better(cur, &H->e[r])) { w = r; }
    if (w == i) break;
    H->e[i] = H->e[w];
    i = w;
  }
  H->e[i] = x;
}

typedef struct {
  const prep *P;
  const orc_query *Q;
  const int32_t *rx;         /* reactions to enumerate */
  const int64_t *task_first; /* [n_rx+1] prefix of first-slot sizes */
  int32_t n_rx;
  atomic_llong *next;
  heap H;
  int64_t n_feasible, n_enumerated;
} topk_job;

static void *topk_worker(void *arg) {
  topk_job *J = (topk_job *)arg;
  const prep *P = J->P;
  const orc_library *L = P->L;
  const orc_query *Q = J->Q;
  int nout = L->dims[L->n_layers];
  double *g = (double *)malloc(sizeof(double) * L->d);
  double *b0 = (double *)malloc(sizeof(double) * P->max_width);
  double *b1 = (double *)malloc(sizeof(double) * P->max_width);
  double *o = (double *)malloc(sizeof(double) * nout);
  int64_t s[64], strides[64];
  int64_t total = J->task_first[J->n_rx];
  for (;;) {
    int64_t task = atomic_fetch_add(J->next, 1);
    if (task >= total) break;
    int lo = 0, hi = J->n_rx - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) / 2;
      if (J->task_first[mid] <= task) lo = mid; else hi = mid - 1;
    }
    int t = J->rx[lo];
    int n = L->n_slots[t];
    const int64_t *sz = L->slot_sizes + P->slot_first[t];
    strides[n - 1] = 1;
    for (int j = n - 2; j >= 0; --j) strides[j] = strides[j + 1] * sz[j + 1];
    s[0] = task - J->task_first[lo];
    for (int j = 1; j < n; ++j) s[j] = 0;
    for (;;) { /* odometer over slots 2..n with slot 1 fixed */
      int64_t id = P->id_first[t];
      for (int j = 0; j < n; ++j) id += s[j] * strides[j];
      embed(P, t, s, g);
      head_eval(P, g, b0, b1, o);
      J->n_enumerated++;
      int ok = 1;
      for (int i = 0; i < Q->n_constraints; ++i) {
        double v = o[Q->output_index[i]];
        if (!(v >= Q->lower[i] && v <= Q->upper[i])) { ok = 0; break; }
      }
      if (ok) {
        double f = 0.0;
        for (int j = 0; j < Q->n_weights; ++j) f += Q->weights[j] * o[j];
        J->n_feasible++;
        heap_push(&J->H, (entry){f, id});
      }
      int j = n - 1;
      while (j >= 1) {
        if (++s[j] < sz[j]) break;
        s[j] = 0;
        --j;
      }
      if (j < 1) break;
    }
  }
  free(g);
  free(b0);
  free(b1);
  free(o);
  return NULL;
}

static int cmp_entry(const void *a, const void *b) {
  const entry *x = (const entry *)a, *y = (const entry *)b;
  if (better(x, y)) return -1;
  if (better(y, x)) return 1;
  return 0;
}

/* Exhaustive top-k (Eq. apex_topk). ids/scores: [k]; outputs: [k * n_outputs] (may be NULL). */
int orc_topk(const orc_library *L, const orc_query *Q, int32_t n_threads, int64_t *ids, double *scores,
             double *outputs, int64_t *n_out, int64_t *n_feasible, int64_t *n_enumerated) {
  prep P;
  if (prep_init(&P, L, 1) != 0) { prep_free(&P); return -1; }
  int nout = L->dims[L->n_layers];
  if (Q->k < 1 || Q->n_weights > nout) { prep_free(&P); return -1; }
  for (int i = 0; i < Q->n_constraints; ++i)
    if (Q->output_index[i] < 0 || Q->output_index[i] >= nout) { prep_free(&P); return -1; }
  int32_t n_rx = Q->n_subset > 0 ? Q->n_subset : L->n_reactions;
  int32_t *rx = (int32_t *)malloc(sizeof(int32_t) * n_rx);
  int64_t *task_first = (int64_t *)calloc((size_t)n_rx + 1, sizeof(int64_t));
  for (int r = 0; r < n_rx; ++r) {
    rx[r] = Q->n_subset > 0 ? Q->subset[r] : r;
    if (rx[r] < 0 || rx[r] >= L->n_reactions) { free(rx); free(task_first); prep_free(&P); return -1; }
    task_first[r + 1] = task_first[r] + L->slot_sizes[P.slot_first[rx[r]]];
  }
  int nt = resolve_threads(n_threads);
  atomic_llong next = 0;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
  topk_job *jobs = (topk_job *)calloc((size_t)nt, sizeof(topk_job));
  for (int i = 0; i < nt; ++i) {
    jobs[i].P = &P;
    jobs[i].Q = Q;
    jobs[i].rx = rx;
    jobs[i].task_first = task_first;
    jobs[i].n_rx = n_rx;
    jobs[i].next = &next;
    jobs[i].H.cap = Q->k;
    jobs[i].H.e = (entry *)malloc(sizeof(entry) * (size_t)Q->k);
    pthread_create(&th[i], NULL, topk_worker, &jobs[i]);
  }
  int64_t all = 0, feas = 0, en = 0;
  for (int i = 0; i < nt; ++i) {
    pthread_join(th[i], NULL);
    all += jobs[i].H.n;
    feas += jobs[i].n_feasible;
    en += jobs[i].n_enumerated;
  }
  entry *merged = (entry *)malloc(sizeof(entry) * (size_t)(all > 0 ? all : 1));
  int64_t m = 0;
  for (int i = 0; i < nt; ++i) {
    memcpy(merged + m, jobs[i].H.e, sizeof(entry) * (size_t)jobs[i].H.n);
    m += jobs[i].H.n;
    free(jobs[i].H.e);
  }
  qsort(merged, (size_t)m, sizeof(entry), cmp_entry);
  int64_t kk = m < Q->k ? m : Q->k;
  for (int64_t i = 0; i < kk; ++i) {
    ids[i] = merged[i].id;
    scores[i] = merged[i].f;
  }
  *n_out = kk;
  if (n_feasible) *n_feasible = feas;
  if (n_enumerated) *n_enumerated = en;
  int rc = 0;
  free(merged);
  free(th);
  free(jobs);
  free(rx);
  free(task_first);
  prep_free(&P);
  if (outputs && kk > 0) rc = orc_score_ids(L, kk, ids, outputs, n_threads);
  return rc;
}
