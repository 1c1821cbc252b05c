// apex_lib.cu -- host side of the C ABI (include/apex.h).
//
//   load:   validate -> upload U and the head -> P32 = W_1 U^T (+ b_1 on slot-1 rows) ->
//           BF16 tables and tensor-core weight images -> per-reaction work plans ->
//           calibration of the pass margins -> worker thread.
//   query:  apex_query queues a request; the worker admits it into one of APEX_MAX_ACTIVE slots
//           when its candidate state fits the memory budget, estimates a starting threshold from
//           a seeded FP32 sample of its scope, and serves it from the shared circular pass over
//           the library (continuous batching: one enumeration launch serves every active query
//           whose reactions it covers). When a query has seen all its items once, it is
//           finalized: exact selection (FP32 rescore of the candidates, FP64 rescore of the
//           boundary band and of near-ties), ordering by (objective desc, id asc), decode.
#include <algorithm>
#include <climits>
#include <atomic>
#include <cstdarg>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <pthread.h>
#include <random>
#include <sched.h>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

// ------------------------------------------------------------------ kernels (other files)
cudaError_t apx_launch_fp32(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, const long long *ids,
                            long long n_ids, float *out, int grid, cudaStream_t st, int id_tile = 32,
                            const unsigned *n_dev = nullptr);
cudaError_t apx_launch_fp64(const DevTables &T, const long long *ids, long long n, double *out, cudaStream_t st,
                            const unsigned *n_dev = nullptr);
cudaError_t apx_launch_prep(const float *U, const float *W1, const float *b1, const unsigned char *bias_row,
                            long long rows, int K, int N, float *P32, cudaStream_t st);
cudaError_t apx_launch_p16(const float *P32, long long n, float scale, int fmt, void *P16, cudaStream_t st);
cudaError_t apx_launch_image(const float *W, int rows_used, int rows, int fmt, void *img, cudaStream_t st);
cudaError_t apx_launch_slot_extremes(const float *P, const long long *row_first, int n_slots, int N, float *mx,
                                     float *mn, cudaStream_t st);
cudaError_t apx_launch_image_e4m3(const float *W, const float *scale, int rows_used, int rows, void *img,
                                  cudaStream_t st);
cudaError_t apx_launch_tc_ids(const DevTables &T, const long long *ids, long long n, float *out, int *err, int n_sm,
                              cudaStream_t st, int fmt, QuerySlot *slots, int spec_slot, const unsigned *n_dev = nullptr);
cudaError_t apx_launch_tc(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int *err, int grid,
                          cudaStream_t st, int fmt);
cudaError_t apx_launch_slot_select(QuerySlot *slots, const int *slot_list, int n_slots, int mode, cudaStream_t st);
cudaError_t apx_launch_eval32(const EvalArgs &a, long long n, float *f32, unsigned char *maybe, unsigned char *sure,
                              cudaStream_t st, const unsigned *n_dev = nullptr);
cudaError_t apx_launch_kth(const float *keys, const unsigned char *flag, long long n, long long k, float *out_tau,
                           int *out_ok, cudaStream_t st, const unsigned *n_dev = nullptr);
cudaError_t apx_launch_kth_multi(const KthJob *jobs, int n_jobs, cudaStream_t st);
cudaError_t apx_launch_build_r(long long n, const long long *cand_ids, const float *f32, const unsigned char *maybe,
                               const unsigned char *sure, const float *tau32, float margin2, RItem *R, unsigned *n_r,
                               cudaStream_t st, const unsigned *n_dev = nullptr);
cudaError_t apx_launch_collect64(RItem *R, unsigned n, long long *ids64, int *pos64, unsigned *n64, cudaStream_t st);
cudaError_t apx_launch_split_scored(const QuerySlot *Q, unsigned n_max, float *f32, unsigned char *maybe,
                                    unsigned char *sure, long long *ids_new, int *pos_new, unsigned *n_new, int n_sm,
                                    cudaStream_t st);
cudaError_t apx_launch_compact(QuerySlot *Q, const float *f32, const unsigned char *maybe, const unsigned char *sure,
                               const float *tau32, const int *ok, float margin2, float eps_f, unsigned *kept,
                               unsigned n_max, int n_sm, cudaStream_t st);
cudaError_t apx_launch_apply64(RItem *R, const int *pos64, const double *out64, unsigned n64, const unsigned *n64_dev,
                               int n_out, const QuerySlot *Q, const double *lo, const double *hi, double *out_rows,
                               cudaStream_t st, const float *out32 = nullptr, unsigned *obs = nullptr);
cudaError_t apx_sort_r(RItem *R, unsigned n_used, unsigned n_pow2, cudaStream_t st, const unsigned *n_dev = nullptr);
cudaError_t apx_launch_mark(RItem *R, unsigned n, unsigned kp1, long long k, double tol, unsigned *n_marked,
                            cudaStream_t st, const unsigned *n_used);
cudaError_t apx_launch_pad_r_dev(RItem *R, const unsigned *n_used, unsigned to, cudaStream_t st);
cudaError_t apx_launch_emit(const RItem *R, unsigned n_final, const unsigned *n_alive, const DevTables &T,
                            const float *out32, const double *out64_rows, long long *ids, int *rxn, long long *syn,
                            double *obj, double *outs, cudaStream_t st);
cudaError_t apx_launch_count_alive(const RItem *R, unsigned n, unsigned *d_out, cudaStream_t st);
cudaError_t apx_launch_mark_near(RItem *R, unsigned n, const float *ref, double tol, unsigned *n_marked,
                                 cudaStream_t st);
cudaError_t apx_launch_wait_selftest(int *err, unsigned long long limit_ns, cudaStream_t st);
cudaError_t apx_launch_linear(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int n_sm, cudaStream_t st);
cudaError_t apx_launch_assoc(const void *blocks, int n_blocks, int d, int d_u, const float *K, const float *V, float *U,
                             cudaStream_t st);
int apx_assoc_blocks(long long n_slots_total, const int64_t *slot_sizes, void *out, int capacity);
size_t apx_assoc_block_bytes();
cudaError_t apx_launch_spec_ids(const int *rxn, const long long *pre, int n_sub, const long long *id_first,
                                long long scope_n, unsigned long long seed, long long S, long long *ids, cudaStream_t st);
cudaError_t apx_launch_spec_select(const float *out, long long S, const SpecArgs &a, float *keys, unsigned char *flag,
                                   QuerySlot *slot, cudaStream_t st);

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;
static apex_status fail(apex_status code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static apex_status fail(apex_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
apex_status apx_fail(apex_status code, const char *msg) {
  g_err = msg;
  return code;
}
#define CU(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) throw CudaFail(e_, #call, __LINE__);                                     \
  } while (0)
struct CudaFail {
  cudaError_t e;
  const char *what;
  int line;
  CudaFail(cudaError_t e_, const char *w, int l) : e(e_), what(w), line(l) {}
};
struct BudgetFail {};

static std::atomic<long long> g_launches{0};
void apx_count_launch(long long n) { g_launches += n; }

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static inline void cpu_relax() {
#if defined(__x86_64__) || defined(__i386__)
  __builtin_ia32_pause();
#endif
}
// Watches an atomic counter until it moves away from seq (true) or limit_ms pass (false). The CPU
// is offered to other threads every yield_mask + 1 checks.
static bool watch(const std::atomic<unsigned long long> &c, unsigned long long seq, double limit_ms, int yield_mask) {
  const double t0 = now_ms();
  for (int i = 0;; ++i) {
    if (c.load(std::memory_order_acquire) != seq) return true;
    if ((i & yield_mask) == yield_mask) {
      if (now_ms() - t0 >= limit_ms) return false;
      sched_yield();
    }
    cpu_relax();
  }
}
// Takes the lock right after a watched counter moved: the thread that moved it still holds the
// lock for a moment, and a blocking lock would put this thread to sleep (its wake-up then costs
// the other thread a wake call and this one tens of microseconds), so it tries for a while first.
static void lock_spin(std::unique_lock<std::mutex> &lk) {
  for (int i = 0; i < 20000; ++i) {
    if (lk.try_lock()) return;
    cpu_relax();
  }
  lk.lock();
}
static double env_ms(const char *name, double dflt) {
  const char *e = getenv(name);
  return e ? std::max(0.0, atof(e)) : dflt;
}
// How long the idle worker watches for work before it sleeps (APEX_WORKER_SPIN_MS, default 3) and
// how long a fetcher watches for completions before it sleeps (APEX_FETCH_SPIN_MS, default 20).
static double worker_spin_ms() {
  static const double v = env_ms("APEX_WORKER_SPIN_MS", 3.0);
  return v;
}
static double fetch_spin_ms() {
  static const double v = env_ms("APEX_FETCH_SPIN_MS", 20.0);
  return v;
}

// ------------------------------------------------------------------ query record
enum QState { Q_QUEUED, Q_ACTIVE, Q_DONE, Q_CANCELED, Q_FAILED };

struct QueryRec {
  apex_query_id id;
  int precision;
  std::vector<float> w;
  std::vector<int> cidx;
  std::vector<double> lo, hi;
  long long k;
  std::vector<int> subset;          // sorted reaction indices
  std::vector<char> need;           // [n_rx]
  long long scope_items = 0, remaining = 0, scope_n = 0;
  QState state = Q_QUEUED;
  int slot = -1;
  apex_status err = APEX_OK;
  std::string err_msg;
  bool cancel = false;
  double t_submit = 0, t_admit = 0, t_done = 0;
  // device state
  unsigned cap = 0;
  float *keys = nullptr, *keys2 = nullptr;
  long long *ids = nullptr, *ids2 = nullptr;
  size_t dev_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool started = false;
  int spec_rank = 0;                // rank used for the speculative start threshold (0 = none)
  float tau_spec = -INFINITY;
  // factors on the library's pass and FP32 margins for this query (raised when the runtime check at
  // finalization observed a larger error than a margin allows)
  double mscale = 1.0;
  // in-pass compaction of the candidate buffer wanted before the next launch (set when a
  // retired launch showed the buffer above the trigger)
  bool want_compact = false;
  // candidate count after the select of the last retired launch of the current pass (0: none yet)
  unsigned seen_count = 0;
  // results
  std::vector<long long> r_ids;
  std::vector<int> r_rxn;
  std::vector<long long> r_syn;
  std::vector<double> r_obj, r_out;
  apex_query_stats_t stats{};
};

// ------------------------------------------------------------------ library
struct apex_library {
  // tunables (apex_autotune): compounds per enumeration launch of the circular pass, rows per CTA
  // tile of the FP32 kernel over id lists (start-threshold sample, candidate rescore)
  std::atomic<long long> chunk_compounds{1LL << 25};
  std::atomic<int> fp32_id_tile{32};
  // shape
  int T = 0, d = 0, n_layers = 0, act = 0, n_obj = 0, n_prop = 0, n_out = 0, max_slots = 0;
  int dims[8] = {0};
  std::vector<int> n_slots;
  std::vector<long long> slot_sizes, slot_first, row_first, id_first;
  long long N = 0, rows = 0;
  uint32_t precisions = 1u;
  bool tc_fmt[3] = {false, false, false};  // tensor-core tables built: [0] BF16, [1] FP16, [2] FP8
  // device
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int n_sm = 148;
  std::vector<void *> allocs;
  size_t bytes = 0, budget = 0, query_bytes = 0;
  DevTables T_{};
  std::vector<RxnPlan> rx;
  long long total_items = 0;
  std::vector<long long> item_first;  // [T+1] prefix of items
  QuerySlot *d_slots = nullptr;
  int *d_err = nullptr;
  int *d_slot_list = nullptr;
  // start-threshold sample of whole-library queries: drawn once (uniform, seeded) and kept
  long long *d_spec_full = nullptr;
  long long spec_full_n = 0;
  std::vector<std::vector<float>> hW, hb;  // host copies of the head (for apex_save_library)
  uint32_t precisions_requested = 1u;
  // calibration
  // admission margins: err16[0] BF16 pass, [1] FP16 pass, [2] FP8 pass; err32 FP32 pass / rescore
  double err16[3][APEX_MAX_OUTPUTS] = {{0}}, err32[APEX_MAX_OUTPUTS] = {0}, rms[APEX_MAX_OUTPUTS] = {0};
  int n_calib = 0;
  double a1_amax = 0;         // FP8: exact max |a_1| over the library (its static activation scale)
  float *d_err32f = nullptr;  // per-output FP32 margin (float) for eval32
  float *d_err16f = nullptr;  // per-output FP16 pass margin (float): FP16 in-pass compactions
  uint64_t seed = 0;
  // engine
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  bool stop = false;
  std::deque<QueryRec *> queued;
  std::map<apex_query_id, std::unique_ptr<QueryRec>> queries;
  QueryRec *active[APEX_MAX_ACTIVE] = {nullptr};
  std::atomic<long long> next_id{1};
  // Wake-ups without a sleep on the short path: the idle worker watches work_seq (bumped under mu
  // with every submission, cancellation and shutdown) for a few milliseconds before it sleeps on
  // cv, and up to two fetchers watch done_seq (bumped under mu when a query finishes) before they
  // sleep on cv_done. A thread woken from a sleep starts tens of microseconds later.
  std::atomic<unsigned long long> work_seq{0}, done_seq{0};
  int spinners = 0;  // fetchers watching done_seq (under mu)
  std::atomic<int> worker_cpu{-2};  // CPU the worker is pinned to, -1 none, -2 not chosen yet
  // timing event pairs of finished queries, reused by the next ones (under mu): creating and
  // destroying two events per query were four CUDA calls on the query's path
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  std::atomic<long long> fin_cover_set{0};  // candidates a queued finalization covers (0: default)
  long long cursor = 0;  // global item index of the circular pass
  apex_query_stats_t last_stats{};
  // serving statistics over fetched queries (apex_stats; under mu). head_evals counts compounds
  // scored by enumeration launches (worker thread), snapshotted at every reset.
  struct Served {
    std::vector<double> lat, queue;  // ring of the last APEX_STATS_WINDOW queries
    size_t next = 0;
    long long n_ok = 0, n_failed = 0;
    double t_first = 0, t_last = 0, query_compounds = 0, lat_sum = 0, lat_max = 0;
    long long evals_at_reset = 0, enum_ns_at_reset = 0, launches_at_reset = 0;
  } served;
  std::atomic<long long> head_evals{0};
  std::atomic<long long> enum_ns{0}, enum_launches{0};  // device time and count of enumeration launches
  std::mt19937_64 rng;
  // reusable device scratch: per-slot candidate buffers (grow-only) and a bump arena for
  // finalization / sampling temporaries (grow-only), pinned host staging, events
  struct SlotBuf {
    float *keys = nullptr, *keys2 = nullptr;
    long long *ids = nullptr, *ids2 = nullptr;
    unsigned cap = 0;
  } slotbuf[APEX_MAX_ACTIVE];
  char *arena = nullptr;
  size_t arena_cap = 0, arena_off = 0;
  size_t dev_total = 0;  // device memory (cudaMemGetInfo at load)
  char *pinned = nullptr;
  size_t pinned_cap = 0;
  // Pinned upload ring: every small host-to-device copy of the worker (slot parameters, slot
  // lists, sample scope, boxes) is staged in its own region, so a copy still queued behind a
  // running launch never sees a later overwrite; the ring wraps only after a stream sync.
  char *up = nullptr;
  size_t up_cap = 0, up_off = 0;
  // Pinned download area of one batch of finalizations (results land here; each query of the
  // batch owns its region until the host has taken its rows).
  char *dl = nullptr;
  size_t dl_cap = 0, dl_off = 0;
  // Enumeration launches whose completion the worker has not observed yet. The worker keeps at
  // most one launch queued behind the running one (it plans launch i + 1 while launch i runs) and
  // reads each launch's kernel status word and duration from a pinned copy when it retires.
  static constexpr int kRing = 4;
  struct InFlight {
    int ring;
    std::vector<std::pair<int, long long>> queries;  // (slot, query id) served by the launch
  };
  cudaEvent_t ev_l0[kRing] = {}, ev_l1[kRing] = {}, ev_ls[kRing] = {};
  int *status_pin = nullptr;
  // claim counter of the enumeration kernel's tail pool (zeroed before every launch that uses it)
  unsigned long long *d_pool_ctr = nullptr;
  bool pool_off = false;  // APEX_NO_TILE_POOL set: CTA ranges only
  // per ring entry: (count, count_compacted) of every slot after the launch's select and
  // compactions (pinned), read when the launch retires to decide the next compactions
  unsigned *cnt_pin = nullptr;
  // per slot: observed errors of the running query (EvalArgs::obs: [0] max |pass key - FP32
  // objective| over every candidate rescored in the pass or at its end, [1 + p] max |FP32 - FP64|
  // of output p), zeroed whenever the slot's parameters are written
  unsigned *d_obs_slots = nullptr;
  cudaEvent_t ev_tr[8] = {};  // GPU timeline marks of a query's phases (APEX_TRACE only)
  std::deque<InFlight> inflight;
  long long launch_seq = 0;

  void *dalloc(size_t n, bool count = true) {
    if (count && budget && bytes + query_bytes + n > budget) throw BudgetFail();
    void *p = nullptr;
    CU(cudaMalloc(&p, n ? n : 16));
    allocs.push_back(p);
    if (count) bytes += n;
    return p;
  }
  void release_all() {
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
  }
  ~apex_library() {}

  // bump allocation from the arena; grow() must be called (with no work in flight) first
  void *aget(size_t n) {
    n = (n + 255) & ~(size_t)255;
    if (arena_off + n > arena_cap) throw CudaFail(cudaErrorMemoryAllocation, "arena exhausted", __LINE__);
    void *p = arena + arena_off;
    arena_off += n;
    return p;
  }
  void arena_reserve(size_t n) {
    arena_off = 0;
    if (n <= arena_cap) return;
    CU(cudaStreamSynchronize(st));
    if (arena) cudaFree(arena);
    arena = nullptr;
    size_t want = std::max(n + (n >> 1), (size_t)(8u << 20));
    if (budget && bytes + query_bytes + want > budget + arena_cap) want = n;
    CU(cudaMalloc(&arena, want));
    query_bytes += want - arena_cap;
    arena_cap = want;
  }
  void upload(void *dst, const void *src, size_t n) {
    if (n == 0) return;
    const size_t a = (n + 63) & ~(size_t)63;
    if (a > up_cap) {
      CU(cudaStreamSynchronize(st));
      if (up) cudaFreeHost(up);
      up = nullptr;
      up_cap = std::max(a, (size_t)(1u << 20));
      CU(cudaMallocHost(&up, up_cap));
      up_off = 0;
    } else if (up_off + a > up_cap) {
      CU(cudaStreamSynchronize(st));
      up_off = 0;
    }
    memcpy(up + up_off, src, n);
    CU(cudaMemcpyAsync(dst, up + up_off, n, cudaMemcpyHostToDevice, st));
    up_off += a;
  }
  void dl_reserve(size_t n) {
    dl_off = 0;
    if (n <= dl_cap) return;
    CU(cudaStreamSynchronize(st));
    if (dl) cudaFreeHost(dl);
    dl = nullptr;
    dl_cap = std::max(n + (n >> 1), (size_t)(1u << 20));
    CU(cudaMallocHost(&dl, dl_cap));
  }
  void *dl_get(size_t n) {
    n = (n + 63) & ~(size_t)63;
    if (dl_off + n > dl_cap) throw CudaFail(cudaErrorMemoryAllocation, "download area exhausted", __LINE__);
    void *p = dl + dl_off;
    dl_off += n;
    return p;
  }
  void *pin(size_t n) {
    if (n > pinned_cap) {
      if (pinned) cudaFreeHost(pinned);
      pinned = nullptr;
      pinned_cap = std::max(n, (size_t)(1u << 20));
      CU(cudaMallocHost(&pinned, pinned_cap));
    }
    return pinned;
  }
};

// ------------------------------------------------------------------ helpers
static bool mul_ok(long long a, long long b, long long *out) {
  if (a <= 0 || b <= 0) return false;
  if (a > (long long)(INT64_MAX / b)) return false;
  *out = a * b;
  return true;
}

extern "C" apex_status apex_count_compounds(int32_t n_reactions, const int32_t *n_slots, const int64_t *slot_sizes,
                                            int64_t *n_out) {
  if (!n_slots || !slot_sizes || !n_out || n_reactions < 1) return fail(APEX_EINVAL, "bad arguments");
  long long total = 0, s = 0;
  for (int t = 0; t < n_reactions; ++t) {
    if (n_slots[t] < 1) return fail(APEX_EINVAL, "reaction %d has %d slots", t, n_slots[t]);
    long long n = 1;
    for (int j = 0; j < n_slots[t]; ++j, ++s) {
      if (slot_sizes[s] < 1) return fail(APEX_EINVAL, "slot %lld has size %lld", s, (long long)slot_sizes[s]);
      if (!mul_ok(n, slot_sizes[s], &n)) return fail(APEX_EINVAL, "reaction %d overflows int64", t);
    }
    if (total > INT64_MAX - n) return fail(APEX_EINVAL, "library size overflows int64");
    total += n;
  }
  *n_out = total;
  return APEX_OK;
}

// Inner/outer split of reaction t (see common.cuh). The outer slot is slot 1 unless the
// reaction has 2 slots and using slot 2 as the outer slot wastes fewer padded tile rows.
static RxnPlan plan_reaction(const apex_library &L, int t, long long target_tiles_per_item) {
  RxnPlan p{};
  const int n = L.n_slots[t];
  const long long *sz = &L.slot_sizes[L.slot_first[t]];
  const long long *rf = &L.row_first[L.slot_first[t]];
  p.id_first = L.id_first[t];
  p.n_slots = n;
  for (int j = 0; j < n; ++j) {
    p.slot_row[j] = rf[j];
    p.slot_size[j] = sz[j];
  }
  auto waste = [](long long m) { return (double)((m + APX_TILE - 1) / APX_TILE * APX_TILE) / (double)m; };
  if (n == 1) {
    p.n_inner = sz[0];
    p.n_outer = 1;
    p.inner_stride = 1;
    p.outer_stride = 0;
    p.outer_row = -1;
    p.n_inner_slots = 1;
    p.inner_row[0] = rf[0];
    p.inner_size[0] = sz[0];
  } else if (n == 2 && waste(sz[0]) < waste(sz[1])) {
    // inner = slot 1 (stride |slot 2|), outer = slot 2 (stride 1)
    p.n_inner = sz[0];
    p.n_outer = sz[1];
    p.inner_stride = sz[1];
    p.outer_stride = 1;
    p.outer_row = rf[1];
    p.n_inner_slots = 1;
    p.inner_row[0] = rf[0];
    p.inner_size[0] = sz[0];
  } else {
    // outer = slot 1, inner = slots 2..n flattened (mixed radix, slot 2 most significant)
    long long ni = 1;
    for (int j = 1; j < n; ++j) ni *= sz[j];
    p.n_inner = ni;
    p.n_outer = sz[0];
    p.inner_stride = 1;
    p.outer_stride = ni;
    p.outer_row = rf[0];
    p.n_inner_slots = n - 1;
    for (int j = 1; j < n; ++j) {
      p.inner_row[j - 1] = rf[j];
      p.inner_size[j - 1] = sz[j];
    }
  }
  p.n_b = (int)((p.n_inner + APX_TILE - 1) / APX_TILE);
  p.L_o = (int)std::max<long long>(1, std::min<long long>(p.n_outer, target_tiles_per_item));
  p.n_oc = (int)((p.n_outer + p.L_o - 1) / p.L_o);
  p.n_items = (long long)p.n_b * p.n_oc;
  return p;
}

// Compounds in items [ib, ie) of a reaction: 128 per tile, except in the tiles of the last inner
// block, which hold n_inner - 128 (n_b - 1) rows each.
static long long items_compounds(const RxnPlan &r, long long ib, long long ie) {
  const long long t0 = apx_tiles_before(r, ib), t1 = apx_tiles_before(r, ie);
  const long long last0 = (long long)(r.n_b - 1) * r.n_outer;  // first tile of the last inner block
  const long long last_rows = r.n_inner - (long long)(r.n_b - 1) * APX_TILE;
  const long long in_last = std::max(0LL, t1 - std::max(t0, last0));
  return (t1 - t0) * APX_TILE - in_last * (APX_TILE - last_rows);
}

static DevTables upload_plans(apex_library &L) {
  RxnPlan *d_rx = (RxnPlan *)L.dalloc(sizeof(RxnPlan) * L.rx.size());
  CU(cudaMemcpy(d_rx, L.rx.data(), sizeof(RxnPlan) * L.rx.size(), cudaMemcpyHostToDevice));
  long long *d_idf = (long long *)L.dalloc(sizeof(long long) * (L.T + 1));
  CU(cudaMemcpy(d_idf, L.id_first.data(), sizeof(long long) * (L.T + 1), cudaMemcpyHostToDevice));
  DevTables T = L.T_;
  T.rx = d_rx;
  T.id_first = d_idf;
  return T;
}

// Builds a launch over [first item, ...) of the given reactions' items (a "chunk").
struct PlanBuilder {
  LaunchPlan P;
  const std::vector<RxnPlan> *rx;
  explicit PlanBuilder(const std::vector<RxnPlan> &r) : rx(&r) { memset(&P, 0, sizeof(P)); }
  bool add(int rxn, long long b, long long e, unsigned long long qmask) {
    if (P.n_seg >= APX_MAX_SEG || e <= b) return false;
    Segment &s = P.seg[P.n_seg];
    s.rxn = rxn;
    s.item_begin = b;
    s.item_end = e;
    s.qmask = qmask;
    P.qmask_all |= qmask;
    P.seg_first[P.n_seg + 1] = P.seg_first[P.n_seg] + (e - b);
    const RxnPlan &p = (*rx)[rxn];
    P.seg_tile_first[P.n_seg + 1] = P.seg_tile_first[P.n_seg] + apx_tiles_before(p, e) - apx_tiles_before(p, b);
    P.n_seg++;
    P.total_items = P.seg_first[P.n_seg];
    P.total_tiles = P.seg_tile_first[P.n_seg];
    return true;
  }
};

static int grid_for(const apex_library &L, long long items) {
  return (int)std::max<long long>(1, std::min<long long>(items, L.n_sm));
}

// tensor-core operand format of a query precision: 0 = BF16, 1 = FP16, 2 = FP8 e4m3, -1 = none
static inline int tc_format(int precision) {
  return precision == APEX_BF16 ? 0 : precision == APEX_FP16 ? 1 : precision == APEX_FP8 ? 2 : -1;
}

// admission margin of a pass precision (per output)
static inline const double *pass_err(const apex_library &L, int precision) {
  const int f = tc_format(precision);
  return f >= 0 ? L.err16[f] : L.err32;
}

// Launch tile ranges of equal estimated cost for the CTAs of the tensor-core kernel. A tile costs 1
// and every run of tiles (consecutive tiles of one inner block: the kernel gathers the block's
// inner rows again at its start and its pipeline refills) costs kRunCost more, about 2.4 tiles as
// measured per CTA on B300 (a reaction whose outer slot has 19 synthons ran ~10 % slower per tile
// than one with long runs, and equal tile counts left its CTAs last). Every CTA gets >= 1 tile.
//
// Tail pool: with 8 queries in a launch the cost of a tile also depends on how many of its compounds
// pass some query's objective threshold (those warps take the box tests and the candidate append),
// which differs between reactions: on c3_slice the slowest CTA ran 17 % above the mean. So for query
// launches of more than two queries and at least kPoolMinPerCta tiles per CTA the ranges cover the
// first (1 - kPoolFrac) of the tiles, and CTAs that finish their range take the rest kPoolChunk
// tiles at a time (each chunk starts a new run for the CTA: the pool costs about 2.4 / kPoolChunk of
// its tiles). With one or two queries the cost-weighted ranges alone end within a few percent of
// each other, and the pool's extra run starts cost more than it balances (c2_10m single query:
// 1.63 ms per launch with the pool, 1.55 ms without).
static constexpr double kPoolFrac = 0.2;
static constexpr int kPoolChunk = 48;
static constexpr long long kPoolMinPerCta = 512;
static void tc_partition(const apex_library &L, LaunchPlan &P, int grid, unsigned long long *pool_ctr) {
  P.cta_n = 0;
  P.pool_ctr = nullptr;
  P.pool_first = P.total_tiles;
  P.pool_chunk = 0;
  if (grid < 2 || grid > APX_MAX_CTA || P.total_tiles < grid) return;
  long long n_static = P.total_tiles;  // tiles covered by the CTA ranges
  if (pool_ctr && P.mode == 0 && __builtin_popcountll(P.qmask_all) > 2 && P.total_tiles >= kPoolMinPerCta * grid) {
    n_static = P.total_tiles - (long long)(kPoolFrac * (double)P.total_tiles);
    P.pool_ctr = pool_ctr;
    P.pool_first = n_static;
    P.pool_chunk = kPoolChunk;
  }
  constexpr double kRunCost = 2.4;
  std::vector<std::pair<long long, long long>> runs;  // (first launch tile, tiles), below n_static
  for (int g = 0; g < P.n_seg; ++g) {
    const Segment &sg = P.seg[g];
    const RxnPlan &p = L.rx[sg.rxn];
    const long long x0 = apx_tiles_before(p, sg.item_begin), x1 = apx_tiles_before(p, sg.item_end);
    for (long long x = x0; x < x1;) {
      const long long e = std::min(x1, (x / p.n_outer + 1) * p.n_outer);
      const long long first = P.seg_tile_first[g] + (x - x0);
      if (first >= n_static) break;
      runs.emplace_back(first, std::min(e - x, n_static - first));
      x = e;
    }
  }
  double total = 0;
  for (const auto &r : runs) total += kRunCost + (double)r.second;
  const double per = total / grid;
  P.cta_first[0] = 0;
  int c = 1;
  double cum = 0;
  for (const auto &r : runs) {
    while (c < grid && (double)c * per <= cum + kRunCost + (double)r.second) {
      const double into = std::max(0.0, (double)c * per - cum - kRunCost);  // tiles into the run
      long long t = r.first + std::min(r.second, (long long)std::ceil(into));
      t = std::max(t, P.cta_first[c - 1] + 1);
      t = std::min(t, n_static - (grid - c));
      P.cta_first[c++] = t;
    }
    cum += kRunCost + (double)r.second;
  }
  for (; c < grid; ++c) P.cta_first[c] = std::min(n_static - (grid - c), P.cta_first[c - 1] + 1);
  P.cta_first[grid] = n_static;
  P.cta_n = grid;
}

static void launch_enum(apex_library &L, const LaunchPlan &P, int precision) {
  if (P.total_items == 0) return;
  const int fmt = tc_format(precision);
  if (fmt >= 0) {  // CTAs take tile ranges of equal estimated cost
    const int grid = grid_for(L, P.total_tiles);
    LaunchPlan Q = P;
    tc_partition(L, Q, grid, L.pool_off ? nullptr : L.d_pool_ctr);
    if (Q.pool_ctr) CU(cudaMemsetAsync(Q.pool_ctr, 0, sizeof(unsigned long long), L.st));
    CU(apx_launch_tc(Q, L.T_, L.d_slots, L.d_err, grid, L.st, fmt));
  } else if (L.n_layers == 1 && P.mode == 0) {  // linear head: per-synthon scalar sums (Eq. apex)
    CU(apx_launch_linear(P, L.T_, L.d_slots, L.n_sm, L.st));
  } else {
    CU(apx_launch_fp32(P, L.T_, L.d_slots, nullptr, 0, nullptr, grid_for(L, P.total_items), L.st));
  }
}

static void check_kernel_status(apex_library &L) {
  int *pe = (int *)L.pin(64) + 8;
  CU(cudaMemcpyAsync(pe, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, L.st));
  CU(cudaStreamSynchronize(L.st));
  const int e = *pe;
  if (e) {
    int z = 0;
    CU(cudaMemcpy(L.d_err, &z, sizeof(int), cudaMemcpyHostToDevice));
    throw CudaFail(cudaErrorLaunchTimeout, "device-side bounded wait expired", e);
  }
}

static bool trace_on() {
  static int on = -1;
  if (on < 0) on = getenv("APEX_TRACE") ? 1 : 0;
  return on == 1;
}
#define TRACE(...)                          \
  do {                                      \
    if (trace_on()) {                       \
      fprintf(stderr, "[apex] " __VA_ARGS__); \
      fputc('\n', stderr);                 \
    }                                       \
  } while (0)

// GPU timeline mark i of the current query (APEX_TRACE only)
static void tmark(apex_library &L, int i) {
  if (L.ev_tr[i]) CU(cudaEventRecord(L.ev_tr[i], L.st));
}
static float tspan(apex_library &L, cudaEvent_t a, cudaEvent_t b) {
  float ms = -1.f;
  if (a && b && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) ms = -1.f;
  return ms;
}

static unsigned fin_cover_base(const apex_library &L, const QueryRec *q);

// Candidate count above which a query's buffer is compacted in FP32 before the next launch: about
// what its end-of-pass finalization covers in one queued chain (so that chain rarely needs its exact
// rerun), at least 2k, at least twice what the last compaction kept (a query with few surely
// feasible candidates cannot shrink its buffer much: no compaction every launch), and at most half
// the buffer (two launches are queued before the compaction runs).
static unsigned compact_trigger(const apex_library &L, const QueryRec *q, unsigned last_kept) {
  const long long base = std::max<long long>(std::min<long long>(q->cap / 4, fin_cover_base(L, q) / 2), 2 * q->k);
  return (unsigned)std::min<long long>(std::max<long long>(base, 2LL * last_kept), q->cap / 2);
}

// Retires the oldest enumeration launch in flight: waits for its status copy, raises a device-side
// wait timeout as an error, adds the launch's duration to the queries it served, and marks for an
// in-pass compaction the queries whose candidate buffer it left above their trigger.
static void retire_launch(apex_library &L) {
  apex_library::InFlight f = std::move(L.inflight.front());
  L.inflight.pop_front();
  CU(cudaEventSynchronize(L.ev_ls[f.ring]));
  if (L.status_pin[f.ring]) {
    L.inflight.clear();
    int z = 0;
    CU(cudaStreamSynchronize(L.st));
    CU(cudaMemcpy(L.d_err, &z, sizeof(int), cudaMemcpyHostToDevice));
    throw CudaFail(cudaErrorLaunchTimeout, "device-side bounded wait expired", L.status_pin[f.ring]);
  }
  float ms = 0;
  CU(cudaEventElapsedTime(&ms, L.ev_l0[f.ring], L.ev_l1[f.ring]));
  L.enum_ns += (long long)(1e6 * (double)ms);
  L.enum_launches++;
  const unsigned *cnt = L.cnt_pin + (size_t)f.ring * 2 * APEX_MAX_ACTIVE;
  for (const auto &sq : f.queries) {
    QueryRec *q = L.active[sq.first];
    if (q && q->id == sq.second) {
      q->stats.enumerate_ms += ms;
      const unsigned c = cnt[2 * sq.first], kept = cnt[2 * sq.first + 1];
      q->seen_count = c;
      if (q->remaining > 0 && !q->want_compact && c > compact_trigger(L, q, kept)) q->want_compact = true;
    }
  }
  TRACE("launch %d queries: %.3f ms", (int)f.queries.size(), (double)ms);
}
static void retire_all(apex_library &L) {
  while (!L.inflight.empty()) retire_launch(L);
}
// Idle worker: launches of queries that are gone; only a stale timeout status is cleared.
static void retire_quietly(apex_library &L) {
  if (L.inflight.empty()) return;
  cudaStreamSynchronize(L.st);
  bool stale = false;
  for (const auto &f : L.inflight) {
    stale = stale || L.status_pin[f.ring] != 0;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, L.ev_l0[f.ring], L.ev_l1[f.ring]) == cudaSuccess) {
      L.enum_ns += (long long)(1e6 * (double)ms);
      L.enum_launches++;
    }
  }
  L.inflight.clear();
  if (stale) {
    int z = 0;
    cudaMemcpy(L.d_err, &z, sizeof(int), cudaMemcpyHostToDevice);
  }
}

// device temporaries released when the scope ends
struct DevBuf {
  std::vector<void *> p;
  void *get(size_t n) {
    void *x = nullptr;
    CU(cudaMalloc(&x, n ? n : 16));
    p.push_back(x);
    return x;
  }
  ~DevBuf() {
    for (void *x : p) cudaFree(x);
  }
};

// ------------------------------------------------------------------ calibration
// Margins of the reduced-precision pass and of the FP32 rescore, measured on a seeded sample:
// the BF16 production kernel and the FP32 kernel score the same work items (dump mode); the
// FP32 gather kernel and the FP64 kernel score the same sampled ids. margin = factor * max
// |difference| + a floor relative to the output RMS. The sample bounds the error empirically;
// there is no closed-form bound through bf16 rounding and tanh.approx.
static void upload_err32(apex_library &L) {
  L.d_err32f = (float *)L.dalloc(sizeof(float) * APEX_MAX_OUTPUTS);
  float e32[APEX_MAX_OUTPUTS] = {0};
  for (int p = 0; p < L.n_out; ++p) e32[p] = (float)L.err32[p];
  CU(cudaMemcpy(L.d_err32f, e32, sizeof(e32), cudaMemcpyHostToDevice));
  bool have16 = L.tc_fmt[1];  // FP16 margins calibrated (a library file of a BF16-only library saved
  for (int p = 0; p < L.n_out; ++p) have16 = have16 && L.err16[1][p] > 0;  // before may lack them)
  if (have16) {  // rounded up: the FP32 test of an FP16 rescore must not be tighter than its margin
    L.d_err16f = (float *)L.dalloc(sizeof(float) * APEX_MAX_OUTPUTS);
    float e16[APEX_MAX_OUTPUTS] = {0};
    for (int p = 0; p < L.n_out; ++p) e16[p] = std::nextafter((float)L.err16[1][p], INFINITY);
    CU(cudaMemcpy(L.d_err16f, e16, sizeof(e16), cudaMemcpyHostToDevice));
  }
}

// Margins saved with a library file (apex_save_library), restored instead of recalibrating.
struct SavedCal {
  int32_t n_calib;
  double err32[APEX_MAX_OUTPUTS], err16[3][APEX_MAX_OUTPUTS], rms[APEX_MAX_OUTPUTS];
};

static void calibrate(apex_library &L) {
  const int no = L.n_out;
  std::mt19937_64 g(L.seed ^ 0x9e3779b97f4a7c15ull);
  // FP32 vs FP64 on sampled ids
  const long long ns = std::min<long long>(L.N, 4096);
  std::vector<long long> ids(ns);
  for (long long i = 0; i < ns; ++i) ids[i] = (long long)(g() % (unsigned long long)L.N);
  long long *d_ids = (long long *)L.dalloc(sizeof(long long) * ns, false);
  float *d_o32 = (float *)L.dalloc(sizeof(float) * ns * no, false);
  double *d_o64 = (double *)L.dalloc(sizeof(double) * ns * no, false);
  CU(cudaMemcpyAsync(d_ids, ids.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, L.st));
  LaunchPlan dummy;
  memset(&dummy, 0, sizeof(dummy));
  CU(apx_launch_fp32(dummy, L.T_, nullptr, d_ids, ns, d_o32, grid_for(L, (ns + APX_TILE - 1) / APX_TILE), L.st));
  CU(apx_launch_fp64(L.T_, d_ids, ns, d_o64, L.st));
  std::vector<float> o32(ns * no);
  std::vector<double> o64(ns * no);
  CU(cudaMemcpyAsync(o32.data(), d_o32, sizeof(float) * ns * no, cudaMemcpyDeviceToHost, L.st));
  CU(cudaMemcpyAsync(o64.data(), d_o64, sizeof(double) * ns * no, cudaMemcpyDeviceToHost, L.st));
  CU(cudaStreamSynchronize(L.st));
  for (int p = 0; p < no; ++p) {
    double m = 0, ss = 0;
    for (long long i = 0; i < ns; ++i) {
      m = std::max(m, std::fabs((double)o32[i * no + p] - o64[i * no + p]));
      ss += o64[i * no + p] * o64[i * no + p];
    }
    L.rms[p] = std::sqrt(ss / (double)ns);
    L.err32[p] = 8.0 * m + 1e-6 * L.rms[p] + 1e-9;
  }
  L.n_calib = (int)ns;
  if (L.tc_fmt[0] || L.tc_fmt[1] || L.tc_fmt[2]) {
    // tensor-core pass vs FP32 on whole work items: one item, chosen at random, of every reaction
    // (of kCalRx reactions chosen at random when the library has more), in launches of up to
    // kCalBatch items. Random items rather than each reaction's first one: the first item always
    // pairs the first inner rows with the first outer synthons.
    constexpr int kCalRx = 1024, kCalBatch = 128;
    std::vector<int> order(L.T);
    for (int t = 0; t < L.T; ++t) order[t] = t;
    std::shuffle(order.begin(), order.end(), g);
    const int n_rx = std::min(L.T, kCalRx);
    double mx[3][APEX_MAX_OUTPUTS] = {{0}};
    long long cnt[3] = {0, 0, 0};
    for (int b0 = 0; b0 < n_rx; b0 += kCalBatch) {
      PlanBuilder pb(L.rx);
      for (int i = b0; i < std::min(n_rx, b0 + kCalBatch); ++i) {
        const int t = order[i];
        const long long item = (long long)(g() % (unsigned long long)L.rx[t].n_items);
        pb.add(t, item, item + 1, 0);
      }
      const long long slots = pb.P.total_tiles * APX_TILE;
      DevBuf B;  // temporaries of this batch (freed when it is done)
      float *d16 = (float *)B.get(sizeof(float) * slots * no);
      float *d32 = (float *)B.get(sizeof(float) * slots * no);
      long long *di16 = (long long *)B.get(sizeof(long long) * slots);
      long long *di32 = (long long *)B.get(sizeof(long long) * slots);
      LaunchPlan P = pb.P;
      P.mode = 2;
      P.dump_n = slots;
      P.dump = d32;
      P.dump_ids = di32;
      CU(cudaMemsetAsync(di32, 0xff, sizeof(long long) * slots, L.st));
      CU(apx_launch_fp32(P, L.T_, nullptr, nullptr, 0, nullptr, grid_for(L, P.total_items), L.st));
      std::vector<float> a(slots * no), b(slots * no);
      std::vector<long long> ia(slots), ib(slots);
      CU(cudaMemcpyAsync(b.data(), d32, sizeof(float) * slots * no, cudaMemcpyDeviceToHost, L.st));
      CU(cudaMemcpyAsync(ib.data(), di32, sizeof(long long) * slots, cudaMemcpyDeviceToHost, L.st));
      CU(cudaStreamSynchronize(L.st));
      for (int f = 0; f < 3; ++f) {
        if (!L.tc_fmt[f]) continue;
        P.dump = d16;
        P.dump_ids = di16;
        CU(cudaMemsetAsync(di16, 0xff, sizeof(long long) * slots, L.st));
        CU(apx_launch_tc(P, L.T_, nullptr, L.d_err, grid_for(L, P.total_tiles), L.st, f));
        check_kernel_status(L);
        CU(cudaMemcpyAsync(a.data(), d16, sizeof(float) * slots * no, cudaMemcpyDeviceToHost, L.st));
        CU(cudaMemcpyAsync(ia.data(), di16, sizeof(long long) * slots, cudaMemcpyDeviceToHost, L.st));
        CU(cudaStreamSynchronize(L.st));
        for (long long i = 0; i < slots; ++i) {
          if (ia[i] < 0 || ia[i] != ib[i]) continue;
          ++cnt[f];
          for (int p = 0; p < no; ++p)
            mx[f][p] = std::max(mx[f][p], std::fabs((double)a[i * no + p] - (double)b[i * no + p]));
        }
      }
    }
    long long cnt_max = 0;
    for (int f = 0; f < 3; ++f) {
      if (!L.tc_fmt[f]) continue;
      for (int p = 0; p < no; ++p) L.err16[f][p] = 4.0 * mx[f][p] + 1e-3 * L.rms[p] + L.err32[p];
      cnt_max = std::max(cnt_max, cnt[f]);
    }
    L.n_calib += (int)cnt_max;
  }
  upload_err32(L);
}

// ------------------------------------------------------------------ load
static void worker_main(apex_library *L);

static apex_status load_impl(const apex_library_desc *D, const SavedCal *cal, apex_library **out);

extern "C" apex_status apex_load_library(const apex_library_desc *D, apex_library **out) {
  return load_impl(D, nullptr, out);
}

static apex_status load_impl(const apex_library_desc *D, const SavedCal *cal, apex_library **out) {
  if (!out) return fail(APEX_EINVAL, "out is NULL");
  *out = nullptr;
  if (!D) return fail(APEX_EINVAL, "desc is NULL");
  if (D->n_reactions < 1 || !D->n_slots || !D->slot_sizes) return fail(APEX_EINVAL, "no reactions");
  if (D->d < 1 || D->d > 1024) return fail(APEX_EINVAL, "d = %d outside 1..1024", D->d);
  if (!D->U) return fail(APEX_EINVAL, "U is NULL");
  if (D->n_layers < 1 || D->n_layers > 7 || !D->dims || !D->W || !D->b)
    return fail(APEX_EINVAL, "n_layers must be 1..7 with dims, W and b");
  if (D->dims[0] != D->d) return fail(APEX_EINVAL, "dims[0] (%d) != d (%d)", D->dims[0], D->d);
  for (int l = 1; l <= D->n_layers; ++l) {
    const int lim = (l == D->n_layers) ? APEX_MAX_OUTPUTS : 256;
    if (D->dims[l] < 1 || D->dims[l] > lim) return fail(APEX_EINVAL, "dims[%d] = %d outside 1..%d", l, D->dims[l], lim);
  }
  for (int l = 0; l < D->n_layers; ++l)
    if (!D->W[l] || !D->b[l]) return fail(APEX_EINVAL, "W[%d] or b[%d] is NULL", l, l);
  if (D->activation < 0 || D->activation > 2) return fail(APEX_EINVAL, "unknown activation %d", D->activation);
  if (D->n_objectives < 1 || D->n_objectives > APEX_MAX_OBJECTIVES || D->n_properties < 0 ||
      D->n_objectives + D->n_properties != D->dims[D->n_layers])
    return fail(APEX_EINVAL, "n_objectives + n_properties must equal the output width");
  int64_t N = 0;
  apex_status s = apex_count_compounds(D->n_reactions, D->n_slots, D->slot_sizes, &N);
  if (s != APEX_OK) return s;
  if (N >= (1LL << 61)) return fail(APEX_EINVAL, "library too large (ids must stay below 2^61)");
  for (int t = 0; t < D->n_reactions; ++t)
    if (D->n_slots[t] > APEX_MAX_SLOTS) return fail(APEX_EUNSUPPORTED, "reaction %d has more than %d slots", t, APEX_MAX_SLOTS);
  if (D->precisions & ~((1u << APEX_FP32) | (1u << APEX_BF16) | (1u << APEX_FP16) | (1u << APEX_FP8)))
    return fail(APEX_EINVAL, "precisions: only the FP32, BF16, FP16 and FP8 bits are defined");
  const bool want_bf16 = (D->precisions >> APEX_BF16) & 1u;
  const bool want_fp8 = (D->precisions >> APEX_FP8) & 1u;
  // the FP8 pass reads the FP16 table; BF16 and FP8 passes rescore their candidates in FP16 between
  // launches (in-pass compactions)
  const bool want_fp16 = ((D->precisions >> APEX_FP16) & 1u) || want_fp8 || want_bf16;
  const bool tc_shape = D->n_layers == 3 && D->dims[1] == 256 && D->dims[2] == 256 && D->dims[3] <= 16;
  if ((want_bf16 || want_fp16) && !tc_shape)
    return fail(APEX_EUNSUPPORTED, "the tensor-core path needs a d -> 256 -> 256 -> <=16 head");

  std::unique_ptr<apex_library> L(new apex_library());
  L->T = D->n_reactions;
  L->d = D->d;
  L->n_layers = D->n_layers;
  for (int l = 0; l <= D->n_layers; ++l) L->dims[l] = D->dims[l];
  L->act = D->activation;
  L->n_obj = D->n_objectives;
  L->n_prop = D->n_properties;
  L->n_out = D->dims[D->n_layers];
  L->N = N;
  L->n_slots.assign(D->n_slots, D->n_slots + L->T);
  L->slot_first.assign(L->T + 1, 0);
  for (int t = 0; t < L->T; ++t) L->slot_first[t + 1] = L->slot_first[t] + L->n_slots[t];
  const long long S = L->slot_first[L->T];
  L->slot_sizes.assign(D->slot_sizes, D->slot_sizes + S);
  L->row_first.assign(S + 1, 0);
  for (long long j = 0; j < S; ++j) L->row_first[j + 1] = L->row_first[j] + L->slot_sizes[j];
  L->rows = L->row_first[S];
  L->id_first.assign(L->T + 1, 0);
  for (int t = 0; t < L->T; ++t) {
    long long n = 1;
    for (long long j = L->slot_first[t]; j < L->slot_first[t + 1]; ++j) n *= L->slot_sizes[j];
    L->id_first[t + 1] = L->id_first[t] + n;
    L->max_slots = std::max(L->max_slots, L->n_slots[t]);
  }
  L->budget = D->device_mem_budget;
  L->device = D->device;
  L->seed = D->seed;
  L->tc_fmt[0] = want_bf16;
  L->tc_fmt[1] = want_fp16;
  L->tc_fmt[2] = want_fp8;
  L->precisions = 1u | (want_bf16 ? (1u << APEX_BF16) : 0u) | (want_fp16 ? (1u << APEX_FP16) : 0u) |
                  (want_fp8 ? (1u << APEX_FP8) : 0u);
  L->rng.seed(D->seed + 17);
  L->precisions_requested = D->precisions;
  for (int l = 0; l < D->n_layers; ++l) {
    L->hW.emplace_back(D->W[l], D->W[l] + (size_t)D->dims[l + 1] * D->dims[l]);
    L->hb.emplace_back(D->b[l], D->b[l] + D->dims[l + 1]);
  }

  try {
    CU(cudaSetDevice(L->device));
    cudaDeviceProp prop;
    CU(cudaGetDeviceProperties(&prop, L->device));
    L->n_sm = prop.multiProcessorCount;
    {
      size_t fr = 0, tot = 0;
      CU(cudaMemGetInfo(&fr, &tot));
      L->dev_total = tot;
    }
    if (D->cuda_stream) {
      L->st = (cudaStream_t)D->cuda_stream;
    } else {
      CU(cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking));
      L->own_stream = true;
    }
    const int d = L->d, h1 = L->dims[1];
    // U (kept for the FP64 plain rescore)
    float *dU = (float *)L->dalloc(sizeof(float) * L->rows * d);
    CU(cudaMemcpyAsync(dU, D->U, sizeof(float) * L->rows * d,
                       D->U_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, L->st));
    L->T_.U = dU;
    L->T_.d = d;
    L->T_.n_layers = L->n_layers;
    for (int l = 0; l <= L->n_layers; ++l) L->T_.dims[l] = L->dims[l];
    L->T_.act = L->act;
    L->T_.n_out = L->n_out;
    L->T_.n_rx = L->T;
    L->T_.n_rows = L->rows;
    // head: FP32 copies (transposed for layers >= 1) and FP64 transposed copies of every layer
    for (int l = 0; l < L->n_layers; ++l) {
      const int K = L->dims[l], Nn = L->dims[l + 1];
      std::vector<float> wt((size_t)K * Nn);
      std::vector<double> wt64((size_t)K * Nn), b64(Nn);
      for (int n = 0; n < Nn; ++n) {
        b64[n] = D->b[l][n];
        for (int k = 0; k < K; ++k) {
          wt[(size_t)k * Nn + n] = D->W[l][(size_t)n * K + k];
          wt64[(size_t)k * Nn + n] = D->W[l][(size_t)n * K + k];
        }
      }
      double *dw64 = (double *)L->dalloc(sizeof(double) * K * Nn);
      double *db64 = (double *)L->dalloc(sizeof(double) * Nn);
      CU(cudaMemcpy(dw64, wt64.data(), sizeof(double) * K * Nn, cudaMemcpyHostToDevice));
      CU(cudaMemcpy(db64, b64.data(), sizeof(double) * Nn, cudaMemcpyHostToDevice));
      L->T_.WT64[l] = dw64;
      L->T_.B64[l] = db64;
      if (l >= 1) {
        float *dw = (float *)L->dalloc(sizeof(float) * K * Nn);
        float *db = (float *)L->dalloc(sizeof(float) * Nn);
        CU(cudaMemcpy(dw, wt.data(), sizeof(float) * K * Nn, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(db, D->b[l], sizeof(float) * Nn, cudaMemcpyHostToDevice));
        L->T_.WT[l] = dw;
        L->T_.B[l] = db;
      }
    }
    // P32 = W_1 u + b_1 on slot-1 rows
    {
      float *dW1 = (float *)L->dalloc(sizeof(float) * h1 * d, false);
      float *db1 = (float *)L->dalloc(sizeof(float) * h1, false);
      CU(cudaMemcpy(dW1, D->W[0], sizeof(float) * h1 * d, cudaMemcpyHostToDevice));
      CU(cudaMemcpy(db1, D->b[0], sizeof(float) * h1, cudaMemcpyHostToDevice));
      std::vector<unsigned char> brow(L->rows, 0);
      for (int t = 0; t < L->T; ++t) {
        const long long j0 = L->slot_first[t];
        for (long long r = L->row_first[j0]; r < L->row_first[j0 + 1]; ++r) brow[r] = 1;
      }
      unsigned char *dbrow = (unsigned char *)L->dalloc(L->rows, false);
      CU(cudaMemcpy(dbrow, brow.data(), L->rows, cudaMemcpyHostToDevice));
      float *P32 = (float *)L->dalloc(sizeof(float) * L->rows * h1);
      CU(apx_launch_prep(dU, dW1, db1, dbrow, L->rows, d, h1, P32, L->st));
      L->T_.P32 = P32;
      if (L->tc_fmt[0] || L->tc_fmt[1] || L->tc_fmt[2]) {
        // tensor-core tables of every requested 16-bit format: P (scaled into the activation's
        // input space), W_2 (same scale) and W_3 (padded to 16 rows) as SW128 images, b_2, b_3
        const float scale = (L->act == APEX_ACT_SILU) ? 0.5f : 1.0f;
        std::vector<float> w2((size_t)256 * 256), w3((size_t)16 * 256, 0.f);
        for (size_t i = 0; i < w2.size(); ++i) w2[i] = scale * D->W[1][i];
        for (int n = 0; n < L->n_out; ++n)
          for (int k = 0; k < 256; ++k) w3[(size_t)n * 256 + k] = D->W[2][(size_t)n * 256 + k];
        float *dw = (float *)L->dalloc(sizeof(float) * (w2.size() + w3.size()), false);
        CU(cudaMemcpy(dw, w2.data(), sizeof(float) * w2.size(), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(dw + w2.size(), w3.data(), sizeof(float) * w3.size(), cudaMemcpyHostToDevice));
        for (int f = 0; f < 2; ++f) {  // 16-bit tables and images
          if (!L->tc_fmt[f]) continue;
          // one more row of zeros (row `rows`): the outer row of reactions without an outer slot
          void *P16 = L->dalloc(sizeof(unsigned short) * (L->rows + 1) * 256);
          CU(apx_launch_p16(P32, L->rows * 256, scale, f, P16, L->st));
          CU(cudaMemsetAsync((unsigned short *)P16 + (size_t)L->rows * 256, 0, sizeof(unsigned short) * 256, L->st));
          unsigned char *d2 = (unsigned char *)L->dalloc(256 * 256 * 2);
          unsigned char *d3 = (unsigned char *)L->dalloc(16 * 256 * 2);
          CU(apx_launch_image(dw, 256, 256, f, d2, L->st));
          CU(apx_launch_image(dw + w2.size(), L->n_out, 16, f, d3, L->st));
          L->T_.P16[f] = (const unsigned short *)P16;
          L->T_.w2img[f] = d2;
          L->T_.w3img[f] = d3;
        }
        if (L->tc_fmt[2]) {
          // FP8 layer 2. Activations: one static scale for the layer, from the exact maximum of
          // |a_1| over the whole library. z_1 of a compound is the sum of one P row per slot, so
          // its extremes over a reaction's Cartesian product are the sums of the per-slot column
          // extremes (computed on the device), and a_1 = act(z_1) is monotone on each side of the
          // activation's minimum. The scale is the power of two 2^floor(log2(448 / amax)), so the
          // multiply in FP16 is exact and |a_1| * scale <= 448 (the e4m3 maximum).
          const long long S = L->slot_first[L->T];
          long long *d_rf = (long long *)L->dalloc(sizeof(long long) * (S + 1), false);
          float *d_mx = (float *)L->dalloc(sizeof(float) * S * h1, false);
          float *d_mn = (float *)L->dalloc(sizeof(float) * S * h1, false);
          CU(cudaMemcpy(d_rf, L->row_first.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice));
          CU(apx_launch_slot_extremes(P32, d_rf, (int)S, h1, d_mx, d_mn, L->st));
          std::vector<float> hmx((size_t)S * h1), hmn((size_t)S * h1);
          CU(cudaMemcpyAsync(hmx.data(), d_mx, sizeof(float) * S * h1, cudaMemcpyDeviceToHost, L->st));
          CU(cudaMemcpyAsync(hmn.data(), d_mn, sizeof(float) * S * h1, cudaMemcpyDeviceToHost, L->st));
          CU(cudaStreamSynchronize(L->st));
          auto act = [&](double z) {
            return L->act == APEX_ACT_SILU ? z / (1.0 + std::exp(-z)) : L->act == APEX_ACT_RELU ? std::max(z, 0.0) : z;
          };
          // SiLU's minimum: SiLU'(z) = 0 <=> z = -(1 + e^z), i.e. z = -1 - W(1/e) (W: Lambert's function)
          const double z_silu_min = -1.2784645427610738;
          double amax = 0;
          for (int t = 0; t < L->T; ++t)
            for (int n = 0; n < h1; ++n) {
              double zx = 0, zn = 0;
              for (long long j = L->slot_first[t]; j < L->slot_first[t + 1]; ++j) {
                zx += hmx[(size_t)j * h1 + n];
                zn += hmn[(size_t)j * h1 + n];
              }
              double a = std::max(std::fabs(act(zx)), std::fabs(act(zn)));
              if (L->act == APEX_ACT_SILU && zn <= z_silu_min && z_silu_min <= zx) a = std::max(a, std::fabs(act(z_silu_min)));
              amax = std::max(amax, a);
            }
          L->a1_amax = amax;
          const double inv = amax > 0 ? std::exp2(std::floor(std::log2(448.0 / amax))) : 1.0;
          L->T_.a1_inv = (float)std::min(inv, 32768.0);
          // weights: every output channel of W_2 (already scaled) quantized with its own scale
          // max|row| / 448; the kernel multiplies the accumulators by s_2[n] / a1_inv
          std::vector<float> s2(256, 1.f), s2a(256, 1.f);
          for (int n = 0; n < 256; ++n) {
            float mx = 0.f;
            for (int k = 0; k < 256; ++k) mx = std::max(mx, std::fabs(w2[(size_t)n * 256 + k]));
            if (mx > 0.f) s2[n] = mx / 448.f;
            s2a[n] = (float)((double)s2[n] / (double)L->T_.a1_inv);
          }
          float *ds2 = (float *)L->dalloc(sizeof(float) * 256);
          float *ds2a = (float *)L->dalloc(sizeof(float) * 256);
          CU(cudaMemcpy(ds2, s2.data(), sizeof(float) * 256, cudaMemcpyHostToDevice));
          CU(cudaMemcpy(ds2a, s2a.data(), sizeof(float) * 256, cudaMemcpyHostToDevice));
          unsigned char *d2 = (unsigned char *)L->dalloc(256 * 256);
          CU(apx_launch_image_e4m3(dw, ds2, 256, 256, d2, L->st));
          L->T_.w2img[2] = d2;
          L->T_.s2 = ds2a;
        }
        std::vector<float> b2s(256), b3(16, 0.f);
        for (int n = 0; n < 256; ++n) b2s[n] = scale * D->b[1][n];
        for (int n = 0; n < L->n_out; ++n) b3[n] = D->b[2][n];
        float *db2 = (float *)L->dalloc(sizeof(float) * 256);
        float *db3 = (float *)L->dalloc(sizeof(float) * 16);
        CU(cudaMemcpy(db2, b2s.data(), sizeof(float) * 256, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(db3, b3.data(), sizeof(float) * 16, cudaMemcpyHostToDevice));
        L->T_.b2s = db2;
        L->T_.b3 = db3;
      }
    }
    // work plans: outer runs sized for ~32 tiles per item, fewer when the library is small
    {
      long long tiles_total = 0;
      for (int t = 0; t < L->T; ++t) {
        RxnPlan p = plan_reaction(*L, t, 1);
        tiles_total += (long long)p.n_b * p.n_outer;
      }
      const long long per_item = std::max<long long>(1, std::min<long long>(32, tiles_total / (L->n_sm * 16LL)));
      L->rx.resize(L->T);
      L->item_first.assign(L->T + 1, 0);
      for (int t = 0; t < L->T; ++t) {
        L->rx[t] = plan_reaction(*L, t, per_item);
        L->item_first[t + 1] = L->item_first[t] + L->rx[t].n_items;
      }
      L->total_items = L->item_first[L->T];
      L->T_ = upload_plans(*L);
    }
    L->d_slots = (QuerySlot *)L->dalloc(sizeof(QuerySlot) * APEX_MAX_ACTIVE);
    CU(cudaMemset(L->d_slots, 0, sizeof(QuerySlot) * APEX_MAX_ACTIVE));
    L->d_err = (int *)L->dalloc(sizeof(int));
    CU(cudaMemset(L->d_err, 0, sizeof(int)));
    L->d_slot_list = (int *)L->dalloc(sizeof(int) * APEX_MAX_ACTIVE);
    L->d_spec_full = (long long *)L->dalloc(sizeof(long long) * 16384);
    for (int i = 0; i < apex_library::kRing; ++i) {
      CU(cudaEventCreate(&L->ev_l0[i]));
      CU(cudaEventCreate(&L->ev_l1[i]));
      CU(cudaEventCreateWithFlags(&L->ev_ls[i], cudaEventDisableTiming));
    }
    CU(cudaMallocHost(&L->status_pin, sizeof(int) * apex_library::kRing));
    CU(cudaMallocHost(&L->cnt_pin, sizeof(unsigned) * 2 * APEX_MAX_ACTIVE * apex_library::kRing));
    memset(L->cnt_pin, 0, sizeof(unsigned) * 2 * APEX_MAX_ACTIVE * apex_library::kRing);
    L->d_obs_slots = (unsigned *)L->dalloc(sizeof(unsigned) * (1 + APEX_MAX_OUTPUTS) * APEX_MAX_ACTIVE);
    L->d_pool_ctr = (unsigned long long *)L->dalloc(sizeof(unsigned long long));
    L->pool_off = getenv("APEX_NO_TILE_POOL") != nullptr;
    if (trace_on())
      for (auto &e : L->ev_tr) CU(cudaEventCreate(&e));
    L->pin(1 << 20);
    CU(cudaStreamSynchronize(L->st));
    // a file's margins are restored when they cover every tensor-core format the library builds
    // (a file saved by a BF16-only library of an earlier build has no FP16 margins: recalibrate)
    bool cal_ok = cal != nullptr;
    for (int f = 0; f < 3 && cal_ok; ++f)
      for (int p = 0; p < L->n_out && cal_ok; ++p) cal_ok = !L->tc_fmt[f] || cal->err16[f][p] > 0;
    if (cal_ok) {
      L->n_calib = cal->n_calib;
      memcpy(L->err32, cal->err32, sizeof(L->err32));
      memcpy(L->err16, cal->err16, sizeof(L->err16));
      memcpy(L->rms, cal->rms, sizeof(L->rms));
      upload_err32(*L);
    } else {
      calibrate(*L);
    }
    CU(cudaStreamSynchronize(L->st));
  } catch (const CudaFail &f) {
    apex_status code = (f.e == cudaErrorMemoryAllocation) ? APEX_ENOMEM : APEX_ECUDA;
    if (f.e == cudaErrorLaunchTimeout) code = APEX_ETIMEDOUT;
    L->release_all();
    if (L->own_stream) cudaStreamDestroy(L->st);
    return fail(code, "load: %s failed: %s (line %d)", f.what, cudaGetErrorString(f.e), f.line);
  } catch (const BudgetFail &) {
    L->release_all();
    if (L->own_stream) cudaStreamDestroy(L->st);
    return fail(APEX_ENOMEM, "load: library tables exceed device_mem_budget");
  }
  apex_library *lib = L.release();
  lib->worker = std::thread(worker_main, lib);
  // the worker chooses its CPU before the first query (the caller is blocked here meanwhile, so
  // it does not disturb the timing of the candidate CPUs)
  const double t_w = now_ms();
  while (lib->worker_cpu.load() == -2 && now_ms() - t_w < 5000.0)
    std::this_thread::sleep_for(std::chrono::microseconds(100));
  *out = lib;
  return APEX_OK;
}

extern "C" apex_status apex_free_library(apex_library *L) {
  if (!L) return APEX_OK;
  {
    std::lock_guard<std::mutex> g(L->mu);
    L->stop = true;
    L->work_seq++;
  }
  L->cv.notify_all();
  if (L->worker.joinable()) L->worker.join();
  cudaSetDevice(L->device);
  cudaStreamSynchronize(L->st);
  for (auto &kv : L->queries) {
    QueryRec *q = kv.second.get();
    if (q->ev0) cudaEventDestroy(q->ev0);
    if (q->ev1) cudaEventDestroy(q->ev1);
  }
  for (auto &e : L->ev_pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto &B : L->slotbuf)
    if (B.cap) {
      cudaFree(B.keys);
      cudaFree(B.keys2);
      cudaFree(B.ids);
      cudaFree(B.ids2);
    }
  if (L->arena) cudaFree(L->arena);
  if (L->pinned) cudaFreeHost(L->pinned);
  if (L->up) cudaFreeHost(L->up);
  if (L->dl) cudaFreeHost(L->dl);
  for (int i = 0; i < apex_library::kRing; ++i) {
    if (L->ev_l0[i]) cudaEventDestroy(L->ev_l0[i]);
    if (L->ev_l1[i]) cudaEventDestroy(L->ev_l1[i]);
    if (L->ev_ls[i]) cudaEventDestroy(L->ev_ls[i]);
  }
  if (L->status_pin) cudaFreeHost(L->status_pin);
  if (L->cnt_pin) cudaFreeHost(L->cnt_pin);
  for (auto &e : L->ev_tr)
    if (e) cudaEventDestroy(e);
  L->release_all();
  if (L->own_stream) cudaStreamDestroy(L->st);
  delete L;
  return APEX_OK;
}

extern "C" apex_status apex_library_info(const apex_library *L, apex_library_info_t *o) {
  if (!L || !o) return fail(APEX_EINVAL, "NULL argument");
  memset(o, 0, sizeof(*o));
  o->n_compounds = L->N;
  o->n_synthon_rows = L->rows;
  o->max_slots = L->max_slots;
  o->n_outputs = L->n_out;
  o->device_bytes = L->bytes;
  o->precisions = L->precisions;
  o->n_calibration = L->n_calib;
  for (int p = 0; p < L->n_out; ++p) {
    o->err_bf16[p] = L->err16[0][p];
    o->err_fp16[p] = L->err16[1][p];
    o->err_fp8[p] = L->err16[2][p];
    o->err_fp32[p] = L->err32[p];
    o->rms[p] = L->rms[p];
  }
  return APEX_OK;
}

extern "C" apex_status apex_decode_ids(const apex_library *L, int64_t n, const int64_t *ids, int32_t *reaction,
                                       int64_t *synthons) {
  if (!L || n < 0 || (n > 0 && !ids)) return fail(APEX_EINVAL, "bad arguments");
  for (int64_t i = 0; i < n; ++i) {
    const long long id = ids[i];
    if (id < 0 || id >= L->N) return fail(APEX_EINVAL, "id %lld outside [0, %lld)", id, L->N);
    const int t = (int)(std::upper_bound(L->id_first.begin(), L->id_first.end(), id) - L->id_first.begin()) - 1;
    long long rem = id - L->id_first[t];
    long long s[APEX_MAX_SLOTS];
    for (int j = APEX_MAX_SLOTS - 1; j >= 0; --j) {
      if (j < L->n_slots[t]) {
        const long long sz = L->slot_sizes[L->slot_first[t] + j];
        s[j] = rem % sz;
        rem /= sz;
      } else {
        s[j] = -1;
      }
    }
    if (reaction) reaction[i] = t;
    if (synthons)
      for (int j = 0; j < APEX_MAX_SLOTS; ++j) synthons[i * APEX_MAX_SLOTS + j] = s[j];
  }
  return APEX_OK;
}

// ------------------------------------------------------------------ query submission
extern "C" apex_status apex_query(apex_library *L, const apex_query_desc *Dq, apex_query_id *out) {
  if (!L || !Dq || !out) return fail(APEX_EINVAL, "NULL argument");
  if (Dq->precision != APEX_FP32 && Dq->precision != APEX_BF16 && Dq->precision != APEX_FP16 &&
      Dq->precision != APEX_FP8)
    return fail(APEX_EINVAL, "unknown precision %d", Dq->precision);
  if (!((L->precisions >> Dq->precision) & 1u))
    return fail(APEX_EUNSUPPORTED, "precision %d tables were not built at load", Dq->precision);
  if (!Dq->objective_weights) return fail(APEX_EINVAL, "objective_weights is NULL");
  if (Dq->k < 1) return fail(APEX_EINVAL, "k must be >= 1");
  if (Dq->k > (1LL << 24)) return fail(APEX_EINVAL, "k must be <= 2^24");
  if (Dq->n_constraints < 0 || Dq->n_constraints > APEX_MAX_CONSTRAINTS)
    return fail(APEX_EINVAL, "n_constraints outside 0..%d", APEX_MAX_CONSTRAINTS);
  if (Dq->n_constraints > 0 && (!Dq->output_index || !Dq->lower || !Dq->upper))
    return fail(APEX_EINVAL, "constraint arrays are NULL");
  std::unique_ptr<QueryRec> q(new QueryRec());
  q->precision = Dq->precision;
  q->w.assign(Dq->objective_weights, Dq->objective_weights + L->n_obj);
  for (float x : q->w)
    if (!std::isfinite(x)) return fail(APEX_EINVAL, "objective weight is not finite");
  for (int i = 0; i < Dq->n_constraints; ++i) {
    if (Dq->output_index[i] < 0 || Dq->output_index[i] >= L->n_out)
      return fail(APEX_EINVAL, "constraint %d: output index %d outside 0..%d", i, Dq->output_index[i], L->n_out - 1);
    if (std::isnan(Dq->lower[i]) || std::isnan(Dq->upper[i]))
      return fail(APEX_EINVAL, "constraint %d: NaN bound", i);
    if (Dq->lower[i] > Dq->upper[i]) return fail(APEX_EINVAL, "constraint %d: lower > upper", i);
    q->cidx.push_back(Dq->output_index[i]);
    q->lo.push_back(Dq->lower[i]);
    q->hi.push_back(Dq->upper[i]);
  }
  q->k = Dq->k;
  q->need.assign(L->T, 0);
  if (Dq->n_reaction_subset > 0) {
    if (!Dq->reactions) return fail(APEX_EINVAL, "reactions is NULL");
    for (int i = 0; i < Dq->n_reaction_subset; ++i) {
      const int t = Dq->reactions[i];
      if (t < 0 || t >= L->T) return fail(APEX_EINVAL, "reaction %d outside 0..%d", t, L->T - 1);
      if (q->need[t]) return fail(APEX_EINVAL, "reaction %d listed twice", t);
      q->need[t] = 1;
    }
  } else if (Dq->n_reaction_subset < 0) {
    return fail(APEX_EINVAL, "negative n_reaction_subset");
  } else {
    std::fill(q->need.begin(), q->need.end(), 1);
  }
  for (int t = 0; t < L->T; ++t)
    if (q->need[t]) {
      q->subset.push_back(t);
      q->scope_items += L->rx[t].n_items;
      q->scope_n += L->id_first[t + 1] - L->id_first[t];
    }
  q->remaining = q->scope_items;
  q->t_submit = now_ms();
  q->id = L->next_id++;
  const apex_query_id id = q->id;
  {
    std::unique_lock<std::mutex> g(L->mu, std::defer_lock);
    lock_spin(g);
    if (L->stop) return fail(APEX_ECANCELED, "library is shutting down");
    L->queued.push_back(q.get());
    L->queries[id] = std::move(q);
    L->work_seq++;
  }
  L->cv.notify_all();
  *out = id;
  return APEX_OK;
}

extern "C" apex_status apex_cancel(apex_library *L, apex_query_id id) {
  if (!L) return fail(APEX_EINVAL, "NULL library");
  std::lock_guard<std::mutex> g(L->mu);
  auto it = L->queries.find(id);
  if (it == L->queries.end()) return fail(APEX_ENOTFOUND, "query %lld not found", (long long)id);
  it->second->cancel = true;
  L->work_seq++;
  L->cv.notify_all();
  return APEX_OK;
}

// ------------------------------------------------------------------ worker: admission
static size_t query_bytes_for(unsigned cap) { return (size_t)cap * (4 + 8) * 2; }

static void free_query_device(apex_library &L, QueryRec *q) {
  (void)L;
  q->keys = q->keys2 = nullptr;
  q->ids = q->ids2 = nullptr;
  q->dev_bytes = 0;
}

static unsigned *slot_obs(apex_library &L, int slot) { return L.d_obs_slots + (size_t)slot * (1 + APEX_MAX_OUTPUTS); }

// Writes the query's slot parameters (boxes widened / shrunk by the pass margin).
static void write_slot(apex_library &L, QueryRec *q, float admit) {
  QuerySlot S;
  memset(&S, 0, sizeof(S));
  const double *err = pass_err(L, q->precision);
  const double sc = q->mscale;
  for (int j = 0; j < L.n_obj; ++j) S.w[j] = q->w[j];
  S.n_obj = L.n_obj;
  S.n_cons = (int)q->cidx.size();
  double df = 0;
  for (int j = 0; j < L.n_obj; ++j) df += std::fabs((double)q->w[j]) * err[j] * sc;
  for (int c = 0; c < S.n_cons; ++c) {
    const int p = q->cidx[c];
    S.cons_idx[c] = p;
    S.lo_w[c] = (float)(q->lo[c] - err[p] * sc);
    S.hi_w[c] = (float)(q->hi[c] + err[p] * sc);
    S.lo_s[c] = (float)(q->lo[c] + err[p] * sc);
    S.hi_s[c] = (float)(q->hi[c] - err[p] * sc);
    float lx = (float)q->lo[c], hx = (float)q->hi[c];  // exact decisions for FP32 values
    if ((double)lx < q->lo[c]) lx = std::nextafter(lx, INFINITY);
    if ((double)hx > q->hi[c]) hx = std::nextafter(hx, -INFINITY);
    S.lo_x[c] = lx;
    S.hi_x[c] = hx;
  }
  S.delta_f = (float)(df * 1.0001 + 1e-12);
  S.admit = admit;
  S.tau = -INFINITY;
  S.tau_spec = q->tau_spec;
  S.k = q->k;
  S.cap = q->cap;
  S.keys = q->keys;
  S.ids = q->ids;
  S.keys2 = q->keys2;
  S.ids2 = q->ids2;
  L.upload(L.d_slots + q->slot, &S, sizeof(S));
  CU(cudaMemsetAsync(slot_obs(L, q->slot), 0, sizeof(unsigned) * (1 + APEX_MAX_OUTPUTS), L.st));
  q->want_compact = false;
  q->seen_count = 0;
}


// Start threshold guess, computed on the device without a host round trip: the rank-r best
// objective among the feasible compounds (exact boxes, outputs of the pass's precision) of a
// uniform sample of the query's scope, r chosen so that ~3k scope compounds are expected above
// it. The kernel writes the slot's start threshold and admission threshold (start - 2 delta_f)
// in stream order before
// the enumeration launch. Only a guess: finalization verifies it (>= k sure entries at or above
// it) or restarts lower. Returns false (and leaves the slot's -inf thresholds) when the sample
// cannot hold rank r.
static bool speculative_start(apex_library &L, QueryRec *q, double margin2) {
  if (q->spec_rank < 0) return false;
  const double t_a = now_ms();
  // the sample is scored by the pass's own kernel when it runs on the tensor cores (a 16,384-id
  // sample costs one tile per CTA), else by the FP32 kernel (4,096 ids)
  const int fmt = tc_format(q->precision);
  const long long S = std::min<long long>(fmt >= 0 ? 16384 : 4096, q->scope_n);
  const double expect = (double)S * (double)q->k / (double)q->scope_n;
  long long r = q->spec_rank > 0 ? q->spec_rank : (long long)std::ceil(3.0 * expect + 5.0);
  q->spec_rank = (int)std::min<long long>(r, 1 << 30);
  if (r >= S) {
    q->spec_rank = -1;
    return false;
  }
  const int n_sub = (int)q->subset.size();
  const int no = L.n_out;
  L.arena_reserve(sizeof(int) * n_sub + sizeof(long long) * (n_sub + 1) + sizeof(long long) * S +
                  sizeof(float) * S * (no + 1) + S + 8 * 256);
  float *d_out = (float *)L.aget(sizeof(float) * S * no);
  float *d_keys = (float *)L.aget(sizeof(float) * S);
  unsigned char *d_flag = (unsigned char *)L.aget(S);
  // a whole-library query reuses the library's own sample (the threshold is a guess that the
  // finalization verifies, so any uniform sample serves); a subset draws one from its scope
  const bool full = n_sub == L.T;
  long long *d_ids = full ? L.d_spec_full : nullptr;
  if (!full || L.spec_full_n < S) {
    std::vector<long long> pre(n_sub + 1, 0);
    for (int i = 0; i < n_sub; ++i) pre[i + 1] = pre[i] + (L.id_first[q->subset[i] + 1] - L.id_first[q->subset[i]]);
    int *d_rxn = (int *)L.aget(sizeof(int) * n_sub);
    long long *d_pre = (long long *)L.aget(sizeof(long long) * (n_sub + 1));
    if (!full) d_ids = (long long *)L.aget(sizeof(long long) * S);
    const long long n_draw = full ? std::min<long long>(16384, q->scope_n) : S;
    L.upload(d_rxn, q->subset.data(), sizeof(int) * n_sub);
    L.upload(d_pre, pre.data(), sizeof(long long) * (n_sub + 1));
    CU(apx_launch_spec_ids(d_rxn, d_pre, n_sub, L.T_.id_first, q->scope_n, L.rng(), n_draw, d_ids, L.st));
    if (full) L.spec_full_n = n_draw;
  }
  if (fmt >= 0) {  // the kernel applies the query's exact boxes and objective: one key per sample
    CU(apx_launch_tc_ids(L.T_, d_ids, S, d_out, L.d_err, L.n_sm, L.st, fmt, L.d_slots, q->slot));
  } else {
    LaunchPlan dummy;
    memset(&dummy, 0, sizeof(dummy));
    CU(apx_launch_fp32(dummy, L.T_, nullptr, d_ids, S, d_out, grid_for(L, (S + APX_TILE - 1) / APX_TILE), L.st,
                       L.fp32_id_tile.load()));
  }
  SpecArgs a;
  memset(&a, 0, sizeof(a));
  for (int j = 0; j < L.n_obj; ++j) a.w[j] = q->w[j];
  a.n_obj = L.n_obj;
  a.n_cons = (int)q->cidx.size();
  a.n_out = no;
  for (int c = 0; c < a.n_cons; ++c) {
    a.cons_idx[c] = q->cidx[c];
    a.lo[c] = q->lo[c];
    a.hi[c] = q->hi[c];
  }
  a.rank = r;
  a.margin2 = (float)margin2;
  a.bits_in = fmt >= 0 ? 1 : 0;
  CU(apx_launch_spec_select(d_out, S, a, d_keys, d_flag, L.d_slots + q->slot, L.st));
  TRACE("start q%lld: host %.3f ms (sample of %lld, rank %lld)", (long long)q->id, now_ms() - t_a, S, r);
  return true;
}

static double pass_delta_f(const apex_library &L, const QueryRec *q) {
  const double *err = pass_err(L, q->precision);
  double df = 0;
  for (int j = 0; j < L.n_obj; ++j) df += std::fabs((double)q->w[j]) * err[j];
  return df * q->mscale;
}
// objective margin of the FP32 rescore for this query
static double fp32_delta_f(const apex_library &L, const QueryRec *q) {
  double e = 0;
  for (int j = 0; j < L.n_obj; ++j) e += std::fabs((double)q->w[j]) * L.err32[j];
  return e * q->mscale;
}
// In-pass compactions of a BF16 or FP8 pass rescore in FP16 on the tensor cores (the id-list form
// of the enumeration kernel): its margins are about a tenth of BF16's and it scores a candidate
// ~30x faster than the FP32 SIMT kernel; the end-of-pass rescore stays FP32. Other passes (and
// libraries without the FP16 tables) compact in FP32.
static bool compact_fp16(const apex_library &L, const QueryRec *q) {
  return L.tc_fmt[1] && L.d_err16f && (q->precision == APEX_BF16 || q->precision == APEX_FP8);
}
// objective margin of the compaction rescore for this query
static double compact_delta_f(const apex_library &L, const QueryRec *q) {
  if (!compact_fp16(L, q)) return fp32_delta_f(L, q);
  double e = 0;
  for (int j = 0; j < L.n_obj; ++j) e += std::fabs((double)q->w[j]) * L.err16[1][j];
  return e * q->mscale;
}

static void start_query(apex_library &L, QueryRec *q) {
  tmark(L, 0);
  q->stats.first_item = L.cursor;
  const double df = pass_delta_f(L, q);
  q->tau_spec = -INFINITY;  // the device-side guess lands in the slot; finalization reads it back
  write_slot(L, q, -INFINITY);
  speculative_start(L, q, 2.0 * df * 1.0001);
  tmark(L, 1);
  q->remaining = q->scope_items;
  q->started = true;
}

static void slot_reserve(apex_library &L, int slot, unsigned cap) {
  apex_library::SlotBuf &B = L.slotbuf[slot];
  if (B.cap >= cap) return;
  if (B.cap) {
    CU(cudaStreamSynchronize(L.st));
    cudaFree(B.keys);
    cudaFree(B.keys2);
    cudaFree(B.ids);
    cudaFree(B.ids2);
    L.query_bytes -= query_bytes_for(B.cap);
    B = apex_library::SlotBuf();
  }
  CU(cudaMalloc(&B.keys, sizeof(float) * cap));
  CU(cudaMalloc(&B.keys2, sizeof(float) * cap));
  CU(cudaMalloc(&B.ids, sizeof(long long) * cap));
  CU(cudaMalloc(&B.ids2, sizeof(long long) * cap));
  B.cap = cap;
  L.query_bytes += query_bytes_for(cap);
}

static void bind_slot(apex_library &L, QueryRec *q) {
  slot_reserve(L, q->slot, q->cap);
  apex_library::SlotBuf &B = L.slotbuf[q->slot];
  q->keys = B.keys;
  q->keys2 = B.keys2;
  q->ids = B.ids;
  q->ids2 = B.ids2;
}

static bool admit_one(apex_library &L, QueryRec *q) {
  int slot = -1;
  for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
    if (!L.active[s]) {
      slot = s;
      break;
    }
  if (slot < 0) return false;
  // candidate buffer: 2^18 entries or 8k for scopes up to 2^28 compounds; above that, where a loose
  // or missing start threshold meets launches of 2^26 - 2^27 compounds, 2^20 entries or 32k (a
  // narrow box can leave fewer than k compounds surely feasible in the start sample, and then the
  // buffer holds every admitted candidate until k sure ones exist); grown 4x after an overflow
  if (q->cap == 0) {
    const bool big = q->scope_n > (1LL << 28);
    // an FP8 pass admits ~7x the band of a BF16 one (its margins): on scopes of 3e10 compounds its
    // buffers overflowed within one launch until they held 2^26 entries (three 4x restarts)
    const long long base = big ? (q->precision == APEX_FP8 ? 1LL << 26 : 1LL << 20) : 1LL << 18;
    q->cap = (unsigned)std::min<long long>(std::max<long long>(base, (big ? 32 : 8) * q->k), 1LL << 30);
  }
  const unsigned have = L.slotbuf[slot].cap;
  if (have < q->cap) {
    const size_t need = query_bytes_for(q->cap) - query_bytes_for(have);
    if (L.budget && L.bytes + L.query_bytes + need > L.budget) return false;
  }
  q->slot = slot;
  bind_slot(L, q);
  L.active[slot] = q;
  q->state = Q_ACTIVE;
  q->t_admit = now_ms();
  if (!q->ev0 && !L.ev_pool.empty()) {
    q->ev0 = L.ev_pool.back().first;
    q->ev1 = L.ev_pool.back().second;
    L.ev_pool.pop_back();
  }
  if (!q->ev0) {
    CU(cudaEventCreate(&q->ev0));
    CU(cudaEventCreate(&q->ev1));
  }
  return true;
}

// ------------------------------------------------------------------ worker: finalization

// A query's finalization after its pass: the slot's last select (threshold raise and
// compaction), then on the device the FP32 rescore of the candidates, their FP32 decisions, the
// result set R, the FP64 rescore of R's boundary band, the ordering of R and the final rows,
// copied to pinned host memory. The chain is queued right behind the pass's last launch, before
// the candidate count is known: it covers up to `cover` candidates and every kernel reads the
// actual count from the slot, so the host waits once per query. After that wait the host checks
// the count and the exactness conditions; a chain that did not fit (count > cover) or whose
// boundary band moved during its FP64 round is queued again, sized exactly, with further rounds
// as needed.
struct FinChain {
  QueryRec *q = nullptr;
  int sl = -1;
  unsigned cover = 0, nr = 0, np = 2, nc1 = 1, n_rows = 0;
  long long k = 0;
  double tol = 0;
  float *out32 = nullptr, *d_tau = nullptr;
  RItem *R = nullptr;
  unsigned *d_cnt = nullptr;  // [0] |R|, [1] FP64 batch, [2] newly marked, [3] alive, [4] FP64-rescored
  long long *ids64 = nullptr;
  int *pos64 = nullptr;
  double *o64 = nullptr, *out64 = nullptr, *dlo = nullptr, *dhi = nullptr;
  long long *e_ids = nullptr, *e_syn = nullptr;
  int *e_rxn = nullptr;
  double *e_obj = nullptr, *e_out = nullptr;
  size_t span = 0;
  char *h = nullptr;          // pinned copy of the rows [e_ids, e_out + n_rows * n_out)
  unsigned *h_cnt = nullptr;  // pinned copy of d_cnt
  QuerySlot *hS = nullptr;    // pinned copy of the slot after its last select
  unsigned *d_obs = nullptr;  // [1 + APEX_MAX_OUTPUTS] observed errors (EvalArgs::obs), float bits
  unsigned *h_obs = nullptr;  // pinned copy of d_obs
  int rounds = 0;
};

static unsigned fin_pow2(unsigned n) {
  unsigned p = 2;
  while (p < n) p <<= 1;
  return p;
}
static size_t fin_row_bytes(const apex_library &L) {
  return 8 + 4 + 8 * APEX_MAX_SLOTS + 8 + 8 * (size_t)L.n_out;
}
// device scratch of a chain covering `cover` candidates (256-byte roundings in the slack)
static size_t fin_arena_bytes(const apex_library &L, const QueryRec *q, unsigned cover) {
  const size_t ncx = std::max(cover, 1u), no = L.n_out;
  const size_t kx = (size_t)std::min<long long>(q->k, (long long)ncx);
  return ncx * (4 * no + 4 + 2 + 8 * no + 8 + 4 + 8 * no) + fin_pow2((unsigned)ncx) * sizeof(RItem) +
         kx * fin_row_bytes(L) + 64 * 1024;
}
// pinned host memory of the same chain: its rows, counters and slot copy
static size_t fin_pinned_bytes(const apex_library &L, const QueryRec *q, unsigned cover) {
  const size_t kx = (size_t)std::min<long long>(q->k, (long long)cover);
  return kx * fin_row_bytes(L) + 5 * 64 + 64 + sizeof(QuerySlot) + 64 + 4 * (1 + APEX_MAX_OUTPUTS) + 64;
}
// candidates an optimistic chain covers: the usual candidate set is a small multiple of k (at most
// 2^20 by default: the scratch grows ~280 bytes per covered candidate)
static unsigned fin_cover_base(const apex_library &L, const QueryRec *q) {
  const long long set = L.fin_cover_set.load();
  const long long c = set > 0 ? set : std::max<long long>(4096, std::min<long long>(4 * q->k, 1LL << 20));
  return (unsigned)std::min<long long>(c, (long long)q->cap);
}
// ... and at least 1.5x the count the query's buffer held after the select of its last retired
// launch (an FP16 compaction keeps a wider band than the FP32 one, so counts above 4k are common
// at the end of a BF16 pass; a chain that does not cover the count takes the exact rerun), at most
// 2^22 candidates
static unsigned fin_cover(const apex_library &L, const QueryRec *q) {
  const unsigned c = fin_cover_base(L, q);
  if (L.fin_cover_set.load() > 0 || q->seen_count == 0) return c;
  const long long want = std::min<long long>((long long)q->seen_count + q->seen_count / 2 + 4096, 1LL << 22);
  return (unsigned)std::min<long long>(std::max<long long>(c, want), (long long)q->cap);
}

// One FP64 round: rescore what is pending (near a box bound, or in the boundary band of the k-th
// score), re-sort, re-mark the band (the FP64 launch reads its batch size on the device).
static void fin_round(apex_library &L, FinChain &C) {
  CU(cudaMemsetAsync(C.d_cnt + 1, 0, sizeof(unsigned) * 2, L.st));
  CU(apx_launch_collect64(C.R, C.nr, C.ids64, C.pos64, C.d_cnt + 1, L.st));
  CU(apx_launch_fp64(L.T_, C.ids64, C.nc1, C.o64, L.st, C.d_cnt + 1));
  CU(apx_launch_apply64(C.R, C.pos64, C.o64, C.nc1, C.d_cnt + 1, L.n_out, L.d_slots + C.sl, C.dlo, C.dhi, C.out64,
                        L.st, C.out32, C.d_obs));
  CU(apx_sort_r(C.R, C.np, C.np, L.st, C.d_cnt));
  CU(apx_launch_mark(C.R, C.nr, (unsigned)std::min<long long>(C.k + 1, C.nr), C.k, C.tol, C.d_cnt + 2, L.st,
                     C.d_cnt));  // boundary band
  C.rounds++;
}

// The final rows, min(k, alive) of them, emitted on the device from the device count, and their
// copy (with the counters) to pinned host memory. No wait.
static void fin_emit(apex_library &L, FinChain &C) {
  CU(cudaMemsetAsync(C.d_cnt + 3, 0, sizeof(unsigned) * 2, L.st));
  CU(apx_launch_count_alive(C.R, C.nr, C.d_cnt + 3, L.st));
  CU(apx_launch_emit(C.R, C.n_rows, C.d_cnt + 3, L.T_, C.out32, C.out64, C.e_ids, C.e_rxn, C.e_syn, C.e_obj,
                     C.e_out, L.st));
  CU(cudaEventRecord(C.q->ev1, L.st));
  if (C.span) CU(cudaMemcpyAsync(C.h, C.e_ids, C.span, cudaMemcpyDeviceToHost, L.st));
  CU(cudaMemcpyAsync(C.h_cnt, C.d_cnt, sizeof(unsigned) * 8, cudaMemcpyDeviceToHost, L.st));
  CU(cudaMemcpyAsync(C.h_obs, C.d_obs, sizeof(unsigned) * (1 + APEX_MAX_OUTPUTS), cudaMemcpyDeviceToHost, L.st));
}

// Queues the chain of query q over up to `cover` candidates (the slot's count, read on the device,
// decides how many are used). Arena and download area must hold fin_arena_bytes /
// fin_pinned_bytes for it.
static void fin_queue(apex_library &L, QueryRec *q, FinChain &C, unsigned cover) {
  const int no = L.n_out;
  C.q = q;
  C.sl = q->slot;
  C.cover = cover;
  C.k = q->k;
  C.rounds = 0;
  const unsigned *d_n = &L.d_slots[C.sl].count;
  const unsigned n1 = std::max(cover, 1u);
  C.nc1 = n1;
  // FP32 rescore of the candidates
  C.out32 = (float *)L.aget(sizeof(float) * n1 * no);
  if (cover > 0) {
    LaunchPlan dummy;
    memset(&dummy, 0, sizeof(dummy));
    CU(apx_launch_fp32(dummy, L.T_, nullptr, q->ids, cover, C.out32, grid_for(L, (cover + APX_TILE - 1) / APX_TILE),
                       L.st, L.fp32_id_tile.load(), d_n));
  }
  float *f32 = (float *)L.aget(sizeof(float) * n1);
  unsigned char *maybe = (unsigned char *)L.aget(n1);
  unsigned char *sure = (unsigned char *)L.aget(n1);
  const int m = (int)q->cidx.size();
  C.dlo = (double *)L.aget(sizeof(double) * std::max(m, 1));
  C.dhi = (double *)L.aget(sizeof(double) * std::max(m, 1));
  if (m > 0) {
    L.upload(C.dlo, q->lo.data(), sizeof(double) * m);
    L.upload(C.dhi, q->hi.data(), sizeof(double) * m);
  }
  const double e32f = fp32_delta_f(L, q);
  C.d_obs = slot_obs(L, C.sl);  // accumulates over the pass's compactions and this chain
  EvalArgs ea{C.out32, no, L.d_slots + C.sl, L.d_err32f, (float)e32f, C.dlo, C.dhi};
  ea.eps_scale = (float)q->mscale;
  ea.pass_keys = q->keys;  // compacted with the ids by the slot's last select
  ea.obs = C.d_obs;
  // keys an in-pass compaction rescored are held to that rescore's margin: scaled up by pass
  // margin / compaction margin, their |key - FP32| counts in the same observed ratio
  ea.ids = q->ids;
  {
    const double ec = compact_delta_f(L, q), ep = pass_delta_f(L, q);
    ea.scored_scale = ec > 0 && ep > ec ? (float)(ep / ec) : 1.f;
  }
  CU(apx_launch_eval32(ea, cover, f32, maybe, sure, L.st, d_n));
  C.d_tau = (float *)L.aget(sizeof(float));
  int *d_ok = (int *)L.aget(sizeof(int));
  CU(apx_launch_kth(f32, sure, cover, C.k, C.d_tau, d_ok, L.st, d_n));
  // R = the candidates that may reach the FP32 top-k band (threshold taken on the device); |R|
  // stays on the device: R is padded to np with dead items from the device count and every later
  // kernel covers np entries (dead ones are skipped)
  C.np = fin_pow2(n1);
  C.R = (RItem *)L.aget(sizeof(RItem) * C.np);
  C.d_cnt = (unsigned *)L.aget(sizeof(unsigned) * 8);
  CU(cudaMemsetAsync(C.d_cnt, 0, sizeof(unsigned) * 8, L.st));
  CU(apx_launch_build_r(cover, q->ids, f32, maybe, sure, C.d_tau, (float)(2.0 * e32f * 1.0001), C.R, C.d_cnt, L.st,
                        d_n));
  CU(apx_launch_pad_r_dev(C.R, C.d_cnt, C.np, L.st));
  tmark(L, 3);
  C.nr = cover > 0 ? C.np : 0;
  C.out64 = (double *)L.aget(sizeof(double) * n1 * no);
  C.ids64 = (long long *)L.aget(sizeof(long long) * n1);  // FP64 batches: at most |R| <= count
  C.pos64 = (int *)L.aget(sizeof(int) * n1);
  C.o64 = (double *)L.aget(sizeof(double) * n1 * no);
  C.tol = 2.0 * e32f * 1.0001 + 1e-300;
  C.n_rows = (unsigned)std::min<long long>(C.k, cover);
  C.span = 0;
  if (C.n_rows > 0) {
    C.e_ids = (long long *)L.aget(sizeof(long long) * C.n_rows);
    C.e_rxn = (int *)L.aget(sizeof(int) * C.n_rows);
    C.e_syn = (long long *)L.aget(sizeof(long long) * C.n_rows * APEX_MAX_SLOTS);
    C.e_obj = (double *)L.aget(sizeof(double) * C.n_rows);
    C.e_out = (double *)L.aget(sizeof(double) * C.n_rows * no);
    C.span = (size_t)((char *)(C.e_out + (size_t)C.n_rows * no) - (char *)C.e_ids);
  }
  C.h = (char *)L.dl_get(std::max<size_t>(C.span, 1));
  C.h_cnt = (unsigned *)L.dl_get(sizeof(unsigned) * 8);
  C.h_obs = (unsigned *)L.dl_get(sizeof(unsigned) * (1 + APEX_MAX_OUTPUTS));
  // the band around the FP32 k-th score is marked before the first round, so one round usually
  // settles it
  if (C.nr > 0) {
    CU(apx_launch_mark_near(C.R, C.nr, C.d_tau, C.tol, C.d_cnt + 2, L.st));
    fin_round(L, C);
  }
  tmark(L, 4);
  fin_emit(L, C);
}

// Copies the rows of a finished chain into the query record.
static void fin_take(apex_library &L, FinChain &C) {
  QueryRec *q = C.q;
  const int no = L.n_out;
  q->stats.n_rescored_fp64 = C.nr > 0 ? (long long)C.h_cnt[4] : 0;
  const long long alive = C.nr > 0 ? (long long)C.h_cnt[3] : 0;
  const long long nf = std::min<long long>(C.k, alive);
  // copied straight from the pinned rows (no zero-fill first)
  const char *b = (const char *)C.e_ids;
  auto at = [&](const void *dev) { return C.h + ((const char *)dev - b); };
  const long long *ids = nf > 0 ? (const long long *)C.h : nullptr;
  const int *rxn = nf > 0 ? (const int *)at(C.e_rxn) : nullptr;
  const long long *syn = nf > 0 ? (const long long *)at(C.e_syn) : nullptr;
  const double *obj = nf > 0 ? (const double *)at(C.e_obj) : nullptr;
  const double *out = nf > 0 ? (const double *)at(C.e_out) : nullptr;
  q->r_ids.assign(ids, ids + (nf > 0 ? nf : 0));
  q->r_rxn.assign(rxn, rxn + (nf > 0 ? nf : 0));
  q->r_syn.assign(syn, syn + (nf > 0 ? nf * APEX_MAX_SLOTS : 0));
  q->r_obj.assign(obj, obj + (nf > 0 ? nf : 0));
  q->r_out.assign(out, out + (nf > 0 ? nf * no : 0));
  q->stats.n_feasible_lower = nf;
  // observed errors against the margins this run was admitted and decided with
  auto bits_f = [](unsigned u) {
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
  };
  const double df = pass_delta_f(L, q);
  q->stats.pass_err_ratio = df > 0 ? bits_f(C.h_obs[0]) / df : 0.0;
  double r32 = 0;
  for (int p = 0; p < no; ++p)
    if (L.err32[p] > 0) r32 = std::max(r32, bits_f(C.h_obs[1 + p]) / (L.err32[p] * q->mscale));
  q->stats.fp32_err_ratio = r32;
}

// After fin_take: whether an observed error exceeded the margin the run used (the run is then
// repeated with wider margins, up to kMaxMarginReruns times).
static constexpr int kMaxMarginReruns = 4;
static bool fin_margin_exceeded(const QueryRec *q) {
  return (q->stats.pass_err_ratio > 1.0 || q->stats.fp32_err_ratio > 1.0) &&
         q->stats.n_margin_reruns < kMaxMarginReruns;
}

// Decides from the slot after its last select whether the query must run its pass again: the
// start guess was too high (fewer than k sure entries reach it) or the candidate buffer
// overflowed with a possible member of the top-k dropped.
static bool fin_needs_restart(const apex_library &L, const QueryRec *q, const QuerySlot &S, bool *spec_bad_out,
                              bool *overflow_out) {
  const bool spec_bad = std::isfinite(S.tau_spec) && (long long)S.n_sure_above_spec < q->k;
  // An overflow is harmless when every dropped candidate's pass key lies below tau - 2 delta_f:
  // every member of the exact top-k has a pass key at or above that (k surely feasible compounds
  // reach tau), so none of them was dropped.
  bool overflow = S.overflow != 0;
  if (overflow && std::isfinite(S.tau)) {
    const unsigned u = S.dropped_bits;
    uint32_t fb = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float dropped_max;
    memcpy(&dropped_max, &fb, 4);
    if (u != 0 && (double)dropped_max < (double)S.tau - 2.0 * pass_delta_f(L, q) * 1.0001) overflow = false;
    TRACE("overflow q%lld: dropped max %g, tau %g -> %s", (long long)q->id, (double)dropped_max, (double)S.tau,
          overflow ? "rerun" : "harmless");
  }
  *spec_bad_out = spec_bad;
  *overflow_out = overflow;
  return spec_bad || overflow;
}

// Prepares the restart of a query's pass (after fin_needs_restart said so).
static void fin_restart(apex_library &L, QueryRec *q, const QuerySlot &S, bool spec_bad, bool overflow) {
  q->stats.n_restarts++;
  const double df = pass_delta_f(L, q);
  bool device_guess = false;
  if (overflow) {
    // the band above the best valid threshold did not fit: more room, and restart from the
    // largest valid threshold found (k real, surely feasible compounds reach S.tau)
    q->cap = (unsigned)std::min<unsigned long long>((unsigned long long)q->cap * 4ull, 1ull << 30);
    bind_slot(L, q);
    if (std::isfinite(S.tau) && !spec_bad) {
      q->tau_spec = S.tau;
    } else {
      q->tau_spec = -INFINITY;
      q->spec_rank = -1;
    }
  } else {
    q->spec_rank = q->spec_rank > 0 ? q->spec_rank * 8 : -1;  // the start guess was too high: lower it
    q->tau_spec = -INFINITY;
    device_guess = q->spec_rank > 0;
  }
  write_slot(L, q, std::isfinite(q->tau_spec) ? (float)(q->tau_spec - 2.0 * df * 1.0001) : -INFINITY);
  if (device_guess) speculative_start(L, q, 2.0 * df * 1.0001);
  q->remaining = q->scope_items;
  q->stats.first_item = L.cursor;
  TRACE("restart q%lld: overflow=%u spec_bad=%d cap=%u tau_spec=%g rank=%d", (long long)q->id, S.overflow,
        (int)spec_bad, q->cap, (double)S.tau_spec, q->spec_rank);
}

// Repeats a query's pass with both margins widened: by at least 2x and at least twice the largest
// observed error ratio. The start threshold is sampled again (its admission bound moved).
static void fin_restart_margin(apex_library &L, QueryRec *q) {
  const double r = std::max(q->stats.pass_err_ratio, q->stats.fp32_err_ratio);
  q->stats.n_margin_reruns++;
  q->mscale *= std::max(2.0, 2.0 * r);
  q->tau_spec = -INFINITY;
  q->spec_rank = 0;
  const double df = pass_delta_f(L, q);
  write_slot(L, q, -INFINITY);
  speculative_start(L, q, 2.0 * df * 1.0001);
  q->remaining = q->scope_items;
  q->stats.first_item = L.cursor;
  TRACE("margin rerun q%lld: ratios pass %.3f fp32 %.3f -> scale %.3f", (long long)q->id, q->stats.pass_err_ratio,
        q->stats.fp32_err_ratio, q->mscale);
}

// The chain of one query sized exactly (its count known), waited for, with further FP64 rounds
// while the boundary band still moves.
static void fin_exact(apex_library &L, QueryRec *q, unsigned nc) {
  L.arena_reserve(fin_arena_bytes(L, q, nc));
  L.dl_reserve(fin_pinned_bytes(L, q, nc));
  FinChain C;
  fin_queue(L, q, C, nc);
  CU(cudaStreamSynchronize(L.st));
  while (C.nr > 0 && C.h_cnt[2] > 0 && C.rounds < 8) {  // rare: the band moved in the last round
    fin_round(L, C);
    fin_emit(L, C);
    CU(cudaStreamSynchronize(L.st));
  }
  fin_take(L, C);
  TRACE("finalize q%lld exactly: nc %u rounds %d", (long long)q->id, nc, C.rounds);
}

// Finalizes the queries whose pass has ended (all slots in one select launch, every chain queued,
// one wait). done[i] = true when qs[i] has its rows, false when it restarts its pass.
static void finalize_batch(apex_library &L, const std::vector<QueryRec *> &qs, std::vector<char> &done) {
  const double t_f0 = now_ms();
  const size_t n = qs.size();
  done.assign(n, 0);
  if (n == 0) return;
  std::vector<unsigned> cover(n);
  size_t ab = 0, pb = 0;
  for (size_t i = 0; i < n; ++i) {
    cover[i] = fin_cover(L, qs[i]);
    ab += fin_arena_bytes(L, qs[i], cover[i]);
    pb += fin_pinned_bytes(L, qs[i], cover[i]);
  }
  // the queued chains' scratch must fit the device budget (and stay below 8 GB without one);
  // otherwise every query takes the exact path after the wait
  const bool queue = ab <= (8ull << 30) && !(L.budget && L.bytes + L.query_bytes - L.arena_cap + ab > L.budget);
  if (queue) {
    L.arena_reserve(ab);
    L.dl_reserve(pb);
  } else {
    L.dl_reserve(n * (sizeof(QuerySlot) + 64));
  }
  std::vector<int> slots(n);
  for (size_t i = 0; i < n; ++i) slots[i] = qs[i]->slot;
  L.upload(L.d_slot_list, slots.data(), sizeof(int) * n);
  CU(apx_launch_slot_select(L.d_slots, L.d_slot_list, (int)n, 1, L.st));
  tmark(L, 2);
  std::vector<FinChain> C(n);
  for (size_t i = 0; i < n; ++i) {
    C[i].hS = (QuerySlot *)L.dl_get(sizeof(QuerySlot));
    CU(cudaMemcpyAsync(C[i].hS, L.d_slots + slots[i], sizeof(QuerySlot), cudaMemcpyDeviceToHost, L.st));
  }
  if (queue)
    for (size_t i = 0; i < n; ++i) fin_queue(L, qs[i], C[i], cover[i]);
  const double t_f1 = now_ms();
  CU(cudaStreamSynchronize(L.st));
  const int last_ring = L.inflight.empty() ? -1 : L.inflight.back().ring;
  retire_all(L);  // status of the pass's launches (all complete now)
  const double t_f2 = now_ms();
  // rows first: a restart or an exact rerun below reuses the arena and the download area
  std::vector<char> redo(n, 0), sbad(n, 0), ovf(n, 0);
  std::vector<QuerySlot> Ss(n);
  std::vector<unsigned> n_r(n, 0);
  for (size_t i = 0; i < n; ++i) {
    Ss[i] = *C[i].hS;
    n_r[i] = C[i].nr > 0 ? C[i].h_cnt[0] : 0u;
    qs[i]->stats.n_candidates = Ss[i].count;
    bool sb = false, of = false;
    if (fin_needs_restart(L, qs[i], Ss[i], &sb, &of)) {
      redo[i] = 2;
      sbad[i] = sb;
      ovf[i] = of;
    } else if (!queue || Ss[i].count > C[i].cover) {
      redo[i] = 1;
    } else if (C[i].nr > 0 && C[i].h_cnt[2] > 0) {
      redo[i] = 4;  // the chain covered every candidate, but its boundary band moved in the FP64 round
    } else {
      fin_take(L, C[i]);
      if (fin_margin_exceeded(qs[i]))
        redo[i] = 3;
      else
        done[i] = 1;
    }
  }
  // Chains whose band moved get further FP64 rounds on their own data (still in the arena and the
  // download area), every such chain queued before one wait per round, until no band moves.
  for (std::vector<size_t> more;;) {
    more.clear();
    for (size_t i = 0; i < n; ++i)
      if (redo[i] == 4 && C[i].h_cnt[2] > 0 && C[i].rounds < 8) more.push_back(i);
    if (more.empty()) break;
    for (size_t i : more) {
      fin_round(L, C[i]);
      fin_emit(L, C[i]);
    }
    CU(cudaStreamSynchronize(L.st));
  }
  for (size_t i = 0; i < n; ++i)
    if (redo[i] == 4) {
      fin_take(L, C[i]);
      if (fin_margin_exceeded(qs[i]))
        redo[i] = 3;
      else
        done[i] = 1;
    }
  for (size_t i = 0; i < n; ++i) {
    if (redo[i] == 2) {
      fin_restart(L, qs[i], Ss[i], sbad[i], ovf[i]);
    } else if (redo[i] == 1) {
      fin_exact(L, qs[i], Ss[i].count);
      if (fin_margin_exceeded(qs[i]))
        fin_restart_margin(L, qs[i]);
      else
        done[i] = 1;
    } else if (redo[i] == 3) {
      fin_restart_margin(L, qs[i]);
    }
  }
  if (trace_on())
    for (size_t i = 0; i < n; ++i) {
      TRACE("finalize q%lld: nc %u nr %u rounds %d redo %d | queue %.3f, wait %.3f, rest %.3f ms", (long long)qs[i]->id,
            Ss[i].count, n_r[i], C[i].rounds, (int)redo[i], t_f1 - t_f0, t_f2 - t_f1, now_ms() - t_f2);
      if (n == 1 && last_ring >= 0)
        TRACE("gpu q%lld: start %.3f | to enum %.3f | enum %.3f | to select end %.3f | rescore32 %.3f | fp64 %.3f | "
              "emit %.3f ms",
              (long long)qs[i]->id, tspan(L, L.ev_tr[0], L.ev_tr[1]), tspan(L, L.ev_tr[1], L.ev_l0[last_ring]),
              tspan(L, L.ev_l0[last_ring], L.ev_l1[last_ring]), tspan(L, L.ev_l1[last_ring], L.ev_tr[2]),
              tspan(L, L.ev_tr[2], L.ev_tr[3]), tspan(L, L.ev_tr[3], L.ev_tr[4]), tspan(L, L.ev_tr[4], qs[i]->ev1));
    }
}

// ------------------------------------------------------------------ worker: main loop
static void finish(apex_library &L, QueryRec *q, QState st, apex_status err, const std::string &msg) {
  if (q->slot >= 0) {
    L.active[q->slot] = nullptr;
    q->slot = -1;
  }
  free_query_device(L, q);
  q->state = st;
  q->err = err;
  q->err_msg = msg;
  q->t_done = now_ms();
  q->stats.queue_ms = q->t_admit > 0 ? q->t_admit - q->t_submit : 0;
  q->stats.latency_ms = q->t_done - q->t_submit;
  q->stats.n_scope = q->scope_n;
  L.done_seq++;
}

// Scratch of one compaction of query q (256-byte roundings in the slack).
static size_t compact_bytes(const apex_library &L, const QueryRec *q) {
  const size_t cover = q->cap, no = L.n_out, m = q->cidx.size();
  return sizeof(float) * cover * (no + 1) + 2 * cover + 12 * cover + 16 * (m + 1) + 10 * 256;
}
// The compactions of queries qs (every one's scratch in the arena at once): per query the split,
// the rescore and the decisions; one launch selects every query's threshold (a CTA each); then
// per query the keep and apply steps.
static void compact_group(apex_library &L, const std::vector<QueryRec *> &qs) {
  const int no = L.n_out;
  size_t need = sizeof(KthJob) * qs.size() + 256;
  for (QueryRec *q : qs) need += compact_bytes(L, q);
  L.arena_reserve(need);
  struct Tail {
    float *f32;
    unsigned char *maybe, *sure;
    float *d_tau;
    int *d_ok;
    unsigned *kept;
    double ecf;
  };
  std::vector<Tail> tails(qs.size());
  std::vector<KthJob> jobs(qs.size());
  for (size_t i = 0; i < qs.size(); ++i) {
    QueryRec *q = qs[i];
    const int m = (int)q->cidx.size();
    const unsigned cover = q->cap;
    float *out32 = (float *)L.aget(sizeof(float) * (size_t)cover * no);
    float *f32 = (float *)L.aget(sizeof(float) * cover);
    unsigned char *maybe = (unsigned char *)L.aget(cover);
    unsigned char *sure = (unsigned char *)L.aget(cover);
    long long *ids_new = (long long *)L.aget(sizeof(long long) * cover);
    int *pos_new = (int *)L.aget(sizeof(int) * cover);
    unsigned *n_new = (unsigned *)L.aget(sizeof(unsigned));
    double *dlo = (double *)L.aget(sizeof(double) * std::max(m, 1));
    double *dhi = (double *)L.aget(sizeof(double) * std::max(m, 1));
    float *d_tau = (float *)L.aget(sizeof(float));
    int *d_ok = (int *)L.aget(sizeof(int));
    unsigned *kept = (unsigned *)L.aget(sizeof(unsigned));
    if (m > 0) {
      L.upload(dlo, q->lo.data(), sizeof(double) * m);
      L.upload(dhi, q->hi.data(), sizeof(double) * m);
    }
    CU(apx_launch_split_scored(L.d_slots + q->slot, cover, f32, maybe, sure, ids_new, pos_new, n_new, L.n_sm, L.st));
    const bool f16 = compact_fp16(L, q);
    if (f16) {
      CU(apx_launch_tc_ids(L.T_, ids_new, cover, out32, L.d_err, L.n_sm, L.st, 1, nullptr, -1, n_new));
    } else {
      LaunchPlan dummy;
      memset(&dummy, 0, sizeof(dummy));
      CU(apx_launch_fp32(dummy, L.T_, nullptr, ids_new, cover, out32, grid_for(L, (cover + APX_TILE - 1) / APX_TILE),
                         L.st, L.fp32_id_tile.load(), n_new));
    }
    const double ecf = compact_delta_f(L, q);  // the rescore's objective margin
    EvalArgs ea{out32, no, L.d_slots + q->slot, f16 ? L.d_err16f : L.d_err32f, (float)ecf, dlo, dhi};
    ea.eps_scale = (float)q->mscale;
    ea.pass_keys = q->keys;
    ea.obs = slot_obs(L, q->slot);
    ea.pos = pos_new;
    CU(apx_launch_eval32(ea, cover, f32, maybe, sure, L.st, n_new));
    jobs[i] = KthJob{f32, sure, (long long)cover, q->k, d_tau, d_ok, &L.d_slots[q->slot].count};
    tails[i] = Tail{f32, maybe, sure, d_tau, d_ok, kept, ecf};
  }
  KthJob *d_jobs = (KthJob *)L.aget(sizeof(KthJob) * qs.size());
  L.upload(d_jobs, jobs.data(), sizeof(KthJob) * qs.size());
  CU(apx_launch_kth_multi(d_jobs, (int)qs.size(), L.st));
  for (size_t i = 0; i < qs.size(); ++i) {
    QueryRec *q = qs[i];
    const Tail &t = tails[i];
    CU(apx_launch_compact(L.d_slots + q->slot, t.f32, t.maybe, t.sure, t.d_tau, t.d_ok, (float)(2.0 * t.ecf * 1.0001),
                          (float)(t.ecf * 1.0001), t.kept, q->cap, L.n_sm, L.st));
    q->want_compact = false;
    q->stats.n_compactions++;
  }
}
// In-pass compaction of the candidate buffers of queries qs (queued behind the select that
// follows an enumeration launch; no host wait): the rescore (FP16 on the tensor cores or FP32) of
// the entries appended since each query's last compaction (the ones it kept already carry their
// rescored objective), their decisions and the k-th sure objective, then each buffer keeps only
// what can still reach the top-k and its admission threshold rises to the certified floor
// (k_compact_keep / k_compact_apply). Queries are grouped so that a group's scratch fits the
// arena limit (below).
static void compact_queries(apex_library &L, const std::vector<QueryRec *> &qs) {
  // without a budget: a quarter of the device, at most 48 GB and at least 8 GB (an FP8 pass over
  // a large scope holds 2^26-entry buffers, ~4.7 GB of compaction scratch per query)
  const size_t unbudgeted = std::max<size_t>(8ull << 30, std::min<size_t>(48ull << 30, L.dev_total / 4));
  const size_t cap = L.budget ? std::min<size_t>(8ull << 30, std::max<size_t>(L.arena_cap, 64ull << 20)) : unbudgeted;
  std::vector<QueryRec *> group;
  size_t bytes = 0;
  for (QueryRec *q : qs) {
    const size_t b = compact_bytes(L, q) + sizeof(KthJob) + 256;
    if (!group.empty() && bytes + b > cap) {
      compact_group(L, group);
      group.clear();
      bytes = 0;
    }
    group.push_back(q);
    bytes += b;
  }
  if (!group.empty()) compact_group(L, group);
}

// One step of the circular pass: a launch over the next chunk of items needed by any active
// query (per precision), then the conditional select of the served queries.
static void pass_step(apex_library &L) {
  const double t_p0 = trace_on() ? now_ms() : 0.0;
  // compactions wanted by the launch retired last: queued before this step's launch, so they run
  // right behind the select of the launch still in flight (one launch of lag)
  {
    std::vector<QueryRec *> cq;
    for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
      if (L.active[s] && L.active[s]->want_compact && L.active[s]->remaining > 0) cq.push_back(L.active[s]);
    if (!cq.empty()) compact_queries(L, cq);
  }
  // a linear head costs ~100x less per compound than the MLP: larger launches. A query's first
  // launches serve it few compounds, 4x more per launch (2^24, 2^26, ...): its admission threshold
  // is only a sampled guess until the select after a launch raises it, and a large first launch at
  // a loose threshold would overflow its candidate buffer. The launch ends where a query it serves
  // reaches that bound; queries it does not serve (other reactions) do not shorten it.
  const long long chunk_compounds = L.chunk_compounds.load() << (L.n_layers == 1 ? 8 : 0);
  long long ramp[APEX_MAX_ACTIVE];
  for (int s = 0; s < APEX_MAX_ACTIVE; ++s) {
    const int f = L.active[s] ? L.active[s]->stats.n_launches : 1 << 20;
    ramp[s] = f < 10 ? std::min(chunk_compounds, 1LL << (24 + 2 * f)) : chunk_compounds;
  }
  std::vector<long long> served_c(APEX_MAX_ACTIVE, 0);  // compounds this launch serves each query
  // build one plan (items from the cursor) with per-precision query masks
  // indexed by pass precision (APEX_FP32, APEX_BF16, APEX_FP16, APEX_FP8; 2 unused)
  PlanBuilder pb[5] = {PlanBuilder(L.rx), PlanBuilder(L.rx), PlanBuilder(L.rx), PlanBuilder(L.rx), PlanBuilder(L.rx)};
  long long served_compounds = 0;
  long long cur = L.cursor;
  long long visited = 0;
  std::vector<long long> served(APEX_MAX_ACTIVE, 0);
  while (visited < L.total_items && served_compounds < chunk_compounds) {
    const int t = (int)(std::upper_bound(L.item_first.begin(), L.item_first.end(), cur) - L.item_first.begin()) - 1;
    const long long b = cur - L.item_first[t];
    const long long e = L.rx[t].n_items;
    // a query is served only the items it still lacks: its unvisited items are exactly the next
    // `remaining` items of its reactions in circular order from the cursor, so a segment never
    // reaches past the end of its cycle (no compound is enumerated twice for it)
    unsigned long long mask[5] = {0, 0, 0, 0, 0};
    long long lack = LLONG_MAX;
    for (int s = 0; s < APEX_MAX_ACTIVE; ++s) {
      QueryRec *q = L.active[s];
      if (q && q->remaining > served[s] && q->need[t]) {
        mask[q->precision] |= 1ull << s;
        lack = std::min(lack, q->remaining - served[s]);
      }
    }
    long long take = e - b;
    const unsigned long long any = mask[0] | mask[1] | mask[3] | mask[4];
    bool ramp_full = false;  // a query served here reached its first-launch bound
    if (any) {
      const long long per_item = (long long)L.rx[t].L_o * APX_TILE;
      long long left = chunk_compounds - served_compounds;
      for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
        if (any >> s & 1ull) left = std::min(left, ramp[s] - served_c[s]);
      const long long room = std::max<long long>(1, (left + per_item - 1) / per_item);
      take = std::min(std::min(take, room), lack);
      bool ok = true;
      for (int p = 0; p < 5; ++p)
        if (mask[p] && pb[p].P.n_seg >= APX_MAX_SEG) ok = false;
      if (!ok) break;
      for (int p = 0; p < 5; ++p)
        if (mask[p]) pb[p].add(t, b, b + take, mask[p]);
      for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
        if (any >> s & 1ull) {
          served[s] += take;
          served_c[s] += take * per_item;
          ramp_full = ramp_full || served_c[s] >= ramp[s];
        }
      served_compounds += take * per_item;
    }
    visited += take;
    cur += take;
    if (cur >= L.total_items) cur = 0;
    if (ramp_full) break;
  }
  L.cursor = cur;
  std::vector<int> list;
  for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
    if (served[s] > 0) list.push_back(s);
  for (int s : list) {
    QueryRec *q = L.active[s];
    if (q->stats.n_launches == 0 && q->stats.n_restarts == 0) CU(cudaEventRecord(q->ev0, L.st));
  }
  const int ring = (int)(L.launch_seq++ % apex_library::kRing);
  const double t_p1 = trace_on() ? now_ms() : 0.0;
  CU(cudaEventRecord(L.ev_l0[ring], L.st));
  for (int p = 0; p < 5; ++p) launch_enum(L, pb[p].P, p);
  CU(cudaEventRecord(L.ev_l1[ring], L.st));
  TRACE("pass step: plan %.3f ms, launch %.3f ms", t_p1 - t_p0, now_ms() - t_p1);
  // select between launches only for queries with work left (a finished pass is selected by
  // its finalization right after)
  std::vector<int> cont;
  for (int s : list)
    if (L.active[s]->remaining > served[s]) cont.push_back(s);
  if (!cont.empty()) {
    L.upload(L.d_slot_list, cont.data(), sizeof(int) * cont.size());
    CU(apx_launch_slot_select(L.d_slots, L.d_slot_list, (int)cont.size(), 0, L.st));
    // every slot's (count, count_compacted) after the select, for the compaction trigger
    CU(cudaMemcpy2DAsync(L.cnt_pin + (size_t)ring * 2 * APEX_MAX_ACTIVE, 2 * sizeof(unsigned), &L.d_slots[0].count,
                         sizeof(QuerySlot), 2 * sizeof(unsigned), APEX_MAX_ACTIVE, cudaMemcpyDeviceToHost, L.st));
  }
  // the kernel status word of this launch, read back without waiting for it
  CU(cudaMemcpyAsync(L.status_pin + ring, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, L.st));
  CU(cudaEventRecord(L.ev_ls[ring], L.st));
  apex_library::InFlight f;
  f.ring = ring;
  for (int s : list) f.queries.emplace_back(s, L.active[s]->id);
  L.inflight.push_back(std::move(f));
  {
    long long launched = 0;
    for (int p = 0; p < 5; ++p)
      for (int g = 0; g < pb[p].P.n_seg; ++g) {
        const Segment &sg = pb[p].P.seg[g];
        launched += items_compounds(L.rx[sg.rxn], sg.item_begin, sg.item_end);
      }
    L.head_evals += launched;
  }
  for (int s : list) {
    QueryRec *q = L.active[s];
    q->remaining -= served[s];
    q->stats.n_launches++;
    long long comp = 0;
    for (int p = 0; p < 5; ++p)
      for (int g = 0; g < pb[p].P.n_seg; ++g)
        if (pb[p].P.seg[g].qmask >> s & 1ull) {
          const Segment &sg = pb[p].P.seg[g];
          comp += items_compounds(L.rx[sg.rxn], sg.item_begin, sg.item_end);
        }
    q->stats.n_scored += comp;
  }
  while (L.inflight.size() > 1) retire_launch(L);  // the GPU keeps this launch queued
}

// The CPU the worker runs on. On the hosts this library was measured on, CUDA calls issued from
// the CPU that created the device context cost about a third of what they cost from any other CPU
// (kernel launch ~3.5 us against ~9-10 us), and a query's host path issues a few dozen of them.
// With APEX_WORKER_CPU=auto the worker times a burst of event records from every allowed CPU and
// stays on the fastest one when it is clearly faster than the typical one; APEX_WORKER_CPU=n pins
// it to CPU n. By default it is not pinned: pinned, it shares its CPU with whatever application
// thread the scheduler puts there, and on the measured hosts the mean query time gained about 1 %
// while the tail grew.
static int pick_worker_cpu(apex_library &L) {
  const char *e = getenv("APEX_WORKER_CPU");
  if (!e) return -1;
  if (strcmp(e, "auto") != 0) return atoi(e);
  cpu_set_t allowed;
  if (sched_getaffinity(0, sizeof(allowed), &allowed) != 0) return -1;
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return -1;
  std::vector<std::pair<double, int>> t;
  for (int c = 0; c < CPU_SETSIZE && c < 256; ++c) {
    if (!CPU_ISSET(c, &allowed)) continue;
    cpu_set_t one;
    CPU_ZERO(&one);
    CPU_SET(c, &one);
    if (pthread_setaffinity_np(pthread_self(), sizeof(one), &one) != 0) continue;
    double best = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
      cudaStreamSynchronize(L.st);
      const double t0 = now_ms();
      for (int j = 0; j < 8; ++j) cudaEventRecord(ev, L.st);
      best = std::min(best, now_ms() - t0);
    }
    t.emplace_back(best, c);
  }
  cudaStreamSynchronize(L.st);
  cudaEventDestroy(ev);
  pthread_setaffinity_np(pthread_self(), sizeof(allowed), &allowed);
  if (t.size() < 2) return -1;
  std::sort(t.begin(), t.end());
  const double median = t[t.size() / 2].first;
  TRACE("worker cpu probe: fastest cpus %d %.2f, %d %.2f us/call, median %.2f us/call", t[0].second,
        1e3 * t[0].first / 8, t[1].second, 1e3 * t[1].first / 8, 1e3 * median / 8);
  return t[0].first < 0.6 * median ? t[0].second : -1;
}

static void worker_main(apex_library *Lp) {
  apex_library &L = *Lp;
  cudaSetDevice(L.device);
  int cpu = pick_worker_cpu(L);
  if (cpu >= 0 && cpu < CPU_SETSIZE) {
    cpu_set_t one;
    CPU_ZERO(&one);
    CPU_SET(cpu, &one);
    if (pthread_setaffinity_np(pthread_self(), sizeof(one), &one) != 0) cpu = -1;
  } else {
    cpu = -1;
  }
  L.worker_cpu.store(cpu);
  for (;;) {
    std::vector<QueryRec *> fresh;
    {
      std::unique_lock<std::mutex> lk(L.mu);
      if (L.stop) break;
      // cancellations
      for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
        if (L.active[s] && L.active[s]->cancel) {
          finish(L, L.active[s], Q_CANCELED, APEX_ECANCELED, "cancelled");
          L.cv_done.notify_all();
        }
      for (auto it = L.queued.begin(); it != L.queued.end();) {
        if ((*it)->cancel) {
          finish(L, *it, Q_CANCELED, APEX_ECANCELED, "cancelled");
          it = L.queued.erase(it);
          L.cv_done.notify_all();
        } else {
          ++it;
        }
      }
      // admission (FIFO while slots and memory allow)
      try {
        while (!L.queued.empty()) {
          QueryRec *q = L.queued.front();
          if (!admit_one(L, q)) {
            bool none_active = true;
            for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
              if (L.active[s]) none_active = false;
            if (none_active) {  // cannot fit even alone
              L.queued.pop_front();
              finish(L, q, Q_FAILED, APEX_ENOMEM, "candidate state exceeds the device memory budget");
              L.cv_done.notify_all();
              continue;
            }
            break;
          }
          L.queued.pop_front();
          fresh.push_back(q);
        }
      } catch (const CudaFail &f) {
        QueryRec *q = L.queued.front();
        L.queued.pop_front();
        finish(L, q, Q_FAILED, APEX_ENOMEM, std::string("admission: ") + cudaGetErrorString(f.e));
        L.cv_done.notify_all();
      }
      bool any = false;
      for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
        if (L.active[s]) any = true;
      if (!any) {
        retire_quietly(L);
        const unsigned long long seq = L.work_seq.load();
        lk.unlock();
        const bool moved = worker_spin_ms() > 0 && watch(L.work_seq, seq, worker_spin_ms(), 63);
        lock_spin(lk);
        if (!moved && L.work_seq.load() == seq) L.cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
    }
    try {
      for (QueryRec *q : fresh) {
        const double t0 = now_ms();
        start_query(L, q);
        q->stats.host_start_ms += now_ms() - t0;
      }
      {
        const double t0 = now_ms();
        pass_step(L);
        const double dt = now_ms() - t0;
        for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
          if (L.active[s]) L.active[s]->stats.host_pass_ms += dt;
      }
      std::vector<QueryRec *> ended;
      for (int s = 0; s < APEX_MAX_ACTIVE; ++s) {
        QueryRec *q = L.active[s];
        if (!q || q->remaining > 0) continue;
        {
          std::lock_guard<std::mutex> g(L.mu);
          if (q->cancel) {  // cancelled while its pass ran: skip the finalization
            finish(L, q, Q_CANCELED, APEX_ECANCELED, "cancelled");
            L.cv_done.notify_all();
            continue;
          }
        }
        ended.push_back(q);
      }
      if (!ended.empty()) {
        const double t0 = now_ms();
        std::vector<char> done;
        finalize_batch(L, ended, done);
        const double dt = now_ms() - t0;
        std::lock_guard<std::mutex> g(L.mu);
        for (size_t i = 0; i < ended.size(); ++i) {
          QueryRec *q = ended[i];
          q->stats.host_finalize_ms += dt;
          if (!done[i]) continue;
          float ms = 0;
          if (cudaEventElapsedTime(&ms, q->ev0, q->ev1) == cudaSuccess) q->stats.gpu_ms = ms;
          finish(L, q, Q_DONE, APEX_OK, "");
        }
        L.cv_done.notify_all();
      }
    } catch (const CudaFail &f) {
      L.inflight.clear();
      cudaStreamSynchronize(L.st);
      std::lock_guard<std::mutex> g(L.mu);
      const apex_status code = (f.e == cudaErrorLaunchTimeout) ? APEX_ETIMEDOUT : APEX_ECUDA;
      char buf[256];
      snprintf(buf, sizeof(buf), "%s failed: %s (line %d)", f.what, cudaGetErrorString(f.e), f.line);
      for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
        if (L.active[s]) finish(L, L.active[s], Q_FAILED, code, buf);
      L.cv_done.notify_all();
    }
  }
  // shutdown: everything still pending is cancelled
  retire_quietly(L);
  std::lock_guard<std::mutex> g(L.mu);
  for (int s = 0; s < APEX_MAX_ACTIVE; ++s)
    if (L.active[s]) finish(L, L.active[s], Q_CANCELED, APEX_ECANCELED, "library freed");
  for (QueryRec *q : L.queued) finish(L, q, Q_CANCELED, APEX_ECANCELED, "library freed");
  L.queued.clear();
  L.cv_done.notify_all();
}

// ------------------------------------------------------------------ fetch / stats
extern "C" apex_status apex_topk_fetch(apex_library *L, apex_query_id id, int64_t capacity, int64_t *ids,
                                       int32_t *reaction, int64_t *synthons, double *objective, double *outputs,
                                       int64_t *n_out, int32_t timeout_ms) {
  if (!L) return fail(APEX_EINVAL, "NULL library");
  if (capacity < 0) return fail(APEX_EINVAL, "negative capacity");
  std::unique_lock<std::mutex> lk(L->mu, std::defer_lock);
  lock_spin(lk);
  // Every wait below releases L->mu, and another fetcher of the same id may finish meanwhile and
  // release the record (queries.erase frees it). So the record is looked up again under the lock
  // after each wait, and the wait predicate itself looks it up instead of holding a pointer: a
  // query whose record is gone was taken by that other fetcher and is reported as not found.
  auto it = L->queries.find(id);
  if (it == L->queries.end()) return fail(APEX_ENOTFOUND, "query %lld not found", (long long)id);
  auto finished = [](const QueryRec *r) {
    return r->state == Q_DONE || r->state == Q_CANCELED || r->state == Q_FAILED;
  };
  auto gone_or_done = [&] {
    auto f = L->queries.find(id);
    return f == L->queries.end() || finished(f->second.get());
  };
  // watch for completions first (no sleep), for at most fetch_spin_ms() or the timeout
  const double t_w0 = now_ms();
  const double spin_ms = timeout_ms < 0 ? fetch_spin_ms() : std::min(fetch_spin_ms(), (double)timeout_ms);
  while (!gone_or_done() && L->spinners < 2) {
    const double left = spin_ms - (now_ms() - t_w0);
    if (left <= 0) break;
    const unsigned long long seq = L->done_seq.load();
    L->spinners++;
    lk.unlock();
    watch(L->done_seq, seq, left, 63);
    lock_spin(lk);
    L->spinners--;
  }
  if (timeout_ms < 0) {
    L->cv_done.wait(lk, gone_or_done);
  } else {
    const double left_ms = std::max(0.0, timeout_ms - (now_ms() - t_w0));
    if (!L->cv_done.wait_for(lk, std::chrono::microseconds((long long)(1000.0 * left_ms)), gone_or_done))
      return fail(APEX_EAGAIN, "query %lld not finished", (long long)id);
  }
  it = L->queries.find(id);
  if (it == L->queries.end()) return fail(APEX_ENOTFOUND, "query %lld not found (fetched by another caller)", (long long)id);
  QueryRec *q = it->second.get();
  apex_status rc = q->err;
  {
    apex_library::Served &V = L->served;
    if (q->state == Q_DONE) {
      if (V.lat.size() < APEX_STATS_WINDOW) {
        V.lat.push_back(q->stats.latency_ms);
        V.queue.push_back(q->stats.queue_ms);
      } else {
        V.lat[V.next] = q->stats.latency_ms;
        V.queue[V.next] = q->stats.queue_ms;
        V.next = (V.next + 1) % APEX_STATS_WINDOW;
      }
      V.t_first = V.n_ok == 0 ? q->t_submit : std::min(V.t_first, q->t_submit);
      V.t_last = V.n_ok == 0 ? q->t_done : std::max(V.t_last, q->t_done);
      V.n_ok++;
      V.query_compounds += (double)q->scope_n;
      V.lat_sum += q->stats.latency_ms;
      V.lat_max = std::max(V.lat_max, q->stats.latency_ms);
    } else {
      V.n_failed++;
    }
  }
  if (q->state == Q_DONE) {
    const long long n = (long long)q->r_ids.size();
    const long long c = std::min<long long>(n, capacity);
    if (ids) memcpy(ids, q->r_ids.data(), sizeof(int64_t) * c);
    if (reaction) memcpy(reaction, q->r_rxn.data(), sizeof(int32_t) * c);
    if (synthons) memcpy(synthons, q->r_syn.data(), sizeof(int64_t) * c * APEX_MAX_SLOTS);
    if (objective) memcpy(objective, q->r_obj.data(), sizeof(double) * c);
    if (outputs) memcpy(outputs, q->r_out.data(), sizeof(double) * c * L->n_out);
    if (n_out) *n_out = n;
  } else {
    if (n_out) *n_out = 0;
    fail(rc, "query %lld: %s", (long long)id, q->err_msg.c_str());
  }
  if (q->ev0 && q->ev1 && L->ev_pool.size() < 256) {
    L->ev_pool.emplace_back(q->ev0, q->ev1);
  } else {
    if (q->ev0) cudaEventDestroy(q->ev0);
    if (q->ev1) cudaEventDestroy(q->ev1);
  }
  L->last_stats = q->stats;
  L->queries.erase(it);
  return rc;
}

extern "C" apex_status apex_query_stats(apex_library *L, apex_query_id id, apex_query_stats_t *out) {
  if (!L || !out) return fail(APEX_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(L->mu);
  if (id < 0) {
    *out = L->last_stats;
    return APEX_OK;
  }
  auto it = L->queries.find(id);
  if (it == L->queries.end()) return fail(APEX_ENOTFOUND, "query %lld not found", (long long)id);
  *out = it->second->stats;
  return APEX_OK;
}

// percentile p (0..100) of v by linear interpolation between the nearest ranks (v is sorted here)
static double pct_linear(std::vector<double> &v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double r = p / 100.0 * (double)(v.size() - 1);
  const size_t i = (size_t)std::floor(r);
  const size_t j = std::min(i + 1, v.size() - 1);
  return v[i] + (r - (double)i) * (v[j] - v[i]);
}

extern "C" apex_status apex_stats(apex_library *L, apex_stats_t *out) {
  if (!L || !out) return fail(APEX_EINVAL, "NULL argument");
  memset(out, 0, sizeof(*out));
  std::vector<double> lat, queue;
  {
    std::lock_guard<std::mutex> g(L->mu);
    const apex_library::Served &V = L->served;
    lat = V.lat;
    queue = V.queue;
    out->n_queries = V.n_ok;
    out->n_failed = V.n_failed;
    out->max_ms = V.lat_max;
    out->mean_ms = V.n_ok > 0 ? V.lat_sum / (double)V.n_ok : 0.0;
    out->wall_ms = V.n_ok > 0 ? V.t_last - V.t_first : 0.0;
    out->query_compounds = V.query_compounds;
    out->head_evaluations = (double)(L->head_evals.load() - V.evals_at_reset);
    out->enumerate_ms = 1e-6 * (double)(L->enum_ns.load() - V.enum_ns_at_reset);
    out->n_enumeration_launches = L->enum_launches.load() - V.launches_at_reset;
  }
  out->p50_ms = pct_linear(lat, 50.0);
  out->p99_ms = pct_linear(lat, 99.0);
  out->queue_p50_ms = pct_linear(queue, 50.0);
  out->queue_p99_ms = pct_linear(queue, 99.0);
  if (out->wall_ms > 0) {
    out->query_compounds_per_s = out->query_compounds / (out->wall_ms * 1e-3);
    out->head_evaluations_per_s = out->head_evaluations / (out->wall_ms * 1e-3);
  }
  return APEX_OK;
}

extern "C" apex_status apex_stats_reset(apex_library *L) {
  if (!L) return fail(APEX_EINVAL, "NULL library");
  std::lock_guard<std::mutex> g(L->mu);
  L->served = apex_library::Served();
  L->served.evals_at_reset = L->head_evals.load();
  L->served.enum_ns_at_reset = L->enum_ns.load();
  L->served.launches_at_reset = L->enum_launches.load();
  return APEX_OK;
}

// ------------------------------------------------------------------ direct scoring (tests)
extern "C" apex_status apex_score_ids(apex_library *L, int32_t precision, int64_t n, const int64_t *ids,
                                      double *outputs) {
  if (!L || n < 0 || (n > 0 && (!ids || !outputs))) return fail(APEX_EINVAL, "bad arguments");
  const int fmt = tc_format(precision);
  if (precision != APEX_FP32 && precision != APEX_FP64 && fmt < 0) return fail(APEX_EINVAL, "unknown precision");
  if (fmt >= 0 && !((L->precisions >> precision) & 1u)) return fail(APEX_EUNSUPPORTED, "precision not built");
  for (int64_t i = 0; i < n; ++i)
    if (ids[i] < 0 || ids[i] >= L->N) return fail(APEX_EINVAL, "id %lld out of range", (long long)ids[i]);
  if (n == 0) return APEX_OK;
  std::lock_guard<std::mutex> g(L->mu);  // keeps the worker from interleaving on the stream
  const int no = L->n_out;
  try {
    CU(cudaSetDevice(L->device));
    DevBuf B;
    long long *d_ids = (long long *)B.get(sizeof(long long) * n);
    CU(cudaMemcpyAsync(d_ids, ids, sizeof(long long) * n, cudaMemcpyHostToDevice, L->st));
    if (precision != APEX_FP64) {
      float *d = (float *)B.get(sizeof(float) * n * no);
      if (fmt >= 0) {  // the tensor-core kernel over the id list (the start-threshold sample's path)
        CU(apx_launch_tc_ids(L->T_, d_ids, n, d, L->d_err, L->n_sm, L->st, fmt, nullptr, -1));
        check_kernel_status(*L);
      } else {
        LaunchPlan dummy;
        memset(&dummy, 0, sizeof(dummy));
        CU(apx_launch_fp32(dummy, L->T_, nullptr, d_ids, n, d, grid_for(*L, (n + APX_TILE - 1) / APX_TILE), L->st));
      }
      std::vector<float> h(n * no);
      CU(cudaMemcpyAsync(h.data(), d, sizeof(float) * n * no, cudaMemcpyDeviceToHost, L->st));
      CU(cudaStreamSynchronize(L->st));
      for (long long i = 0; i < n * no; ++i) outputs[i] = h[i];
    } else {
      double *d = (double *)B.get(sizeof(double) * n * no);
      CU(apx_launch_fp64(L->T_, d_ids, n, d, L->st));
      CU(cudaMemcpyAsync(outputs, d, sizeof(double) * n * no, cudaMemcpyDeviceToHost, L->st));
      CU(cudaStreamSynchronize(L->st));
    }
  } catch (const CudaFail &f) {
    return fail(APEX_ECUDA, "score_ids: %s failed: %s", f.what, cudaGetErrorString(f.e));
  }
  return APEX_OK;
}

extern "C" apex_status apex_dump_outputs(apex_library *L, int32_t precision, int32_t reaction, float *outputs,
                                         int64_t capacity) {
  if (!L || !outputs || reaction < -1 || reaction >= L->T) return fail(APEX_EINVAL, "bad arguments");
  if (precision != APEX_FP32 && precision != APEX_BF16 && precision != APEX_FP16 && precision != APEX_FP8)
    return fail(APEX_EINVAL, "unknown precision");
  if (!((L->precisions >> precision) & 1u)) return fail(APEX_EUNSUPPORTED, "precision not built");
  const int t0 = reaction < 0 ? 0 : reaction, t1 = reaction < 0 ? L->T : reaction + 1;
  const long long nt = L->id_first[t1] - L->id_first[t0];
  if (capacity < nt) return fail(APEX_EINVAL, "capacity %lld < %lld compounds", (long long)capacity, nt);
  const int no = L->n_out;
  if ((double)nt * no * sizeof(float) > (double)(16ull << 30))
    return fail(APEX_EINVAL, "dump of %lld compounds exceeds 16 GB of outputs", nt);
  std::lock_guard<std::mutex> g(L->mu);
  try {
    CU(cudaSetDevice(L->device));
    DevBuf B;
    float *d = (float *)B.get(sizeof(float) * nt * no);
    // launches shaped like those of a query's pass: consecutive items in library order, about the
    // library's compounds-per-launch each, cost-weighted CTA ranges (launch_enum)
    const long long chunk = reaction < 0 ? L->chunk_compounds.load() : (1LL << 62);
    PlanBuilder pb(L->rx);
    long long in_plan = 0;
    auto flush = [&] {
      if (pb.P.n_seg == 0) return;
      LaunchPlan P = pb.P;
      P.mode = 1;
      P.dump = d;
      P.dump_base = L->id_first[t0];
      P.dump_n = nt;
      launch_enum(*L, P, precision);
      check_kernel_status(*L);
      pb = PlanBuilder(L->rx);
      in_plan = 0;
    };
    for (int t = t0; t < t1; ++t) {
      const long long items = L->rx[t].n_items, per_item = (long long)L->rx[t].L_o * APX_TILE;
      long long b = 0;
      while (b < items) {
        const long long room = std::max<long long>(1, (chunk - in_plan + per_item - 1) / per_item);
        const long long e = std::min(items, b + std::min<long long>(room, 1LL << 30));
        if (!pb.add(t, b, e, 0)) {
          flush();
          continue;
        }
        in_plan += (e - b) * per_item;
        b = e;
        if (in_plan >= chunk) flush();
      }
    }
    flush();
    CU(cudaMemcpy(outputs, d, sizeof(float) * nt * no, cudaMemcpyDeviceToHost));
  } catch (const CudaFail &f) {
    return fail(f.e == cudaErrorLaunchTimeout ? APEX_ETIMEDOUT : APEX_ECUDA, "dump: %s failed: %s", f.what,
                cudaGetErrorString(f.e));
  }
  return APEX_OK;
}

extern "C" apex_status apex_selftest_wait_timeout(apex_library *L, int32_t limit_ms) {
  if (!L) return fail(APEX_EINVAL, "NULL library");
  if (limit_ms < 1 || limit_ms > 2000) return fail(APEX_EINVAL, "limit_ms = %d outside 1..2000", limit_ms);
  std::lock_guard<std::mutex> g(L->mu);
  int code = 0;
  try {
    CU(cudaSetDevice(L->device));
    DevBuf B;
    int *d_err = (int *)B.get(sizeof(int));  // a status word of its own: queries never see this one
    CU(cudaMemsetAsync(d_err, 0, sizeof(int), L->st));
    CU(apx_launch_wait_selftest(d_err, (unsigned long long)limit_ms * 1000000ull, L->st));
    CU(cudaMemcpyAsync(&code, d_err, sizeof(int), cudaMemcpyDeviceToHost, L->st));  // pageable: complete after the sync
    CU(cudaStreamSynchronize(L->st));
  } catch (const CudaFail &f) {
    return fail(APEX_ECUDA, "wait self-test: %s failed: %s", f.what, cudaGetErrorString(f.e));
  }
  if (code == APX_ERR_TIMEOUT) return fail(APEX_ETIMEDOUT, "device wait gave up after %d ms (expected)", limit_ms);
  return fail(APEX_ECUDA, "wait self-test: the wait returned without timing out (status %d)", code);
}

// ------------------------------------------------------------------ autotuner
// Trial queries shaped like the workload's: seeded convex weights over the objectives, two boxes
// of +-1 RMS around 0 on seeded properties, the caller's k, precision and reaction subset.
static std::vector<apex_query_id> autotune_trials(apex_library *L, const apex_autotune_desc *d, std::mt19937_64 &g,
                                                  apex_status *rc) {
  std::vector<apex_query_id> ids;
  std::uniform_real_distribution<double> U(0.0, 1.0);
  for (int i = 0; i < d->n_queries; ++i) {
    float w[APEX_MAX_OBJECTIVES] = {0};
    double sw = 0;
    for (int j = 0; j < L->n_obj; ++j) sw += (w[j] = (float)(-std::log(1.0 - U(g))));
    for (int j = 0; j < L->n_obj; ++j) w[j] = (float)(w[j] / sw);
    int32_t idx[2];
    double lo[2], hi[2];
    const int m = L->n_prop > 0 ? 2 : 0;
    for (int c = 0; c < m; ++c) {
      idx[c] = L->n_obj + (int)(g() % (unsigned long long)L->n_prop);
      lo[c] = -L->rms[idx[c]];
      hi[c] = L->rms[idx[c]];
    }
    apex_query_desc q{};
    q.precision = d->precision;
    q.objective_weights = w;
    q.n_constraints = m;
    q.output_index = idx;
    q.lower = lo;
    q.upper = hi;
    q.k = d->k;
    q.n_reaction_subset = d->n_reaction_subset;
    q.reactions = d->reactions;
    apex_query_id id = 0;
    *rc = apex_query(L, &q, &id);
    if (*rc != APEX_OK) return ids;
    ids.push_back(id);
  }
  return ids;
}

static double autotune_run(apex_library *L, const apex_autotune_desc *d, uint64_t seed, apex_status *rc) {
  std::mt19937_64 g(seed);
  const double t0 = now_ms();
  std::vector<apex_query_id> ids = autotune_trials(L, d, g, rc);
  for (apex_query_id id : ids) {
    int64_t n = 0;
    const apex_status r = apex_topk_fetch(L, id, 0, nullptr, nullptr, nullptr, nullptr, nullptr, &n, -1);
    if (r != APEX_OK && *rc == APEX_OK) *rc = r;
  }
  return now_ms() - t0;
}

extern "C" apex_status apex_set_launch_shape(apex_library *L, int64_t chunk_compounds, int32_t fp32_id_tile) {
  if (!L) return fail(APEX_EINVAL, "NULL library");
  if (chunk_compounds < APX_TILE) return fail(APEX_EINVAL, "chunk_compounds %lld < %d", (long long)chunk_compounds, APX_TILE);
  if (fp32_id_tile != 32 && fp32_id_tile != 128) return fail(APEX_EINVAL, "fp32_id_tile must be 32 or 128");
  L->chunk_compounds.store(chunk_compounds);
  L->fp32_id_tile.store(fp32_id_tile);
  return APEX_OK;
}

extern "C" apex_status apex_autotune(apex_library *L, const apex_autotune_desc *d, apex_autotune_result_t *out) {
  if (!L || !d || !out) return fail(APEX_EINVAL, "NULL argument");
  if (d->n_queries < 1 || d->n_queries > APEX_MAX_ACTIVE) return fail(APEX_EINVAL, "n_queries outside 1..64");
  if (d->k < 1) return fail(APEX_EINVAL, "k must be >= 1");
  if (!((L->precisions >> d->precision) & 1u) || d->precision == APEX_FP64)
    return fail(APEX_EUNSUPPORTED, "precision %d not available", d->precision);
  memset(out, 0, sizeof(*out));
  const long long chunks[APEX_AUTOTUNE_MAX_CANDIDATES] = {1LL << 23, 1LL << 24, 1LL << 25, 1LL << 26, 1LL << 27};
  const int n_chunks = 5;
  apex_status rc = APEX_OK;
  autotune_run(L, d, L->seed + 101, &rc);  // warm-up: buffers, plans, caches
  if (rc != APEX_OK) return rc;
  double best = 1e300;
  long long best_chunk = L->chunk_compounds.load();
  for (int i = 0; i < n_chunks; ++i) {
    L->chunk_compounds = chunks[i];
    const double ms = autotune_run(L, d, L->seed + 202, &rc);
    if (rc != APEX_OK) return rc;
    out->chunk_compounds[i] = chunks[i];
    out->chunk_ms[i] = ms;
    if (ms < best) {
      best = ms;
      best_chunk = chunks[i];
    }
  }
  out->n_chunk_candidates = n_chunks;
  L->chunk_compounds = best_chunk;
  const int tiles[2] = {32, 128};
  double best_t = 1e300;
  int best_tile = 32;
  for (int i = 0; i < 2; ++i) {
    L->fp32_id_tile = tiles[i];
    const double ms = autotune_run(L, d, L->seed + 303, &rc);
    if (rc != APEX_OK) return rc;
    out->fp32_id_tile_ms[i] = ms;
    if (ms < best_t) {
      best_t = ms;
      best_tile = tiles[i];
    }
  }
  L->fp32_id_tile = best_tile;
  out->chosen_chunk_compounds = best_chunk;
  out->chosen_fp32_id_tile = best_tile;
  return APEX_OK;
}

extern "C" apex_status apex_associative_embeddings(int64_t n_slots_total, const int64_t *slot_sizes, int32_t d,
                                                   int32_t d_u, const float *K, const float *V, float *U,
                                                   int32_t device_pointers, void *cuda_stream) {
  if (n_slots_total < 1 || !slot_sizes || !K || !V || !U) return fail(APEX_EINVAL, "bad arguments");
  if (d < 1 || d > 4096 || d_u < 1 || d_u > 4096) return fail(APEX_EINVAL, "d / d_u outside 1..4096");
  long long rows = 0;
  for (int64_t s = 0; s < n_slots_total; ++s) {
    if (slot_sizes[s] < 1) return fail(APEX_EINVAL, "slot %lld has no synthon", (long long)s);
    rows += slot_sizes[s];
  }
  const int nb = apx_assoc_blocks(n_slots_total, slot_sizes, nullptr, 0);
  if (nb <= 0 || (long long)nb * 64 < rows - 64 * n_slots_total) return fail(APEX_EINVAL, "too many rows");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf B;
  try {
    std::vector<unsigned char> hb(apx_assoc_block_bytes() * nb);
    apx_assoc_blocks(n_slots_total, slot_sizes, hb.data(), nb);
    void *db = B.get(hb.size());
    CU(cudaMemcpyAsync(db, hb.data(), hb.size(), cudaMemcpyHostToDevice, st));
    const size_t kb = sizeof(float) * (size_t)n_slots_total * d * d_u, vb = sizeof(float) * (size_t)rows * d_u,
                 ub = sizeof(float) * (size_t)rows * d;
    const float *dK = K, *dV = V;
    float *dU = U;
    if (!device_pointers) {
      float *k2 = (float *)B.get(kb), *v2 = (float *)B.get(vb);
      CU(cudaMemcpyAsync(k2, K, kb, cudaMemcpyHostToDevice, st));
      CU(cudaMemcpyAsync(v2, V, vb, cudaMemcpyHostToDevice, st));
      dK = k2;
      dV = v2;
      dU = (float *)B.get(ub);
    }
    CU(apx_launch_assoc(db, nb, d, d_u, dK, dV, dU, st));
    if (!device_pointers) CU(cudaMemcpyAsync(U, dU, ub, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
  } catch (const CudaFail &f) {
    return fail(APEX_ECUDA, "associative embeddings: %s failed: %s", f.what, cudaGetErrorString(f.e));
  }
  return APEX_OK;
}

// ------------------------------------------------------------------ library files
static const char kMagic[8] = {'A', 'P', 'E', 'X', 'L', 'I', 'B', '1'};

extern "C" apex_status apex_save_library(const apex_library *L, const char *path) {
  if (!L || !path) return fail(APEX_EINVAL, "NULL argument");
  std::vector<float> U((size_t)L->rows * L->d);
  if (cudaMemcpy(U.data(), L->T_.U, sizeof(float) * U.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(APEX_ECUDA, "save: reading U back failed");
  FILE *f = fopen(path, "wb");
  if (!f) return fail(APEX_EINVAL, "save: cannot open %s", path);
  bool ok = true;
  auto put = [&](const void *p, size_t n) { ok = ok && fwrite(p, 1, n, f) == n; };
  const int32_t hdr[8] = {1, L->T, L->d, L->n_layers, L->act, L->n_obj, L->n_prop, (int32_t)L->precisions_requested};
  put(kMagic, 8);
  put(hdr, sizeof(hdr));
  put(&L->seed, sizeof(L->seed));
  put(L->n_slots.data(), sizeof(int32_t) * L->T);
  put(L->slot_sizes.data(), sizeof(int64_t) * L->slot_sizes.size());
  put(L->dims, sizeof(int32_t) * (L->n_layers + 1));
  for (int l = 0; l < L->n_layers; ++l) {
    put(L->hW[l].data(), sizeof(float) * L->hW[l].size());
    put(L->hb[l].data(), sizeof(float) * L->hb[l].size());
  }
  put(U.data(), sizeof(float) * U.size());
  SavedCal c;
  memset(&c, 0, sizeof(c));
  c.n_calib = L->n_calib;
  memcpy(c.err32, L->err32, sizeof(c.err32));
  memcpy(c.err16, L->err16, sizeof(c.err16));
  memcpy(c.rms, L->rms, sizeof(c.rms));
  put(&c, sizeof(c));
  put(kMagic, 8);  // trailer: a truncated file is rejected at load
  ok = (fclose(f) == 0) && ok;
  return ok ? APEX_OK : fail(APEX_EINVAL, "save: write to %s failed", path);
}

extern "C" apex_status apex_load_library_file(const char *path, int32_t device, void *cuda_stream,
                                              uint64_t device_mem_budget, apex_library **out) {
  if (!path || !out) return fail(APEX_EINVAL, "NULL argument");
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) return fail(APEX_EINVAL, "load: cannot open %s", path);
  bool ok = true;
  auto get = [&](void *p, size_t n) { ok = ok && fread(p, 1, n, f) == n; };
  char magic[8];
  int32_t hdr[8];
  uint64_t seed = 0;
  get(magic, 8);
  get(hdr, sizeof(hdr));
  get(&seed, sizeof(seed));
  if (!ok || memcmp(magic, kMagic, 8) != 0 || hdr[0] != 1) {
    fclose(f);
    return fail(APEX_EINVAL, "load: %s is not a library file of this version", path);
  }
  const int T = hdr[1], d = hdr[2], n_layers = hdr[3];
  if (T < 1 || T > (1 << 24) || d < 1 || d > 1024 || n_layers < 1 || n_layers > 7) {
    fclose(f);
    return fail(APEX_EINVAL, "load: %s has an invalid header", path);
  }
  std::vector<int32_t> n_slots(T);
  get(n_slots.data(), sizeof(int32_t) * T);
  long long S = 0;
  for (int t = 0; ok && t < T; ++t) {
    if (n_slots[t] < 1 || n_slots[t] > APEX_MAX_SLOTS) ok = false;
    S += n_slots[t];
  }
  std::vector<int64_t> sizes(ok ? S : 0);
  get(sizes.data(), sizeof(int64_t) * sizes.size());
  long long rows = 0;
  for (long long j = 0; ok && j < S; ++j) {
    if (sizes[j] < 1 || sizes[j] > (1LL << 40)) ok = false;
    rows += sizes[j];
  }
  std::vector<int32_t> dims(n_layers + 1);
  get(dims.data(), sizeof(int32_t) * dims.size());
  for (int l = 0; ok && l <= n_layers; ++l)
    if (dims[l] < 1 || dims[l] > 1024) ok = false;
  std::vector<std::vector<float>> W, b;
  for (int l = 0; ok && l < n_layers; ++l) {
    W.emplace_back((size_t)dims[l + 1] * dims[l]);
    b.emplace_back((size_t)dims[l + 1]);
    get(W.back().data(), sizeof(float) * W.back().size());
    get(b.back().data(), sizeof(float) * b.back().size());
  }
  std::vector<float> U(ok ? (size_t)rows * d : 0);
  get(U.data(), sizeof(float) * U.size());
  SavedCal cal;
  get(&cal, sizeof(cal));
  get(magic, 8);
  fclose(f);
  if (!ok || memcmp(magic, kMagic, 8) != 0) return fail(APEX_EINVAL, "load: %s is truncated or corrupt", path);
  std::vector<const float *> Wp(n_layers), bp(n_layers);
  for (int l = 0; l < n_layers; ++l) {
    Wp[l] = W[l].data();
    bp[l] = b[l].data();
  }
  apex_library_desc D;
  memset(&D, 0, sizeof(D));
  D.n_reactions = T;
  D.n_slots = n_slots.data();
  D.slot_sizes = sizes.data();
  D.d = d;
  D.U = U.data();
  D.U_on_device = 0;
  D.n_layers = n_layers;
  D.dims = dims.data();
  D.W = Wp.data();
  D.b = bp.data();
  D.activation = hdr[4];
  D.n_objectives = hdr[5];
  D.n_properties = hdr[6];
  D.precisions = (uint32_t)hdr[7];
  D.device_mem_budget = device_mem_budget;
  D.cuda_stream = cuda_stream;
  D.device = device;
  D.seed = seed;
  return load_impl(&D, &cal, out);
}

extern "C" apex_status apex_kernel_launches(int64_t *out) {
  if (!out) return fail(APEX_EINVAL, "NULL argument");
  *out = g_launches.load();
  return APEX_OK;
}

extern "C" apex_status apex_set_finalize_cover(apex_library *L, int64_t cover) {
  if (!L) return fail(APEX_EINVAL, "NULL library");
  if (cover < 0 || cover > (1LL << 30)) return fail(APEX_EINVAL, "cover outside 0..2^30");
  L->fin_cover_set.store(cover);
  return APEX_OK;
}

extern "C" apex_status apex_worker_cpu(const apex_library *L, int32_t *cpu) {
  if (!L || !cpu) return fail(APEX_EINVAL, "NULL argument");
  const double t0 = now_ms();
  while (L->worker_cpu.load() == -2 && now_ms() - t0 < 2000.0)
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  const int c = L->worker_cpu.load();
  *cpu = c < 0 ? -1 : c;
  return APEX_OK;
}

extern "C" const char *apex_last_error(void) { return g_err.c_str(); }
