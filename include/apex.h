/*
 * apex.h -- C ABI of the B300 (sm_103a) exhaustive CSL enumeration library.
 *
 * The library answers the retrieval problem of Sec. 3 (Eq. orig_topk, relaxed to the
 * factorized surrogate in Eq. apex_topk): among all compounds of a combinatorial synthesis
 * library (reactions -> R-group slots -> synthons, Sec. 3.2 / App. A.1), return the k with
 * the largest objective sum_j w_j o_j whose constrained outputs lie in [lower_i, upper_i].
 * A compound's outputs are o = head(g) with g = sum over its slots of the synthon embedding
 * u_{t,j,s} (Eq. factorizer); the first layer is applied per synthon once at load
 * (P_{t,j,s} = W_1 u_{t,j,s}, the substitution of Eq. apex_subtitution..apex generalized to a
 * matrix), so enumeration only sums rows of P and runs the remaining layers.
 *
 * Conventions for every entry point:
 *   - returns apex_status: APEX_OK (0) or a negative code; no C++ exception crosses the ABI;
 *     apex_last_error() returns a thread-local message for the last failure on this thread.
 *   - "host" pointers are ordinary CPU memory owned by the caller, read (or written) only
 *     during the call unless stated otherwise; the caller may free them when the call returns.
 *   - device memory the library allocates is owned by the library and released by
 *     apex_free_library (per-query state: when the query is fetched or cancelled).
 *   - global compound id: off_t + mixed radix of (s_1..s_n), slot 1 most significant, where
 *     off_t = number of compounds of the reactions before t (library order).
 *   - all device work of a library runs on one CUDA stream (the one given at load, or one the
 *     library creates) from a host worker thread owned by the library.
 */
#ifndef APEX_H
#define APEX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t apex_status;
#define APEX_OK 0
#define APEX_EINVAL (-1)        /* malformed descriptor or argument */
#define APEX_ENOMEM (-2)        /* device memory budget or allocation exhausted */
#define APEX_EBUSY (-3)         /* no query slot can ever admit this request */
#define APEX_EAGAIN (-4)        /* query not finished within timeout_ms */
#define APEX_ETIMEDOUT (-5)     /* a device-side bounded wait gave up (kernel status word) */
#define APEX_ECANCELED (-6)     /* the query was cancelled */
#define APEX_ECUDA (-7)         /* a CUDA runtime call failed */
#define APEX_ENOTFOUND (-8)     /* unknown query id */
#define APEX_EUNSUPPORTED (-9)  /* shape/precision combination this build does not implement */

#define APEX_ACT_IDENTITY 0
#define APEX_ACT_RELU 1
#define APEX_ACT_SILU 2

/* Query precision of the enumeration pass. FP32: every layer in FP32 on the CUDA cores.
 * BF16 / FP16: layers 2.. on tcgen05 tensor cores (16-bit operands and activations, FP32
 * accumulators in TMEM); FP16 carries 3 more mantissa bits at the same tensor rate, so its
 * calibrated margins are tighter. FP8: layer 2 with e4m3 operands (activations quantized from
 * FP16, W_2 quantized per output channel with scale max|row| / 448, FP32 accumulators multiplied
 * back by the scales), layer 3 in FP16; twice the dense tensor rate on layer 2, much wider
 * margins (three mantissa bits). Between the launches of a pass, a query whose candidate buffer
 * fills up has it rescored (FP16 on the tensor cores for BF16 and FP8 passes, else FP32) and cut
 * to what can still reach the top-k. At the end of the pass the candidates are rescored in FP32
 * and the top-k boundary band in FP64, so the returned set equals the FP64 top-k when the
 * calibrated error bounds hold. APEX_FP64 is accepted by apex_score_ids only. */
#define APEX_FP32 0
#define APEX_BF16 1
#define APEX_FP64 2
#define APEX_FP16 3
#define APEX_FP8 4

#define APEX_MAX_SLOTS 4          /* slots per reaction */
#define APEX_MAX_OUTPUTS 32       /* head outputs */
#define APEX_MAX_OBJECTIVES 16
#define APEX_MAX_CONSTRAINTS 16
#define APEX_MAX_ACTIVE 64        /* queries sharing one enumeration pass */

typedef struct apex_library apex_library;
typedef int64_t apex_query_id;

/* Library descriptor (Sec. 3.2 hierarchy + head). Read during apex_load_library only. */
typedef struct {
  int32_t n_reactions;          /* >= 1 */
  const int32_t *n_slots;       /* host [n_reactions], each in 1..APEX_MAX_SLOTS */
  const int64_t *slot_sizes;    /* host [sum n_slots], reaction-major, each >= 1 */
  int32_t d;                    /* embedding width, == dims[0] */
  const float *U;               /* [sum slot_sizes x d] row-major float32, rows reaction -> slot ->
                                   synthon; host memory, or device memory when U_on_device != 0
                                   (then 16-byte aligned; the library copies it either way) */
  int32_t U_on_device;
  int32_t n_layers;             /* >= 1 */
  const int32_t *dims;          /* host [n_layers + 1]; hidden widths <= 256; dims[n_layers] <= 32 */
  const float *const *W;        /* host [n_layers] of host float32 [dims[l+1] x dims[l]] row-major */
  const float *const *b;        /* host [n_layers] of host float32 [dims[l+1]] */
  int32_t activation;           /* APEX_ACT_*, applied after every layer but the last */
  int32_t n_objectives;         /* outputs [0, n_objectives) may carry objective weight */
  int32_t n_properties;         /* n_objectives + n_properties == dims[n_layers] */
  uint32_t precisions;          /* bits (1 << APEX_BF16), (1 << APEX_FP16), (1 << APEX_FP8) build the
                                   tensor-core tables (BF16 and FP8 also build the FP16 ones: FP8
                                   reads them, and both rescore candidates in FP16 between the
                                   launches of a pass); FP32 always */
  uint64_t device_mem_budget;   /* bytes the library may hold on the device; 0 = unlimited */
  void *cuda_stream;            /* cudaStream_t to run on; NULL = the library creates one */
  int32_t device;               /* CUDA device ordinal */
  uint64_t seed;                /* seed of the calibration sample */
} apex_library_desc;

/* Query descriptor (Eq. orig_topk: objective weights, constraint boxes, k). Copied by
 * apex_query; the caller may free it when the call returns. */
typedef struct {
  int32_t precision;            /* APEX_FP32, APEX_BF16, APEX_FP16 or APEX_FP8 */
  const float *objective_weights; /* host [n_objectives]; the objective is maximized */
  int32_t n_constraints;        /* 0..APEX_MAX_CONSTRAINTS */
  const int32_t *output_index;  /* host [n_constraints], any output index */
  const double *lower;          /* host [n_constraints]; inclusive; -INFINITY allowed */
  const double *upper;          /* host [n_constraints]; inclusive; +INFINITY allowed; lower <= upper */
  int64_t k;                    /* >= 1 */
  int32_t n_reaction_subset;    /* 0 = every reaction */
  const int32_t *reactions;     /* host [n_reaction_subset], distinct reaction indices */
} apex_query_desc;

typedef struct {
  int64_t n_compounds;          /* N = sum_t prod_j |slot_{t,j}| (App. A.1) */
  int64_t n_synthon_rows;       /* sum of slot sizes */
  int32_t max_slots;
  int32_t n_outputs;
  uint64_t device_bytes;        /* device memory held by the library tables */
  uint32_t precisions;          /* tables built */
  int32_t n_calibration;        /* compounds in the calibration sample */
  double err_bf16[APEX_MAX_OUTPUTS]; /* per-output admission margin of the BF16 pass */
  double err_fp16[APEX_MAX_OUTPUTS]; /* per-output admission margin of the FP16 pass */
  double err_fp8[APEX_MAX_OUTPUTS];  /* per-output admission margin of the FP8 pass */
  double err_fp32[APEX_MAX_OUTPUTS]; /* per-output margin of the FP32 rescore */
  double rms[APEX_MAX_OUTPUTS];      /* output RMS over the calibration sample */
} apex_library_info_t;

typedef struct {
  int64_t n_scope;              /* compounds in the query's reaction subset */
  int64_t n_scored;             /* head evaluations of enumeration launches that served it */
  int64_t n_candidates;         /* first-pass candidates rescored in FP32 */
  int64_t n_rescored_fp64;      /* compounds rescored in FP64 */
  int64_t n_feasible_lower;     /* results found (<= k) */
  int32_t n_restarts;           /* reruns after a candidate buffer overflow or a failed start guess */
  int32_t n_launches;           /* enumeration launches that served this query */
  double queue_ms;              /* host wall time from apex_query to admission */
  double latency_ms;            /* host wall time from apex_query until the results were ready */
  double gpu_ms;                /* device time (CUDA events) from its first to its last kernel */
  double enumerate_ms;          /* device time of the enumeration launches that served it */
  double host_start_ms;         /* worker wall time spent estimating the start threshold */
  double host_pass_ms;          /* worker wall time of the pass steps that served it */
  double host_finalize_ms;      /* worker wall time of exact selection, ordering and decode */
  /* Runtime check of the calibrated margins on the compounds that matter (the candidates, i.e. the
   * tail of the objective distribution, not a uniform sample): at finalization every candidate has
   * its pass objective and its FP32 rescore, and every FP64-rescored member its FP32 and FP64
   * outputs. pass_err_ratio = max |pass - FP32| objective / the pass's objective margin;
   * fp32_err_ratio = max over outputs of max |FP32 - FP64| / that output's FP32 margin. A ratio
   * above 1 means a margin was too small for this query: its pass is rerun with both margins
   * widened (at least 2x, and at least twice the observed ratio), up to 4 times; the ratios
   * reported are those of the final run. */
  int32_t n_margin_reruns;
  int32_t n_compactions;        /* in-pass compactions of its candidate buffer (a buffer filled
                                   between launches is rescored -- FP16 on the tensor cores for
                                   BF16 and FP8 passes, else FP32 -- and cut to what can still
                                   reach the top-k; the admission threshold rises accordingly) */
  double pass_err_ratio;
  double fp32_err_ratio;
  int64_t first_item;           /* work item of the library's circular pass at which the query's (last)
                                   pass began: queries that arrive while others run join at the
                                   pass's current position */
} apex_query_stats_t;

/* Pure host: N = sum_t prod_j slot_sizes (App. A.1). EINVAL on bad shapes or int64 overflow. */
apex_status apex_count_compounds(int32_t n_reactions, const int32_t *n_slots, const int64_t *slot_sizes,
                                 int64_t *n_out);

/* Validates desc (before touching the GPU), uploads U and the head, builds P = W_1 U^T (+ b_1
 * folded into slot 1 rows) in FP32 and, if requested, the BF16 tables and tensor-core weight
 * images, calibrates the error margins on a seeded sample, and starts the worker thread.
 * EINVAL bad desc; ENOMEM over budget; EUNSUPPORTED e.g. BF16 with hidden widths != 256;
 * ECUDA on a CUDA failure. On error *out is NULL and nothing is leaked. */
apex_status apex_load_library(const apex_library_desc *desc, apex_library **out);

/* Stops the worker (pending queries end as ECANCELED), frees every device buffer. NULL is OK. */
apex_status apex_free_library(apex_library *lib);

apex_status apex_library_info(const apex_library *lib, apex_library_info_t *out);

/* Submits a query (Eq. apex_topk) and returns at once with its id. The worker admits it
 * when a slot (APEX_MAX_ACTIVE) and device memory for its candidate state are free, and
 * serves it from the shared enumeration pass (continuous batching); queries that arrive
 * while others run join the pass at its current position and leave after one revolution
 * over their own reactions. EINVAL bad desc (NaN bound, lower > upper, index out of range,
 * k < 1, duplicate or out-of-range reaction); EUNSUPPORTED precision not built. */
apex_status apex_query(apex_library *lib, const apex_query_desc *desc, apex_query_id *out);

/* Waits up to timeout_ms (< 0: forever) for the query, then copies min(capacity, n) results,
 * n = min(k, feasible compounds in scope), ordered by (objective desc, id asc):
 *   ids [cap], reaction [cap], synthons [cap x APEX_MAX_SLOTS] (-1 padded),
 *   objective [cap], outputs [cap x n_outputs]   -- host buffers; any may be NULL.
 * Objectives and outputs are the FP32 rescore, replaced by FP64 for every compound in the
 * top-k boundary band (within the FP32 margin of the k-th objective) or within the FP32 margin
 * of a constraint bound; the returned set is the FP64 top-k, and results whose FP32 objectives
 * are closer than the FP32 margin are ordered by those. *n_out = n.
 * EAGAIN: not done yet (the query stays alive); otherwise the query is released.
 * Several threads may fetch the same id at once: the first to see it finished receives its rows
 * (or its error) and releases it; the others then return APEX_ENOTFOUND.
 * Waiting: up to two concurrent callers first watch a completion counter (busy, yielding the CPU
 * every few microseconds) for at most APEX_FETCH_SPIN_MS (default 20) of the timeout, then sleep
 * until the query finishes; more callers sleep at once. */
apex_status apex_topk_fetch(apex_library *lib, apex_query_id id, int64_t capacity, int64_t *ids,
                            int32_t *reaction, int64_t *synthons, double *objective, double *outputs,
                            int64_t *n_out, int32_t timeout_ms);

/* Cancels a queued or running query; a later fetch returns ECANCELED. */
apex_status apex_cancel(apex_library *lib, apex_query_id id);

/* Statistics of a finished (not yet fetched) query, or of the last fetched one when id < 0. */
apex_status apex_query_stats(apex_library *lib, apex_query_id id, apex_query_stats_t *out);

/* Serving statistics of the library over the queries fetched since the load or the last
 * apex_stats_reset (the request loop's view: continuous batching serves many queries at once, so
 * latency and throughput are properties of the mix, not of one query). Latencies are host wall
 * times from apex_query until the query's results were ready; percentiles interpolate linearly
 * between the two nearest ranks (rank p/100 * (n - 1) of the sorted sample), over the last
 * APEX_STATS_WINDOW fetched queries. The window of the throughput figures runs from the earliest
 * submission to the latest completion among the counted queries. */
#define APEX_STATS_WINDOW (1 << 20)
typedef struct {
  int64_t n_queries;            /* fetched with APEX_OK */
  int64_t n_failed;             /* fetched with an error (cancelled, failed, timed out) */
  double p50_ms, p99_ms, max_ms, mean_ms;   /* latency of the APEX_OK queries */
  double queue_p50_ms, queue_p99_ms;        /* time from apex_query to admission into a slot */
  double wall_ms;               /* earliest submission -> latest completion of the counted queries */
  double query_compounds;       /* sum over those queries of the compounds in their reaction subsets */
  double head_evaluations;      /* compounds scored by enumeration launches since the load or reset
                                   (one per compound and launch, whatever the number of queries the
                                   launch served) */
  double query_compounds_per_s; /* query_compounds / wall */
  double head_evaluations_per_s;/* head_evaluations / wall */
  double enumerate_ms;          /* device time (CUDA events) of the enumeration launches retired since
                                   the load or reset */
  int64_t n_enumeration_launches;
} apex_stats_t;
apex_status apex_stats(apex_library *lib, apex_stats_t *out);
apex_status apex_stats_reset(apex_library *lib);

/* Scores given compounds (host ids [n]) through the gather kernels: precision APEX_FP32
 * (CUDA cores), APEX_FP64 (plain form g = sum u, then the head), or a reduced precision the
 * library was built with (APEX_BF16, APEX_FP16, APEX_FP8: the tensor-core kernel over the id
 * list, every slot's P row summed per compound; the path of a query's start-threshold sample).
 * outputs: host [n x n_outputs]. Synchronous. Returns APEX_EINVAL for an unknown precision or an
 * id out of range, APEX_EUNSUPPORTED for a reduced precision the library does not hold. Used for
 * calibration checks and parity tests. */
apex_status apex_score_ids(apex_library *lib, int32_t precision, int64_t n, const int64_t *ids,
                           double *outputs);

/* Runs the production enumeration kernel of the given precision over one reaction and
 * writes the raw outputs of every compound, in id order: host float [N_t x n_outputs].
 * reaction = -1: the whole library, in launches shaped like those of a query's pass (consecutive
 * work items in library order, about the library's compounds per launch each, apex_set_launch_shape
 * / apex_autotune) into host float [N x n_outputs]; at most 16 GB of outputs, else APEX_EINVAL.
 * capacity is the number of rows of outputs. Synchronous; meant for tests of raw scores. */
apex_status apex_dump_outputs(apex_library *lib, int32_t precision, int32_t reaction, float *outputs,
                              int64_t capacity);

/* Decodes global ids into (reaction, synthon indices); host buffers; pure host work. */
apex_status apex_decode_ids(const apex_library *lib, int64_t n, const int64_t *ids, int32_t *reaction,
                            int64_t *synthons);

/* Top-k selection step on device data (Sec. 3.3 queue, realised as a radix select): among n
 * keys (device float [n]) with ids (device int64 [n]), writes the k largest keys, ties by
 * smaller id, in (key desc, id asc) order to out_keys / out_ids (device [k]) and *n_out =
 * min(k, n) (host). Scratch comes from cudaMalloc inside the call. cuda_stream may be NULL. */
apex_status apex_topk_select(const float *keys, const int64_t *ids, int64_t n, int64_t k, float *out_keys,
                             int64_t *out_ids, int64_t *n_out, void *cuda_stream);

/* apex_topk_select for callers that cannot allocate device memory (a caller-owned memory
 * pool or arena that forbids outside allocations, a host callback or latency-critical loop
 * that must not pay cudaMalloc's synchronization, a plugin whose host framework owns every
 * allocation). Same arguments, same result and order as apex_topk_select; no counterpart in
 * the paper. Its scratch is one file-scope device array of fixed size (about 1.6 MB, held by
 * every GPU that loads the library until the process exits), so it calls no cudaMalloc,
 * cudaFree or allocating routine. min(k, n) must be <= APEX_SELECT_NOALLOC_MAX_K, else EINVAL.
 * The first call on a device looks up the array's device address (with that device current) and,
 * under CUDA's lazy module loading, is also where the select kernels' module gets loaded, so it
 * takes longer than later calls; make that first call before any stream capture. All calls share
 * the one array and it keeps the last call's contents: calls that overlap on the GPU (other
 * streams, other host threads) race. Each call clears the state it needs, and before returning
 * it waits for its stream to finish (cudaStreamSynchronize on cuda_stream). */
#define APEX_SELECT_NOALLOC_MAX_K 65536
apex_status apex_topk_select_noalloc(const float *keys, const int64_t *ids, int64_t n, int64_t k, float *out_keys,
                                     int64_t *out_ids, int64_t *n_out, void *cuda_stream);

/* Number of kernel launches this process has issued through the library so far (all
 * libraries, all entry points). Pure host counter. */
apex_status apex_kernel_launches(int64_t *out);

/* Library files. apex_save_library writes everything a library was loaded from (reaction
 * shapes, U read back from the device, the head, activation, objective/property split, the
 * requested precisions, the seed) plus its calibrated margins to one binary file (little
 * endian, "APEXLIB1" magic at both ends, host-native layout). apex_load_library_file rebuilds
 * the library from such a file on `device`, with the given stream (NULL: own stream) and memory
 * budget (0: none), restoring the margins instead of recalibrating. Errors: APEX_EINVAL (cannot
 * open, wrong magic or version, truncated or invalid contents), plus apex_load_library's. */
apex_status apex_save_library(const apex_library *lib, const char *path);
apex_status apex_load_library_file(const char *path, int32_t device, void *cuda_stream, uint64_t device_mem_budget,
                                   apex_library **out);

/* Associative embeddings, Eq. assoc_embeds: u_{r,s} = K_r v_s for every synthon row of every
 * R-group slot r (Sec. 3.2: an R-group key matrix times a synthon value vector), the table U that
 * apex_library_desc.U takes. Slots are in library order (reaction -> slot) and rows slot-major,
 * as in apex_library_desc. K: [n_slots_total x d x d_u] float, each K_r row-major (d rows of d_u);
 * V: [sum slot_sizes x d_u]; U (out): [sum slot_sizes x d]. FP32 on the CUDA cores, one pass.
 * device_pointers = 1: K, V, U are device pointers (U may be handed to apex_load_library with
 * U_on_device = 1); 0: host pointers, copied in and out. cuda_stream: cudaStream_t or NULL.
 * Synchronizes the stream before returning. Errors: APEX_EINVAL (empty slot, d or d_u outside
 * 1..4096, NULL pointer), APEX_ECUDA. */
apex_status apex_associative_embeddings(int64_t n_slots_total, const int64_t *slot_sizes, int32_t d, int32_t d_u,
                                        const float *K, const float *V, float *U, int32_t device_pointers,
                                        void *cuda_stream);

/* Autotuner. Picks the library's launch shapes by timing trial queries through the normal query
 * path (apex_query / apex_topk_fetch; no other query should be running): (1) the number of
 * compounds per enumeration launch of the circular pass (2^23 .. 2^27): smaller launches tighten
 * the running admission thresholds sooner, larger ones cost fewer launches and synchronizations;
 * (2) the rows per CTA tile of the FP32 kernel over id lists (32 or 128), used for the
 * start-threshold sample and the candidate rescore. Trial queries: n_queries (1..64) submitted
 * together, seeded convex objective weights, two boxes of +-1 RMS around 0 on seeded properties,
 * the given k, precision and reaction subset (0/NULL = all). The choices stay in effect for the
 * library; out receives every candidate's wall time (ms) and the choices. */
#define APEX_AUTOTUNE_MAX_CANDIDATES 8
typedef struct {
  int32_t precision;
  int32_t n_queries;
  int64_t k;
  int32_t n_reaction_subset;
  const int32_t *reactions;
} apex_autotune_desc;
typedef struct {
  int32_t n_chunk_candidates;
  int64_t chunk_compounds[APEX_AUTOTUNE_MAX_CANDIDATES];
  double chunk_ms[APEX_AUTOTUNE_MAX_CANDIDATES];
  double fp32_id_tile_ms[2];          /* tiles of 32 and 128 rows */
  int64_t chosen_chunk_compounds;
  int32_t chosen_fp32_id_tile;
} apex_autotune_result_t;
apex_status apex_autotune(apex_library *lib, const apex_autotune_desc *desc, apex_autotune_result_t *out);

/* Sets the launch shape by hand (the two values apex_autotune picks): compounds per enumeration
 * launch of the circular pass (chunk_compounds >= 128; the planner rounds it to whole work items,
 * and a query's first launches stay at most 2^24, 2^26, ... compounds) and rows per CTA tile of
 * the FP32 kernel over id lists (fp32_id_tile: 32 or 128). Affects launches planned after the call.
 * APEX_EINVAL for other values. */
apex_status apex_set_launch_shape(apex_library *lib, int64_t chunk_compounds, int32_t fp32_id_tile);

/* Candidates covered by the finalization chain that is queued behind a query's last enumeration
 * launch before its candidate count is known (0 restores the default, max(4096, 4 k), capped by
 * the query's candidate buffer). A query with more candidates than that has its chain queued
 * again, sized exactly, after one more host wait: a smaller cover trades device scratch for that
 * rerun; results do not depend on it. Affects finalizations that start after the call.
 * APEX_EINVAL for a NULL library or a cover outside 0..2^30. */
apex_status apex_set_finalize_cover(apex_library *lib, int64_t cover);

/* CPU the library's worker thread is pinned to (-1: not pinned), waiting up to 2 s for the worker
 * to choose it after the load. The worker issues every CUDA call of the query path; CUDA calls from
 * the CPU that created the device context were measured about three times cheaper than from any
 * other CPU. The worker is not pinned unless the environment says so at load: APEX_WORKER_CPU=auto
 * pins it to the CPU with the cheapest calls when one is clearly cheaper, APEX_WORKER_CPU=n to CPU
 * n. An application thread that busy-polls or computes on a pinned worker's CPU slows the worker
 * down: keep such threads off it.
 * APEX_EINVAL for a NULL argument. */
apex_status apex_worker_cpu(const apex_library *lib, int32_t *cpu);

/* Failure-detection self-test of the bounded device waits. Every wait inside this library's
 * kernels (mbarrier phases between warp roles) gives up after a time limit (2 s in production
 * kernels), records a timeout in the launch's status word and returns; the host then fails the
 * affected queries with APEX_ETIMEDOUT and the CUDA context stays usable. This call launches one
 * thread that waits, with the same routine and a limit of limit_ms (1..2000), on a barrier phase
 * that nothing completes, on the library's stream, with a status word of its own (running
 * queries are not affected, but their next synchronization waits for it).
 * Returns APEX_ETIMEDOUT when the wait gave up as designed, APEX_ECUDA if it did not. */
apex_status apex_selftest_wait_timeout(apex_library *lib, int32_t limit_ms);

/* Thread-local message describing the last error returned on this thread ("" if none). */
const char *apex_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* APEX_H */
