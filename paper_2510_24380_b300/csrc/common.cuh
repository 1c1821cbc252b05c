// common.cuh -- structures shared by the host library and the kernels, and small device helpers.
//
// Work decomposition (the enumeration of Sec. 3.3 over each reaction's Cartesian product,
// App. GPU implementation): every reaction's slots are split into one "outer" slot and the
// "inner" slots (flattened, mixed radix). A work item is a block of APX_TILE consecutive inner
// indices (one per tile row) times a run of L_o outer indices; each tile row keeps the sum of
// its inner synthons' first-layer rows resident while the outer index advances, so a new tile
// costs one broadcast row instead of APX_TILE gathers. Compound id = id_first + q *
// inner_stride + o * outer_stride (the mixed radix split into its inner and outer parts).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/apex.h"

#define APX_TILE 128
#define APX_MAX_SEG 160
#define APX_MAX_CTA 160  // CTAs of a launch that can take cost-weighted tile ranges
#define APX_SIMT_THREADS 256

struct RxnPlan {
  long long id_first;
  long long n_inner, n_outer;
  long long inner_stride, outer_stride;
  long long outer_row;                       // first table row of the outer slot, -1 = none
  long long inner_row[APEX_MAX_SLOTS];       // first table row of each inner slot (most significant first)
  long long inner_size[APEX_MAX_SLOTS];
  long long n_items;                         // n_b * n_oc
  long long slot_row[APEX_MAX_SLOTS];        // first table row of each slot, library order
  long long slot_size[APEX_MAX_SLOTS];
  int n_slots;
  int n_inner_slots;
  int n_b;                                   // inner tiles = ceil(n_inner / APX_TILE)
  int L_o;                                   // outer indices per item
  int n_oc;                                  // outer runs = ceil(n_outer / L_o)
};

struct Segment {
  int rxn;
  int pad;
  long long item_begin, item_end;           // item range of this reaction
  unsigned long long qmask;                 // query slots served by this segment
};

// One enumeration launch: a list of item ranges, passed by value as a kernel parameter.
struct LaunchPlan {
  int n_seg;
  int mode;                                  // 0 = queries, 1 = dump by id, 2 = dump by launch tile,
                                             // 3 = outputs of an id list (tensor-core kernel)
  int pad;
  long long total_items;
  long long seg_first[APX_MAX_SEG + 1];      // prefix of items
  long long total_tiles;
  long long seg_tile_first[APX_MAX_SEG + 1]; // prefix of tiles (128 inner rows x one outer index)
  Segment seg[APX_MAX_SEG];
  unsigned long long qmask_all;              // union of the segments' query masks
  // dump mode
  float *dump;                               // [dump_n x n_out]
  long long *dump_ids;                       // mode 2: [dump_n], row r of launch tile t at t * 128 + r,
                                             // -1 = padding row; mode 3: the input ids [dump_n]
  long long dump_base, dump_n;
  const unsigned *dump_n_dev;                // mode 3, optional: the list's length on the device
                                             // (at most dump_n; the launch is sized for dump_n)
  // tensor-core kernel, tail pool: tiles [pool_first, total_tiles) are not in any CTA's range; a CTA
  // done with its own range claims them pool_chunk at a time (atomicAdd on *pool_ctr, zeroed before
  // the launch). pool_ctr == nullptr: no pool, the CTA ranges cover every tile.
  unsigned long long *pool_ctr;
  long long pool_first;
  int pool_chunk;
  // tensor-core kernel: CTA c takes launch tiles [cta_first[c], cta_first[c + 1]) when cta_n equals
  // the launch's grid (ranges of equal estimated cost), else an equal count of tiles
  int cta_n;
  long long cta_first[APX_MAX_CTA + 1];
};

// Per-query device state (one per active slot).
struct QuerySlot {
  float w[APEX_MAX_OBJECTIVES];
  int n_obj;
  int n_cons;
  int cons_idx[APEX_MAX_CONSTRAINTS];
  float lo_w[APEX_MAX_CONSTRAINTS], hi_w[APEX_MAX_CONSTRAINTS];  // admission box (widened by the pass margin)
  float lo_s[APEX_MAX_CONSTRAINTS], hi_s[APEX_MAX_CONSTRAINTS];  // sure box (shrunk by the margin)
  float lo_x[APEX_MAX_CONSTRAINTS], hi_x[APEX_MAX_CONSTRAINTS];  // exact box as FP32 bounds: smallest
                                                                 // float >= lo, largest float <= hi
  float admit;        // admission threshold on the pass objective
  float delta_f;      // objective margin of the pass
  float tau;          // k-th largest sure key seen so far (-inf until k sure keys exist)
  float tau_spec;     // speculative start threshold (validated at the end)
  long long k;
  unsigned cap;
  unsigned count;     // appended entries (atomic)
  unsigned count_compacted;  // entries kept by the last in-pass FP32 compaction (0 = none yet)
  unsigned overflow;
  unsigned dropped_bits;  // order-preserving bits of the largest key that did not fit (0 = none)
  unsigned n_sure_above_spec;
  float *keys;
  long long *ids;     // bit 62 set = not surely feasible
  float *keys2;
  long long *ids2;
};

// Speculative start threshold of one query, evaluated on the device: the rank-th best objective
// (exact boxes) of a uniform sample of the query's scope.
struct SpecArgs {
  float w[APEX_MAX_OBJECTIVES];
  int n_obj, n_cons, n_out;
  int bits_in;  // 1: the sample's keys come as order-preserving objective bits (0 = infeasible)
  int cons_idx[APEX_MAX_CONSTRAINTS];
  double lo[APEX_MAX_CONSTRAINTS], hi[APEX_MAX_CONSTRAINTS];
  long long rank;
  float margin2;  // admission threshold = start threshold - margin2 (twice the pass objective margin)
};

#define APX_UNSURE_BIT (1LL << 62)
// A candidate an in-pass compaction kept: its key is the compaction's rescore of its objective (FP16
// on the tensor cores or FP32) and those outputs lie inside the box widened by that rescore's
// margin; the next compaction reuses it.
#define APX_SCORED_BIT (1LL << 61)
#define APX_ID_MASK ((1LL << 61) - 1)

// Kernel status word values (device-side failures; never trap).
#define APX_ERR_TIMEOUT 1
#define APX_ERR_BOUNDS 2

// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned apx_key_bits(float f) {
  // order-preserving map float -> uint32 (larger float -> larger uint)
  unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float apx_bits_key(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// A candidate that did not fit its query's buffer: the buffer has overflowed, and the largest
// dropped key is kept, so finalization can tell whether any dropped compound could still reach
// the top-k (only then is the query rerun).
__device__ __forceinline__ void apx_note_dropped(QuerySlot *Q, float key) {
  atomicExch(&Q->overflow, 1u);
  atomicMax(&Q->dropped_bits, apx_key_bits(key));
}

template <int N>
__device__ __forceinline__ float apx_sel(const float (&o)[N], int idx) {
  // o[idx] for a register array without dynamic indexing
  float v = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) v = (j == idx) ? o[j] : v;
  return v;
}

// Applies every query of qmask to one compound (one row per lane; all 32 lanes call it).
// Sec. 3 / Eq. apex_topk: objective sum_j w_j o_j; feasibility = every constrained output
// inside its box. A compound is admitted when its pass objective reaches the slot's admission
// threshold and it lies inside the widened box; it is marked "sure" if it also lies inside the
// shrunk box (then its feasibility cannot change under the margin).
template <int NOUT>
__device__ __forceinline__ void apx_apply_queries(QuerySlot *__restrict__ slots, unsigned long long qmask, bool valid,
                                                  long long id, const float (&o)[NOUT]) {
  const unsigned lane = threadIdx.x & 31;
  while (qmask) {
    const int s = __ffsll((long long)qmask) - 1;
    qmask &= qmask - 1;
    QuerySlot *Q = slots + s;
    const int n_obj = Q->n_obj;
    float f = 0.f;
#pragma unroll
    for (int j = 0; j < APEX_MAX_OBJECTIVES && j < NOUT; ++j)
      if (j < n_obj) f = fmaf(__ldg(&Q->w[j]), o[j], f);
    bool pass = valid && (f >= *((volatile float *)&Q->admit));
    if (__ballot_sync(0xffffffffu, pass) == 0u) continue;
    bool sure = true;
    const int nc = Q->n_cons;
    for (int i = 0; i < nc; ++i) {
      const float v = apx_sel<NOUT>(o, Q->cons_idx[i]);
      pass = pass && (v >= Q->lo_w[i]) && (v <= Q->hi_w[i]);
      sure = sure && (v >= Q->lo_s[i]) && (v <= Q->hi_s[i]);
    }
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    if (m == 0u) continue;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(&Q->count, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pass) {
      const unsigned pos = base + __popc(m & ((1u << lane) - 1u));
      if (pos < Q->cap) {
        Q->keys[pos] = f;
        Q->ids[pos] = id | (sure ? 0LL : APX_UNSURE_BIT);
      } else {
        apx_note_dropped(Q, f);
      }
    }
  }
}

// Host-side count of kernel launches issued by this library (all launch wrappers add to it).
void apx_count_launch(long long n = 1);

// Warp-aggregated reservation of slots in an append-only array: every lane of the warp calls
// it (uniformly); lanes with take = true get distinct positions from *counter.
__device__ __forceinline__ unsigned apx_warp_reserve(unsigned *counter, bool take) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, take);
  unsigned base = 0;
  if (m && lane == (unsigned)(__ffs(m) - 1)) base = atomicAdd(counter, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, m ? __ffs(m) - 1 : 0);
  return base + __popc(m & ((1u << lane) - 1u));
}

// a / b (returned) and a % b (*rem) for a >= 0, b > 0: in 32-bit arithmetic when both fit, the
// usual case (a 64-bit integer division is a long instruction sequence, and every role of the
// enumeration kernel divides at the start of each run of tiles).
__host__ __device__ __forceinline__ long long apx_divmod(long long a, long long b, long long *rem) {
  if (((unsigned long long)a | (unsigned long long)b) < 4294967296ull) {
    const unsigned q = (unsigned)a / (unsigned)b;
    *rem = (long long)((unsigned)a - q * (unsigned)b);
    return (long long)q;
  }
  const long long q = a / b;
  *rem = a - q * b;
  return q;
}

// Locates item `it` of a launch: segment (binary search) and local item index.
// Tiles of a reaction before its item i, in (inner block b, outer index o) order: item
// b * n_oc + oc covers the tiles b * n_outer + [oc * L_o, min((oc + 1) * L_o, n_outer)).
__host__ __device__ __forceinline__ long long apx_tiles_before(const RxnPlan &p, long long i) {
  long long oc;
  const long long b = apx_divmod(i, p.n_oc, &oc);
  const long long r = oc * p.L_o;
  return b * p.n_outer + (r < p.n_outer ? r : p.n_outer);
}

// A run of consecutive tiles of one segment that share their inner block: rows q0 + [0, 128),
// outer indices [o_begin, o_end).
struct TileRun {
  const RxnPlan *rp;
  int sg;
  long long b, q0, o_begin, o_end;
  unsigned long long qmask;
};

// The run that starts at launch tile `tile` and ends at the segment's end, the inner block's
// end or t_end, whichever comes first.
__device__ __forceinline__ TileRun apx_tile_run(const LaunchPlan &L, const RxnPlan *rx, long long tile,
                                                long long t_end) {
  int lo = 0, hi = L.n_seg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.seg_tile_first[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  const Segment &seg = L.seg[lo];
  TileRun r;
  r.sg = lo;
  r.rp = rx + seg.rxn;
  const long long x = apx_tiles_before(*r.rp, seg.item_begin) + (tile - L.seg_tile_first[lo]);
  const long long x_end = apx_tiles_before(*r.rp, seg.item_end);
  r.b = apx_divmod(x, r.rp->n_outer, &r.o_begin);
  long long n = r.rp->n_outer - r.o_begin;
  if (x_end - x < n) n = x_end - x;
  if (t_end - tile < n) n = t_end - tile;
  r.o_end = r.o_begin + n;
  r.q0 = r.b * APX_TILE;
  r.qmask = seg.qmask;
  return r;
}

__device__ __forceinline__ int apx_find_seg(const LaunchPlan &L, long long it) {
  int lo = 0, hi = L.n_seg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.seg_first[mid] <= it) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// FP32 candidate evaluation arguments (exact box, per-output FP32 margins).
struct EvalArgs {
  const float *out32;       // [n x n_out] FP32 outputs of the candidates
  int n_out;
  const QuerySlot *Q;       // objective weights and constrained output indices
  const float *eps;         // per-output FP32 margin [n_out]
  float eps_f;              // objective margin
  const double *lo, *hi;    // exact box [n_cons]
  float eps_scale;          // this query's factor on eps (1 unless a margin check widened it)
  const float *pass_keys;   // [n] pass objective of every candidate (nullptr: not checked)
  unsigned *obs;            // [1 + n_out] observed maxima as float bits: [0] max |pass key - FP32
                            // objective| (here), [1 + p] max |FP32 - FP64| of output p (k_apply64)
  const int *pos = nullptr; // [n] buffer position of out32 row i (f32 / maybe / sure / pass_keys are
                            // indexed by it); nullptr: row i is position i
  const long long *ids = nullptr;  // candidate ids: an entry with APX_SCORED_BIT has its |key - FP32|
  float scored_scale = 1.f;        // multiplied by this (pass margin / compaction margin) in obs[0]
};

// One selection of k_kth_multi: out_tau = the k-th largest key among flagged entries of [0, n)
// (n clamped to *n_dev when given), -inf with out_ok = 0 when fewer than k are flagged.
struct KthJob {
  const float *keys;
  const unsigned char *flag;
  long long n, k;
  float *out_tau;
  int *out_ok;
  const unsigned *n_dev;
};

// One member of the result set under exact selection.
struct RItem {
  double s;          // best score so far (FP32 rescore, or FP64 once rescored)
  long long id;      // global id (no flag bits)
  int src;           // index into the FP32 candidate arrays
  unsigned char alive, is64, need64, pad;
};

// Device pointers and shapes of a loaded library (passed by value to the kernels).
struct DevTables {
  int n_layers;
  int dims[8];
  int act;                     // APEX_ACT_*
  int n_out;
  int d;
  int n_rx;
  long long n_rows;
  const RxnPlan *rx;           // [n_rx]
  const long long *id_first;   // [n_rx + 1]
  // FP32 path
  const float *P32;            // [n_rows x dims[1]]: W_1 u + b_1 on slot-1 rows
  const float *WT[8];          // layer l >= 1, transposed: [dims[l] x dims[l+1]]
  const float *B[8];           // layer l >= 1
  // FP64 plain path
  const float *U;              // [n_rows x d]
  const double *WT64[8];       // every layer, transposed: [dims[l] x dims[l+1]]
  const double *B64[8];
  // tensor-core path (3-layer heads with dims[1] == dims[2] == 256, <= 16 outputs). P tables and
  // W_3 images per 16-bit format: [0] = BF16, [1] = FP16 (the FP8 pass uses the FP16 ones); W_2
  // images per operand format: [0] = BF16, [1] = FP16, [2] = FP8 e4m3 with per-channel scales s2.
  const unsigned short *P16[2];   // [n_rows + 1 x 256] 16-bit bits, scaled into the activation's input
                                  // space; row n_rows is zero
  const unsigned char *w2img[3];  // W_2 as the SW128 K-major shared-memory image (128 KB; FP8: 64 KB)
  const unsigned char *w3img[2];  // W_3 padded to 16 rows, same layout (8 KB)
  const float *s2;                // FP8: dequantization scale of every W_2 output channel, times the
                                  // inverse of a1_inv (both operands' scales undone in one multiply)
  float a1_inv;                   // FP8: power-of-two factor on a_1 before its e4m3 conversion
                                  // (the layer's static activation scale, 448 / amax rounded down)
  const float *b2s;            // b_2 in the same scaled space [256]
  const float *b3;             // b_3 padded [16]
};
