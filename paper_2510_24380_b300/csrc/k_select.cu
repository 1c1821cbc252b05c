// k_select.cu -- streaming top-k state of the queries (the size-k priority queue of Sec. 3.3
// realised as threshold-filtered candidate buffers), radix selection, candidate evaluation,
// bitonic ordering by (objective desc, id asc), decode of the final ids (App. GPU impl.:
// "index decoding"), and the standalone select entry point.
#include <cfloat>
#include <cmath>
#include <algorithm>
#include "common.cuh"

#define SEL_THREADS 1024

// ------------------------------------------------------------------ block radix select
// k-th largest 32-bit key (order-preserving bits) among n entries; include(i) filters.
// Returns true and *out_bits when at least k entries are included.
struct SelSrc {
  const float *keys;          // float keys
  const long long *ids;       // optional: entries with APX_UNSURE_BIT are excluded
  const unsigned char *flag;  // optional: entries with flag == 0 are excluded
  __device__ __forceinline__ bool get(long long i, unsigned &bits) const {
    if (ids && (ids[i] & APX_UNSURE_BIT)) return false;
    if (flag && !flag[i]) return false;
    bits = apx_key_bits(keys[i]);
    return true;
  }
};

// Keys staged in shared memory as order-preserving bits, 0 = excluded (no finite key maps to 0).
struct SelSmem {
  const unsigned *bits;
  __device__ __forceinline__ bool get(long long i, unsigned &b) const {
    b = bits[i];
    return b != 0u;
  }
};

template <class Src>
__device__ bool block_kth_largest(const Src &src, long long n, long long k, unsigned *out_bits,
                                  unsigned long long *out_included) {
  // Keys of a top-k buffer share their leading bits, so many lanes hit the same histogram bin:
  // lanes with equal digits are merged first (match.any) and one lane adds the group's count.
  __shared__ unsigned hist[256];
  __shared__ unsigned prefix_s;
  __shared__ long long kk_s;
  __shared__ unsigned long long total_s;
  if (threadIdx.x == 0) {
    prefix_s = 0;
    kk_s = k;
  }
  const unsigned lane = threadIdx.x & 31;
  const long long warp_base = (long long)(threadIdx.x >> 5) * 32;
  const long long stride = (long long)blockDim.x;
  unsigned mask = 0;
  for (int pass = 3; pass >= 0; --pass) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const unsigned prefix = prefix_s;
    for (long long b = warp_base; b < n; b += stride) {   // uniform trip count within a warp
      const long long i = b + lane;
      unsigned bits = 0;
      const bool use = (i < n) && src.get(i, bits) && ((bits & mask) == prefix);
      const unsigned dig = use ? ((bits >> (8 * pass)) & 255u) : 256u;
      const unsigned grp = __match_any_sync(0xffffffffu, dig);
      if (use && (int)lane == __ffs(grp) - 1) atomicAdd(&hist[dig], (unsigned)__popc(grp));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // the digit of the kk-th largest key: bins from the top, 8 per lane (lane l holds digits
      // 255 - 8l down to 248 - 8l), a warp prefix sum, then the one lane whose range crosses kk
      // walks its bins. No crossing (fewer than kk keys): digit 0, every key counted.
      const unsigned long long kk = (unsigned long long)kk_s;
      unsigned c[8];
      unsigned long long own = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        c[j] = hist[255 - 8 * (int)lane - j];
        own += c[j];
      }
      unsigned long long incl = own;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
        if ((int)lane >= off) incl += v;
      }
      const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
      unsigned long long cum = incl - own;
      const unsigned hit = __ballot_sync(0xffffffffu, cum < kk && incl >= kk);
      if (lane == 0 && pass == 3) total_s = total;
      if (hit == 0u) {
        if (lane == 0) {
          kk_s = (long long)(kk - total);
          prefix_s = prefix;
        }
      } else if ((int)lane == __ffs(hit) - 1) {
        int dsel = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (cum + c[j] >= kk) {
            dsel = 255 - 8 * (int)lane - j;
            break;
          }
          cum += c[j];
        }
        kk_s = (long long)(kk - cum);
        prefix_s = prefix | ((unsigned)dsel << (8 * pass));
      }
    }
    __syncthreads();
    mask |= 255u << (8 * pass);
    if (total_s < (unsigned long long)k) break;
  }
  if (out_included) *out_included = total_s;
  *out_bits = prefix_s;
  const bool ok = total_s >= (unsigned long long)k;
  __syncthreads();
  return ok;
}

// ------------------------------------------------------------------ per-slot select / compaction
// mode 0 (between the launches of a pass): whenever the buffer holds more than k entries, so the
// admission threshold tightens after the first launch instead of waiting for the buffer to
// fill; mode 1: always (end of the pass).
// Raises tau (k-th largest sure key) and the admission threshold tau - 2 delta_f, then keeps
// only entries at or above the admission threshold.
#define SEL_SMEM_KEYS 49152  // buffers up to this size are selected from shared memory (192 KB)
#define SEL_SKIP_ABOVE (1u << 17)
__global__ void __launch_bounds__(SEL_THREADS) k_slot_select(QuerySlot *slots, const int *slot_list, int mode) {
  QuerySlot *Q = slots + slot_list[blockIdx.x];
  extern __shared__ unsigned sel_bits[];  // SEL_SMEM_KEYS entries
  __shared__ unsigned kept;
  __shared__ unsigned n_spec;
  const unsigned n = min(*((volatile unsigned *)&Q->count), Q->cap);
  if (mode == 0 && (long long)n <= Q->k) return;
  // Between launches, a buffer of more than SEL_SKIP_ABOVE entries whose query was already
  // compacted is left to the next compaction: its admission floor is already the compaction's
  // certified one, and one CTA would take milliseconds over the whole buffer (FP8 passes).
  if (mode == 0 && n > SEL_SKIP_ABOVE && Q->count_compacted > 0) return;
  unsigned bits;
  bool found;
  if (n <= SEL_SMEM_KEYS) {
    // one coalesced pass stages the keys (unsure entries excluded), the radix passes read shared memory
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x)
      sel_bits[i] = (Q->ids[i] & APX_UNSURE_BIT) ? 0u : apx_key_bits(Q->keys[i]);
    __syncthreads();
    found = block_kth_largest(SelSmem{sel_bits}, n, Q->k, &bits, nullptr);
  } else {
    found = block_kth_largest(SelSrc{Q->keys, Q->ids, nullptr}, n, Q->k, &bits, nullptr);
  }
  if (found) {
    if (threadIdx.x == 0) {
      const float tau = apx_bits_key(bits);
      if (!(tau <= Q->tau)) Q->tau = tau;
      const float adm = Q->tau - 2.0f * Q->delta_f;
      if (!(adm <= Q->admit)) Q->admit = adm;
    }
  }
  if (threadIdx.x == 0) {
    kept = 0;
    n_spec = 0;
  }
  __syncthreads();
  const float admit = Q->admit;
  const float spec = Q->tau_spec;
  const unsigned lane = threadIdx.x & 31;
  for (unsigned b = (threadIdx.x >> 5) * 32; b < n; b += blockDim.x) {
    const unsigned i = b + lane;
    float key = 0.f;
    long long id = 0;
    if (i < n) {
      key = Q->keys[i];
      id = Q->ids[i];
    }
    const bool spec_hit = (i < n) && mode == 1 && !(id & APX_UNSURE_BIT) && key >= spec;
    const unsigned sm = __ballot_sync(0xffffffffu, spec_hit);
    if (lane == 0 && sm) atomicAdd(&n_spec, (unsigned)__popc(sm));
    const bool keep = (i < n) && key >= admit;
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    unsigned base = 0;
    if (lane == 0 && km) base = atomicAdd(&kept, (unsigned)__popc(km));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) {
      const unsigned p = base + __popc(km & ((1u << lane) - 1u));
      Q->keys2[p] = key;
      Q->ids2[p] = id;
    }
  }
  __syncthreads();
  const unsigned m = kept;
  for (unsigned i = threadIdx.x; i < m; i += blockDim.x) {
    Q->keys[i] = Q->keys2[i];
    Q->ids[i] = Q->ids2[i];
  }
  if (threadIdx.x == 0) {
    Q->count = m;
    if (mode == 1) Q->n_sure_above_spec = n_spec;
  }
}

cudaError_t apx_launch_slot_select(QuerySlot *slots, const int *slot_list, int n_slots, int mode, cudaStream_t st) {
  if (n_slots <= 0) return cudaSuccess;
  apx_count_launch();
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_slot_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(SEL_SMEM_KEYS * sizeof(unsigned)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_slot_select<<<n_slots, SEL_THREADS, SEL_SMEM_KEYS * sizeof(unsigned), st>>>(slots, slot_list, mode);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 candidate evaluation
// From FP32 outputs of the candidates: objective, maybe-feasible (box widened by the FP32
// margin eps) and sure-feasible (box shrunk by eps).

__global__ void k_eval32(EvalArgs a, long long n, float *f32, unsigned char *maybe, unsigned char *sure,
                         const unsigned *n_dev) {
  if (n_dev && (long long)*n_dev < n) n = *n_dev;  // candidate count on the device
  // the widened and shrunk boxes as FP32 bounds deciding exactly like the FP64 arithmetic for FP32
  // values (FP64 compares run at a small fraction of the FP32 rate)
  __shared__ float mlo[APEX_MAX_CONSTRAINTS], mhi[APEX_MAX_CONSTRAINTS], slo[APEX_MAX_CONSTRAINTS],
      shi[APEX_MAX_CONSTRAINTS];
  const int m = a.Q->n_cons;
  if (threadIdx.x < (unsigned)m) {
    const int c = threadIdx.x, p = a.Q->cons_idx[c];
    const double e = (double)a.eps[p] * (double)a.eps_scale;
    mlo[c] = __double2float_ru(a.lo[c] - e);
    mhi[c] = __double2float_rd(a.hi[c] + e);
    slo[c] = __double2float_ru(a.lo[c] + e);
    shi[c] = __double2float_rd(a.hi[c] - e);
  }
  __syncthreads();
  float dmax = 0.f;  // largest |pass key - FP32 objective| this thread saw
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float *o = a.out32 + i * a.n_out;
    float f = 0.f;
    for (int j = 0; j < a.Q->n_obj; ++j) f = fmaf(a.Q->w[j], o[j], f);
    bool mb = true, sr = true;
    for (int c = 0; c < m; ++c) {
      const float v = o[a.Q->cons_idx[c]];
      mb = mb && v >= mlo[c] && v <= mhi[c];
      sr = sr && v >= slo[c] && v <= shi[c];
    }
    const long long t = a.pos ? (long long)a.pos[i] : i;
    f32[t] = f;
    maybe[t] = mb;
    sure[t] = sr;
    if (a.pass_keys) {
      float d = __fsub_ru(fmaxf(a.pass_keys[t], f), fminf(a.pass_keys[t], f));
      if (a.ids && (a.ids[t] & APX_SCORED_BIT)) d = __fmul_ru(d, a.scored_scale);  // against its own margin
      dmax = fmaxf(dmax, d);
    }
  }
  if (a.obs) {  // every thread of the block reaches this point
    for (int off = 16; off > 0; off >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    if ((threadIdx.x & 31) == 0 && dmax > 0.f) atomicMax(a.obs, __float_as_uint(dmax));
  }
}

// tau32 = k-th largest f32 among sure entries (one CTA)
__device__ __forceinline__ void kth_block(const float *keys, const unsigned char *flag, long long n, long long k,
                                          float *out_tau, int *out_ok, const unsigned *n_dev) {
  extern __shared__ unsigned sel_bits[];
  if (n_dev && (long long)*n_dev < n) n = *n_dev;
  unsigned bits;
  bool ok;
  if (n <= SEL_SMEM_KEYS) {  // stage once, select from shared memory
    for (long long i = threadIdx.x; i < n; i += blockDim.x) sel_bits[i] = flag[i] ? apx_key_bits(keys[i]) : 0u;
    __syncthreads();
    ok = block_kth_largest(SelSmem{sel_bits}, n, k, &bits, nullptr);
  } else {
    ok = block_kth_largest(SelSrc{keys, nullptr, flag}, n, k, &bits, nullptr);
  }
  if (threadIdx.x == 0) {
    *out_tau = ok ? apx_bits_key(bits) : -INFINITY;
    *out_ok = ok;
  }
}
__global__ void __launch_bounds__(SEL_THREADS) k_kth(const float *keys, const unsigned char *flag, long long n, long long k,
                                                     float *out_tau, int *out_ok, const unsigned *n_dev) {
  kth_block(keys, flag, n, k, out_tau, out_ok, n_dev);
}
// several independent selections, one CTA each (the in-pass compactions queued at one launch
// boundary: their selects run side by side instead of one after another)
__global__ void __launch_bounds__(SEL_THREADS) k_kth_multi(const KthJob *jobs) {
  const KthJob J = jobs[blockIdx.x];
  kth_block(J.keys, J.flag, J.n, J.k, J.out_tau, J.out_ok, J.n_dev);
}

// ------------------------------------------------------------------ result set R

// R = {maybe && f32 >= thr}, thr = tau32 - margin2 (-inf when fewer than k sure entries exist);
// need64 = !sure
__global__ void k_build_r(long long n, const long long *cand_ids, const float *f32, const unsigned char *maybe,
                          const unsigned char *sure, const float *tau32, float margin2, RItem *R, unsigned *n_r,
                          const unsigned *n_dev) {
  if (n_dev && (long long)*n_dev < n) n = *n_dev;
  const float tau = *tau32;
  const float thr = isfinite(tau) ? tau - margin2 : -INFINITY;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
    const long long i = b + (threadIdx.x & 31);
    const bool take = (i < n) && maybe[i] && f32[i] >= thr;
    const unsigned p = apx_warp_reserve(n_r, take);
    if (take) {
      RItem it;
      it.s = (double)f32[i];
      it.id = cand_ids[i] & APX_ID_MASK;
      it.src = (int)i;
      it.alive = 1;
      it.is64 = 0;
      it.need64 = sure[i] ? 0 : 1;
      it.pad = 0;
      R[p] = it;
    }
  }
}

// ------------------------------------------------------------------ in-pass compaction
// Between the launches of a pass, a query whose candidate buffer fills up has its candidates
// rescored in FP32 (k_eval32, k_kth: tau32 = k-th largest FP32 objective among FP32-sure entries).
// k surely feasible compounds then have exact objectives >= B = tau32 - eps_f, so the final k-th
// exact objective is >= B: a candidate can still be a member only if its FP32 objective is >=
// B - eps_f = tau32 - 2 eps_f and its FP32 outputs lie in the box widened by eps, and a compound
// of a later launch only if its pass objective is >= B - delta_f. The buffer keeps the first kind
// (the key becomes the rescored objective, within eps_f <= delta_f of the exact one, so the selects
// between launches keep their guarantee; an entry becomes "sure" when the rescore finds it sure) and the
// admission threshold rises to the second, so the buffer holds about k entries plus the FP32 band
// after every compaction, whatever the width of the pass margin (Sec. 3.3 queue with the precision
// pattern's FP32 rescore moved into the pass).
// The rescore is FP32 (SIMT) or, when the library has its FP16 tables and the pass is BF16 or FP8,
// FP16 on the tensor cores; eps and eps_f above are then that format's margins (the argument holds
// for any rescore whose margin is below the pass's). Entries a previous compaction kept carry
// APX_SCORED_BIT: their key is already their rescored objective and they are inside the widened
// box (both rescores are deterministic), so only the entries appended since are rescored
// (k_split_scored lists them).
// Split step: entries with APX_SCORED_BIT get f32 = key, maybe = 1, sure = no APX_UNSURE_BIT; the
// others are listed (id, buffer position) for the FP32 rescore, their count -> *n_new.
__global__ void k_split_scored(const QuerySlot *Q, unsigned n_max, float *f32, unsigned char *maybe,
                               unsigned char *sure, long long *ids_new, int *pos_new, unsigned *n_new) {
  const unsigned n = min(Q->count, min(Q->cap, n_max));
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned b = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
    const unsigned i = b + (threadIdx.x & 31);
    const long long id = i < n ? Q->ids[i] : 0;
    const bool scored = (i < n) && (id & APX_SCORED_BIT);
    const bool fresh = (i < n) && !(id & APX_SCORED_BIT);
    if (scored) {
      f32[i] = Q->keys[i];
      maybe[i] = 1;
      sure[i] = (id & APX_UNSURE_BIT) ? 0 : 1;
    }
    const unsigned p = apx_warp_reserve(n_new, fresh);
    if (fresh) {
      ids_new[p] = id;
      pos_new[p] = (int)i;
    }
  }
}
// Keep step: surviving entries -> keys2/ids2 (order not kept), their count -> *kept.
__global__ void k_compact_keep(QuerySlot *Q, const float *f32, const unsigned char *maybe, const unsigned char *sure,
                               const float *tau32, const int *ok, float margin2, unsigned *kept, unsigned n_max) {
  const unsigned n = min(Q->count, min(Q->cap, n_max));
  const float tau = *tau32;
  const float thr = (*ok && isfinite(tau)) ? __fsub_rd(tau, margin2) : -INFINITY;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned b = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
    const unsigned i = b + (threadIdx.x & 31);
    const bool take = (i < n) && maybe[i] && f32[i] >= thr;
    const unsigned p = apx_warp_reserve(kept, take);
    if (take) {
      const long long id = Q->ids[i];
      Q->keys2[p] = f32[i];
      Q->ids2[p] = (sure[i] ? (id & ~APX_UNSURE_BIT) : id) | APX_SCORED_BIT;
    }
  }
}
// Apply step: keys2/ids2 [0, kept) back into the buffer, the new count, the admission floor
// B - delta_f, and the start guess marked verified when its admission threshold (tau_spec -
// 2 delta_f) was at or below that floor (every member of the top-k was then admitted).
__global__ void k_compact_apply(QuerySlot *Q, const unsigned *kept, const float *tau32, const int *ok, float eps_f) {
  const unsigned m = *kept;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    Q->keys[i] = Q->keys2[i];
    Q->ids[i] = Q->ids2[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Q->count = m;
    Q->count_compacted = m;
    const float tau = *tau32;
    if (*ok && isfinite(tau)) {
      const float B = __fsub_rd(tau, eps_f);
      const float floor_adm = __fsub_rd(B, Q->delta_f);
      if (floor_adm > Q->admit) Q->admit = floor_adm;
      if (isfinite(Q->tau_spec) && __fadd_rd(B, Q->delta_f) >= Q->tau_spec) Q->tau_spec = -INFINITY;
    }
  }
}

// list of R positions whose FP64 rescore is pending
__global__ void k_collect64(RItem *R, unsigned n, long long *ids64, int *pos64, unsigned *n64) {
  for (unsigned b = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += gridDim.x * blockDim.x) {
    const unsigned i = b + (threadIdx.x & 31);
    const bool take = (i < n) && R[i].alive && R[i].need64 && !R[i].is64;
    const unsigned p = apx_warp_reserve(n64, take);
    if (take) {
      ids64[p] = R[i].id;
      pos64[p] = (int)i;
    }
  }
}

// apply FP64 outputs: exact objective and box; drop infeasible
__global__ void k_apply64(RItem *R, const int *pos64, const double *out64, unsigned n64_max, const unsigned *n64_dev,
                          int n_out, const QuerySlot *Q, const double *lo, const double *hi,
                          double *out_rows /* [n_candidates x n_out], by src */, const float *out32, unsigned *obs) {
  const unsigned n64 = n64_dev ? min(n64_max, *n64_dev) : n64_max;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n64; i += gridDim.x * blockDim.x) {
    const double *o = out64 + (size_t)i * n_out;
    double f = 0.0;
    for (int j = 0; j < Q->n_obj; ++j) f += (double)Q->w[j] * o[j];
    bool ok = true;
    for (int c = 0; c < Q->n_cons; ++c) {
      const double v = o[Q->cons_idx[c]];
      ok = ok && (v >= lo[c]) && (v <= hi[c]);
    }
    RItem &it = R[pos64[i]];
    it.s = f;
    it.is64 = 1;
    it.alive = ok ? 1 : 0;
    for (int j = 0; j < n_out; ++j) out_rows[(size_t)it.src * n_out + j] = o[j];
    if (out32 && obs)  // observed FP32 error of every output on this member (rounded up to float)
      for (int j = 0; j < n_out; ++j) {
        const float e = __double2float_ru(fabs(o[j] - (double)out32[(size_t)it.src * n_out + j]));
        if (e > 0.f) atomicMax(obs + 1 + j, __float_as_uint(e));
      }
  }
}

// ------------------------------------------------------------------ bitonic sort of R
// order: alive first, then s desc, then id asc
// Order-preserving 64-bit key of a score (larger score, larger key; -0 and +0 equal), so the
// orderings compare integers: FP64 comparisons issue at a small fraction of the integer rate
// on this part. Dead items take key 0, below every score (-inf included).
__device__ __forceinline__ unsigned long long r_key(double s) {
  unsigned long long b = (unsigned long long)__double_as_longlong(s);
  if (b == 0x8000000000000000ull) b = 0ull;
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ bool r_before(const RItem &a, const RItem &b) {
  const unsigned long long ka = a.alive ? r_key(a.s) : 0ull, kb = b.alive ? r_key(b.s) : 0ull;
  if (a.alive != b.alive) return a.alive > b.alive;
  if (ka != kb) return ka > kb;
  return a.id < b.id;
}

__global__ void k_bitonic_global(RItem *R, unsigned n, unsigned j, unsigned kk, const unsigned *n_used) {
  if (n_used) {  // only the power-of-two prefix holding the used entries is sorted
    unsigned p2 = 2;
    while (p2 < *n_used) p2 <<= 1;
    if (kk > p2) return;
    n = min(n, p2);
  }
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned l = i ^ j;
    if (l > i) {
      const bool up = ((i & kk) == 0);
      RItem a = R[i], b = R[l];
      const bool swap = up ? r_before(b, a) : r_before(a, b);
      if (swap) {
        R[i] = b;
        R[l] = a;
      }
    }
  }
}

#define BITONIC_SMEM 2048
// every (kk, j) step with j < block inside blocks of `block` (power of two <= BITONIC_SMEM) elements.
// The network runs on the sort keys only, as separate arrays in shared memory (conflict-free
// 8-byte accesses): key (r_key(s), id) with dead items mapped to (0, max id), which reproduces the
// (alive, s desc, id asc) order, plus the item's position; the items are permuted once at the end.
// n_used (optional): sort just the smallest power of two p2 holding the *n_used leading entries
// (the rest is dead padding, already in its place at the end): blocks past p2 and stages past
// p2 do nothing, a block longer than p2 sorts its first p2 entries.
__global__ void __launch_bounds__(1024) k_bitonic_shared(RItem *R, unsigned block, unsigned kk_from, unsigned kk_to,
                                                         const unsigned *n_used) {
  __shared__ unsigned long long ks[BITONIC_SMEM];
  __shared__ long long kid[BITONIC_SMEM];
  __shared__ unsigned short ix[BITONIC_SMEM];
  if (n_used) {
    unsigned p2 = 2;
    while (p2 < *n_used) p2 <<= 1;
    if (blockIdx.x * block >= p2 || kk_from > p2) return;
    if (p2 < block) block = p2;
    kk_to = min(kk_to, p2);
  }
  const unsigned base = blockIdx.x * block;
  for (unsigned t = threadIdx.x; t < block; t += blockDim.x) {
    const RItem it = R[base + t];
    ks[t] = it.alive ? r_key(it.s) : 0ull;
    kid[t] = it.alive ? it.id : 0x7fffffffffffffffLL;
    ix[t] = (unsigned short)t;
  }
  __syncthreads();
  for (unsigned kk = kk_from; kk <= kk_to; kk <<= 1) {
    for (unsigned j = min(kk >> 1, block >> 1); j > 0; j >>= 1) {
      for (unsigned h = threadIdx.x; h < (block >> 1); h += blockDim.x) {
        const unsigned t = ((h & ~(j - 1)) << 1) | (h & (j - 1));  // the pair (t, t + j)
        const unsigned l = t + j;
        const bool up = (((base + t) & kk) == 0);
        const unsigned long long sa = ks[t], sb = ks[l];
        const long long ia = kid[t], ib = kid[l];
        const bool b_first = (sb > sa) || (sb == sa && ib < ia);
        const bool a_first = (sa > sb) || (sa == sb && ia < ib);
        if (up ? b_first : a_first) {
          ks[t] = sb;
          ks[l] = sa;
          kid[t] = ib;
          kid[l] = ia;
          const unsigned short x = ix[t];
          ix[t] = ix[l];
          ix[l] = x;
        }
      }
      __syncthreads();
    }
  }
  // permute the items: read every source first, then write
  RItem mine[BITONIC_SMEM / 1024];
  unsigned c = 0;
  for (unsigned t = threadIdx.x; t < block; t += blockDim.x) mine[c++] = R[base + ix[t]];
  __syncthreads();
  c = 0;
  for (unsigned t = threadIdx.x; t < block; t += blockDim.x) R[base + t] = mine[c++];
}

__global__ void k_pad_r(RItem *R, unsigned from, unsigned to) {
  for (unsigned i = from + blockIdx.x * blockDim.x + threadIdx.x; i < to; i += gridDim.x * blockDim.x) {
    RItem it;
    it.s = -INFINITY;
    it.id = 0x3fffffffffffffffLL;
    it.src = -1;
    it.alive = 0;
    it.is64 = 1;
    it.need64 = 0;
    it.pad = 0;
    R[i] = it;
  }
}

// Pads R[*n_used, to) with dead items, the used count read on the device (no host round trip).
__global__ void k_pad_r_dev(RItem *R, const unsigned *n_used, unsigned to) {
  const unsigned from = *n_used;
  for (unsigned i = from + blockIdx.x * blockDim.x + threadIdx.x; i < to; i += gridDim.x * blockDim.x) {
    RItem it;
    it.s = -INFINITY;
    it.id = 0x3fffffffffffffffLL;
    it.src = -1;
    it.alive = 0;
    it.is64 = 1;
    it.need64 = 0;
    it.pad = 0;
    R[i] = it;
  }
}

cudaError_t apx_launch_pad_r_dev(RItem *R, const unsigned *n_used, unsigned to, cudaStream_t st) {
  if (to == 0) return cudaSuccess;
  apx_count_launch();
  k_pad_r_dev<<<std::min<unsigned>((to + 255) / 256, 148u * 4u), 256, 0, st>>>(R, n_used, to);
  return cudaGetLastError();
}

// Sorts R[0, n_pow2) (n_pow2 a power of two) into (alive, s desc, id asc) order. With n_dev (a
// device count of leading used entries; the rest dead padding) only the power-of-two prefix that
// holds them is sorted, whatever n_pow2 the launches were sized for.
cudaError_t apx_sort_r(RItem *R, unsigned n_used, unsigned n_pow2, cudaStream_t st, const unsigned *n_dev) {
  if (n_pow2 < 2) return cudaSuccess;
  if (n_used < n_pow2) {
    apx_count_launch();
    k_pad_r<<<64, 256, 0, st>>>(R, n_used, n_pow2);
  }
  if (n_pow2 <= BITONIC_SMEM) {
    apx_count_launch();
    // one thread per compare-exchange pair (fewer idle warps at every barrier)
    k_bitonic_shared<<<1, std::max(32u, n_pow2 / 2), 0, st>>>(R, n_pow2, 2, n_pow2, n_dev);
    return cudaGetLastError();
  }
  const unsigned nb = n_pow2 / BITONIC_SMEM;
  apx_count_launch();
  k_bitonic_shared<<<nb, 1024, 0, st>>>(R, BITONIC_SMEM, 2, BITONIC_SMEM, n_dev);
  for (unsigned kk = BITONIC_SMEM * 2; kk <= n_pow2; kk <<= 1) {
    for (unsigned j = kk >> 1; j >= BITONIC_SMEM; j >>= 1) {
      apx_count_launch();
      k_bitonic_global<<<std::min<unsigned>(nb * 8, 148u * 16u), 256, 0, st>>>(R, n_pow2, j, kk, n_dev);
    }
    apx_count_launch();
    k_bitonic_shared<<<nb, 1024, 0, st>>>(R, BITONIC_SMEM, kk, kk, n_dev);
  }
  return cudaGetLastError();
}

// Marks for FP64 every alive, not-yet-FP64 item whose score is within tol of the k-th score (the
// top-k boundary band, on either side of it): only those can change the returned set. Items
// well inside keep their FP32 score; near-ties among them are ordered by it.
// n_used (optional, a device count <= n): entries of R that came from the candidates; the
// rest is padding.
__global__ void k_mark_ties(RItem *R, unsigned n, unsigned kp1, long long k, double tol, unsigned *n_marked,
                            const unsigned *n_used) {
  __shared__ double sk;
  if (threadIdx.x == 0) {
    const unsigned nu = n_used ? min(n, *n_used) : n;
    const unsigned kk = (unsigned)(k < (long long)nu ? k : (long long)nu) - 1u;
    sk = (nu > 0 && R[kk].alive) ? R[kk].s : -INFINITY;
  }
  __syncthreads();
  (void)kp1;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    RItem &it = R[i];
    if (!it.alive || it.is64) continue;
    if (fabs(it.s - sk) <= tol) {
      it.need64 = 1;
      atomicAdd(n_marked, 1u);
    }
  }
}

// The same band marked around a reference score already on the device (the FP32 k-th score),
// without sorting first: used before the first FP64 round; the band is re-marked around the
// sorted k-th score after every round, so a differing reference only costs another round.
__global__ void k_mark_near(RItem *R, unsigned n, const float *ref, double tol, unsigned *n_marked) {
  const double sk = (double)*ref;
  if (!(sk > -INFINITY)) return;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    RItem &it = R[i];
    if (!it.alive || it.is64) continue;
    if (fabs(it.s - sk) <= tol) {
      it.need64 = 1;
      atomicAdd(n_marked, 1u);
    }
  }
}

cudaError_t apx_launch_mark_near(RItem *R, unsigned n, const float *ref, double tol, unsigned *n_marked,
                                 cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  apx_count_launch();
  k_mark_near<<<std::min<unsigned>((n + 255) / 256, 148u * 16u), 256, 0, st>>>(R, n, ref, tol, n_marked);
  return cudaGetLastError();
}

// Final rows: ids, reaction, synthons, objective, outputs (FP64 where rescored, else FP32)
__global__ void k_emit(const RItem *R, unsigned n_max, const unsigned *n_alive, const __grid_constant__ DevTables T,
                       const float *out32, const double *out64_rows, long long *ids, int *rxn, long long *syn,
                       double *obj, double *outs) {
  const unsigned n_final = n_alive ? min(n_max, *n_alive) : n_max;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n_final; i += gridDim.x * blockDim.x) {
    const RItem it = R[i];
    const long long id = it.id;
    int lo = 0, hi = T.n_rx - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (T.id_first[mid] <= id) lo = mid; else hi = mid - 1;
    }
    const RxnPlan *p = T.rx + lo;
    long long rem = id - p->id_first;
    long long s[APEX_MAX_SLOTS];
    for (int j = APEX_MAX_SLOTS - 1; j >= 0; --j) {
      if (j < p->n_slots) {
        s[j] = rem % p->slot_size[j];
        rem /= p->slot_size[j];
      } else {
        s[j] = -1;
      }
    }
    ids[i] = id;
    rxn[i] = lo;
    for (int j = 0; j < APEX_MAX_SLOTS; ++j) syn[(size_t)i * APEX_MAX_SLOTS + j] = s[j];
    obj[i] = it.s;
    // outputs are kept per candidate (src), so the permutation of R by the sorts does not matter
    for (int j = 0; j < T.n_out; ++j)
      outs[(size_t)i * T.n_out + j] =
          it.is64 ? out64_rows[(size_t)it.src * T.n_out + j] : (double)out32[(size_t)it.src * T.n_out + j];
  }
}

// n_dev (optional): the actual count on the device, at most n (grids are sized for n)
cudaError_t apx_launch_eval32(const EvalArgs &a, long long n, float *f32, unsigned char *maybe, unsigned char *sure,
                              cudaStream_t st, const unsigned *n_dev) {
  if (n <= 0) return cudaSuccess;
  apx_count_launch();
  k_eval32<<<(unsigned)std::min<long long>((n + 255) / 256, 148 * 16), 256, 0, st>>>(a, n, f32, maybe, sure, n_dev);
  return cudaGetLastError();
}
cudaError_t apx_launch_kth(const float *keys, const unsigned char *flag, long long n, long long k, float *out_tau,
                           int *out_ok, cudaStream_t st, const unsigned *n_dev) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_kth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SEL_SMEM_KEYS * sizeof(unsigned)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  apx_count_launch();
  k_kth<<<1, SEL_THREADS, SEL_SMEM_KEYS * sizeof(unsigned), st>>>(keys, flag, n, k, out_tau, out_ok, n_dev);
  return cudaGetLastError();
}
cudaError_t apx_launch_kth_multi(const KthJob *jobs, int n_jobs, cudaStream_t st) {
  if (n_jobs <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_kth_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(SEL_SMEM_KEYS * sizeof(unsigned)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  apx_count_launch();
  k_kth_multi<<<n_jobs, SEL_THREADS, SEL_SMEM_KEYS * sizeof(unsigned), st>>>(jobs);
  return cudaGetLastError();
}
cudaError_t apx_launch_build_r(long long n, const long long *cand_ids, const float *f32, const unsigned char *maybe,
                               const unsigned char *sure, const float *tau32, float margin2, RItem *R, unsigned *n_r,
                               cudaStream_t st, const unsigned *n_dev) {
  if (n <= 0) return cudaSuccess;
  apx_count_launch();
  k_build_r<<<(unsigned)std::min<long long>((n + 255) / 256, 148 * 16), 256, 0, st>>>(n, cand_ids, f32, maybe, sure, tau32,
                                                                                 margin2, R, n_r, n_dev);
  return cudaGetLastError();
}
// n_max: entries the scratch arrays (f32, maybe, sure) cover; the slot's count decides how many
// are used. kept: a device counter, zeroed here.
cudaError_t apx_launch_split_scored(const QuerySlot *Q, unsigned n_max, float *f32, unsigned char *maybe,
                                    unsigned char *sure, long long *ids_new, int *pos_new, unsigned *n_new, int n_sm,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(n_new, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = std::max(1u, std::min<unsigned>((n_max + 255) / 256, (unsigned)n_sm * 4u));
  apx_count_launch();
  k_split_scored<<<grid, 256, 0, st>>>(Q, n_max, f32, maybe, sure, ids_new, pos_new, n_new);
  return cudaGetLastError();
}
cudaError_t apx_launch_compact(QuerySlot *Q, const float *f32, const unsigned char *maybe, const unsigned char *sure,
                               const float *tau32, const int *ok, float margin2, float eps_f, unsigned *kept,
                               unsigned n_max, int n_sm, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(kept, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = std::max(1u, std::min<unsigned>((n_max + 255) / 256, (unsigned)n_sm * 4u));
  apx_count_launch(2);
  k_compact_keep<<<grid, 256, 0, st>>>(Q, f32, maybe, sure, tau32, ok, margin2, kept, n_max);
  k_compact_apply<<<grid, 256, 0, st>>>(Q, kept, tau32, ok, eps_f);
  return cudaGetLastError();
}
cudaError_t apx_launch_collect64(RItem *R, unsigned n, long long *ids64, int *pos64, unsigned *n64, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  apx_count_launch();
  k_collect64<<<std::min<unsigned>((n + 255) / 256, 148u * 16u), 256, 0, st>>>(R, n, ids64, pos64, n64);
  return cudaGetLastError();
}
// n64_dev (optional): device count, at most n64
cudaError_t apx_launch_apply64(RItem *R, const int *pos64, const double *out64, unsigned n64, const unsigned *n64_dev,
                               int n_out, const QuerySlot *Q, const double *lo, const double *hi, double *out_rows,
                               cudaStream_t st, const float *out32, unsigned *obs) {
  if (n64 == 0) return cudaSuccess;
  apx_count_launch();
  k_apply64<<<std::min<unsigned>((n64 + 255) / 256, 148u * 16u), 256, 0, st>>>(R, pos64, out64, n64, n64_dev, n_out, Q,
                                                                                lo, hi, out_rows, out32, obs);
  return cudaGetLastError();
}
cudaError_t apx_launch_mark(RItem *R, unsigned n, unsigned kp1, long long k, double tol, unsigned *n_marked,
                            cudaStream_t st, const unsigned *n_used) {
  if (n == 0) return cudaSuccess;
  apx_count_launch();
  k_mark_ties<<<std::min<unsigned>((n + 255) / 256 + 1, 148u * 16u), 256, 0, st>>>(R, n, kp1, k, tol, n_marked,
                                                                                   n_used);
  return cudaGetLastError();
}
// rows emitted: min(n_final, *n_alive) (n_alive optional, a device count)
cudaError_t apx_launch_emit(const RItem *R, unsigned n_final, const unsigned *n_alive, const DevTables &T,
                            const float *out32, const double *out64_rows, long long *ids, int *rxn, long long *syn,
                            double *obj, double *outs, cudaStream_t st) {
  if (n_final == 0) return cudaSuccess;
  apx_count_launch();
  k_emit<<<std::min<unsigned>((n_final + 127) / 128, 148u * 4u), 128, 0, st>>>(R, n_final, n_alive, T, out32, out64_rows,
                                                                               ids, rxn, syn, obj, outs);
  return cudaGetLastError();
}

// out[0] += alive entries of R[0, n); out[1] (optional) += entries rescored in FP64
__global__ void k_count_alive(const RItem *R, unsigned n, unsigned *out, unsigned *out64) {
  unsigned c = 0, c64 = 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const RItem it = R[i];
    c += it.alive;
    c64 += (it.is64 && it.src >= 0) ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, o);
    c64 += __shfl_down_sync(0xffffffffu, c64, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c) atomicAdd(out, c);
    if (out64 && c64) atomicAdd(out64, c64);
  }
}

// alive entries of R[0, n) added to d_out[0] and FP64-rescored ones to d_out[1] (both zeroed by
// the caller), no host synchronization
cudaError_t apx_launch_count_alive(const RItem *R, unsigned n, unsigned *d_out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  apx_count_launch();
  k_count_alive<<<std::min<unsigned>((n + 255) / 256, 148u * 4u), 256, 0, st>>>(R, n, d_out, d_out + 1);
  return cudaGetLastError();
}

int apx_count_alive(const RItem *R, unsigned n, cudaStream_t st, unsigned *d_tmp, cudaError_t *e) {
  unsigned h = 0;
  *e = cudaMemsetAsync(d_tmp, 0, sizeof(unsigned), st);
  if (*e != cudaSuccess) return 0;
  apx_count_launch();
  k_count_alive<<<std::min<unsigned>((n + 255) / 256, 148u * 4u), 256, 0, st>>>(R, n, d_tmp, nullptr);
  *e = cudaGetLastError();
  if (*e != cudaSuccess) return 0;
  *e = cudaMemcpyAsync(&h, d_tmp, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (*e != cudaSuccess) return 0;
  *e = cudaStreamSynchronize(st);
  return (int)h;
}

// ------------------------------------------------------------------ speculative start threshold
// SplitMix64 output function (Steele, Lea and Flood, 2014): a counter-based 64-bit generator.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// S compound ids drawn uniformly from the scope: pre[] = prefix counts of the scope's reactions
// rxn[] (n_sub + 1 entries, pre[n_sub] = scope size), id_first[] = first id of every reaction.
__global__ void k_spec_ids(const int *rxn, const long long *pre, int n_sub, const long long *id_first, long long scope_n,
                           unsigned long long seed, long long S, long long *ids) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
    const long long u = (long long)(splitmix64(seed + (unsigned long long)i * 0x2545f4914f6cdd1dull) %
                                    (unsigned long long)scope_n);
    int lo = 0, hi = n_sub - 1;  // last r with pre[r] <= u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= u) lo = mid; else hi = mid - 1;
    }
    ids[i] = id_first[rxn[lo]] + (u - pre[lo]);
  }
}

// Objective of the feasible sample entries (exact boxes on the sample's outputs), its rank-th
// largest value, and the query slot's start and admission thresholds (-inf when fewer than rank
// sample entries are feasible). One CTA; samples of up to SPEC_SMEM_KEYS entries are selected
// from shared memory.
#define SPEC_SMEM_KEYS 16384
// Rank-r largest of at most 16 * SEL_THREADS keys (order-preserving bits, 0 = excluded) for a small
// rank: r rounds of a block-wide maximum, each removing one instance of it (so equal keys count
// with their multiplicity). Keys stay in registers. Returns false when fewer than r keys are
// non-zero.
#define SPEC_FAST_RANK 32
__device__ bool block_rank_small(const unsigned *bits, long long n, long long r, unsigned *out_bits) {
  __shared__ unsigned wmax[SEL_THREADS / 32];
  __shared__ unsigned bmax;
  __shared__ int claimed;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const long long i = (long long)tid + (long long)j * SEL_THREADS;
    v[j] = i < n ? bits[i] : 0u;
  }
  unsigned last = 0;
  bool ok = true;
  for (long long round = 0; round < r; ++round) {
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) m = max(m, v[j]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) wmax[warp] = m;
    if (tid == 0) claimed = 0;
    __syncthreads();
    if (warp == 0) {
      unsigned x = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0u;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, off));
      if (lane == 0) bmax = x;
    }
    __syncthreads();
    const unsigned M = bmax;
    if (M == 0u) {  // uniform: fewer than r keys
      ok = false;
      break;
    }
    last = M;
    bool has = false;
#pragma unroll
    for (int j = 0; j < 16; ++j) has = has || v[j] == M;
    if (has && atomicCAS(&claimed, 0, 1) == 0) {  // one instance leaves
      bool gone = false;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (!gone && v[j] == M) {
          v[j] = 0u;
          gone = true;
        }
    }
    __syncthreads();
  }
  *out_bits = last;
  return ok;
}

__global__ void __launch_bounds__(SEL_THREADS) k_spec_select(const float *out, long long S, const __grid_constant__ SpecArgs a,
                                                             float *keys, unsigned char *flag, QuerySlot *slot) {
  if (a.bits_in && S <= 16LL * SEL_THREADS && a.rank <= SPEC_FAST_RANK && blockDim.x == SEL_THREADS) {
    unsigned bits;  // keys already formed by the scoring kernel; a small rank
    const bool ok = block_rank_small(reinterpret_cast<const unsigned *>(out), S, a.rank, &bits);
    if (threadIdx.x == 0) {
      const float t = ok ? apx_bits_key(bits) : -INFINITY;
      slot->tau_spec = t;
      slot->admit = ok ? t - a.margin2 : -INFINITY;
    }
    return;
  }
  extern __shared__ unsigned spec_bits[];  // the sample's objective bits, 0 = infeasible
  const bool in_smem = S <= SPEC_SMEM_KEYS;
  // the boxes as FP32 bounds that decide exactly like the FP64 ones for FP32 values: the smallest
  // float >= lo and the largest float <= hi (FP64 compares run at a small fraction of the FP32 rate)
  __shared__ float lo_f[APEX_MAX_CONSTRAINTS], hi_f[APEX_MAX_CONSTRAINTS];
  if (threadIdx.x < (unsigned)a.n_cons) {
    lo_f[threadIdx.x] = __double2float_ru(a.lo[threadIdx.x]);
    hi_f[threadIdx.x] = __double2float_rd(a.hi[threadIdx.x]);
  }
  __syncthreads();
  for (long long i = threadIdx.x; i < S; i += blockDim.x) {
    if (a.bits_in) {  // keys already formed by the scoring kernel
      const unsigned kb = reinterpret_cast<const unsigned *>(out)[i];
      if (in_smem) {
        spec_bits[i] = kb;
      } else {
        keys[i] = kb ? apx_bits_key(kb) : 0.f;
        flag[i] = kb != 0u;
      }
      continue;
    }
    const float *o = out + i * a.n_out;
    bool ok = true;
    for (int c = 0; c < a.n_cons; ++c) {
      const float v = o[a.cons_idx[c]];
      ok = ok && v >= lo_f[c] && v <= hi_f[c];
    }
    float f = 0.f;
    for (int j = 0; j < a.n_obj; ++j) f = fmaf(a.w[j], o[j], f);
    if (in_smem) {
      spec_bits[i] = ok ? apx_key_bits(f) : 0u;
    } else {
      keys[i] = f;
      flag[i] = ok;
    }
  }
  __syncthreads();
  unsigned bits;
  const bool ok = in_smem ? block_kth_largest(SelSmem{spec_bits}, S, a.rank, &bits, nullptr)
                          : block_kth_largest(SelSrc{keys, nullptr, flag}, S, a.rank, &bits, nullptr);
  if (threadIdx.x == 0) {
    const float t = ok ? apx_bits_key(bits) : -INFINITY;
    slot->tau_spec = t;
    slot->admit = ok ? t - a.margin2 : -INFINITY;
  }
}

cudaError_t apx_launch_spec_ids(const int *rxn, const long long *pre, int n_sub, const long long *id_first,
                                long long scope_n, unsigned long long seed, long long S, long long *ids, cudaStream_t st) {
  if (S <= 0 || n_sub <= 0) return cudaSuccess;
  apx_count_launch();
  k_spec_ids<<<(unsigned)std::min<long long>((S + 255) / 256, 148 * 4), 256, 0, st>>>(rxn, pre, n_sub, id_first, scope_n,
                                                                                    seed, S, ids);
  return cudaGetLastError();
}

cudaError_t apx_launch_spec_select(const float *out, long long S, const SpecArgs &a, float *keys, unsigned char *flag,
                                   QuerySlot *slot, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_spec_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(SPEC_SMEM_KEYS * sizeof(unsigned)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  apx_count_launch();
  const size_t smem = S <= SPEC_SMEM_KEYS ? (size_t)S * sizeof(unsigned) : 0;
  k_spec_select<<<1, SEL_THREADS, smem, st>>>(out, S, a, keys, flag, slot);
  return cudaGetLastError();
}
