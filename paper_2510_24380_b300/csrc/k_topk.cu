// k_topk.cu -- standalone top-k selection on device arrays (apex_topk_select).
//
// The k largest keys, ties broken by the smaller id, returned in (key desc, id asc) order: the
// result a size-k priority queue over (key, id) holds after the whole stream (Sec. 3.3), found
// here as a multi-CTA radix select instead of a heap:
//   stage 0: four 8-bit passes over the order-preserving key bits find the k-th key tau and how
//            many entries equal to tau still belong to the top k;
//   stage 1: eight 8-bit passes over ~id among the entries equal to tau find the largest id that
//            still belongs (smallest ids first);
//   compaction of the members, then a bitonic sort of the k members.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include "common.cuh"

struct SelState {
  unsigned long long prefix, mask;
  long long kk;
  unsigned tau;
  unsigned pad;
  unsigned long long id_max;  // largest member id among the entries equal to tau
  unsigned count;             // members written
  unsigned pad2;
  unsigned long long hist[256];
};

__device__ __forceinline__ unsigned long long sel_value(int stage, float key, long long id, unsigned tau, bool &use) {
  const unsigned kb = apx_key_bits(key);
  if (stage == 0) {
    use = true;
    return (unsigned long long)kb;
  }
  use = (kb == tau);
  return ~(unsigned long long)id;
}

__global__ void k_sel_init(SelState *S, long long k) {
  if (threadIdx.x == 0) {
    S->prefix = 0;
    S->mask = 0;
    S->kk = k;
    S->tau = 0;
    S->id_max = 0;
    S->count = 0;
  }
  for (int d = threadIdx.x; d < 256; d += blockDim.x) S->hist[d] = 0;
}

__global__ void k_sel_hist(const float *keys, const long long *ids, long long n, SelState *S, int stage, int shift) {
  __shared__ unsigned long long h[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
  __syncthreads();
  const unsigned long long prefix = S->prefix, mask = S->mask;
  const unsigned tau = S->tau;
  const unsigned lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
    const long long i = b + lane;
    bool use = false;
    unsigned long long v = 0;
    if (i < n) v = sel_value(stage, keys[i], ids[i], tau, use);
    use = use && (v & mask) == prefix;
    const unsigned dig = use ? (unsigned)((v >> shift) & 255ull) : 256u;
    const unsigned grp = __match_any_sync(0xffffffffu, dig);   // merge lanes with equal digits
    if (use && (int)lane == __ffs(grp) - 1) atomicAdd(&h[dig], (unsigned long long)__popc(grp));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x)
    if (h[d]) atomicAdd(&S->hist[d], h[d]);
}

// one thread: digit holding the kk-th largest value, then clears the histogram
__global__ void k_sel_scan(SelState *S, int shift, int last_of_stage, int stage) {
  if (threadIdx.x != 0) return;
  long long kk = S->kk;
  unsigned long long cum = 0;
  int dsel = 0;
  for (int d = 255; d >= 0; --d) {
    if (cum + S->hist[d] >= (unsigned long long)kk) {
      dsel = d;
      break;
    }
    cum += S->hist[d];
  }
  S->kk = kk - (long long)cum;
  S->prefix |= (unsigned long long)dsel << shift;
  S->mask |= 255ull << shift;
  for (int d = 0; d < 256; ++d) S->hist[d] = 0;
  if (last_of_stage && stage == 0) {
    S->tau = (unsigned)S->prefix;
    S->prefix = 0;
    S->mask = 0;  // stage 1 keeps kk = members still needed among the ties
  } else if (last_of_stage && stage == 1) {
    S->id_max = ~S->prefix;
  }
}

__global__ void k_sel_compact(const float *keys, const long long *ids, long long n, SelState *S, long long k,
                              RItem *out) {
  const unsigned tau = S->tau;
  const long long id_max = (long long)S->id_max;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
    const long long i = b + (threadIdx.x & 31);
    bool member = false;
    float key = 0.f;
    long long id = 0;
    if (i < n) {
      key = keys[i];
      id = ids[i];
      const unsigned kb = apx_key_bits(key);
      member = kb > tau || (kb == tau && id <= id_max);
    }
    const unsigned p = apx_warp_reserve(&S->count, member);
    if (member && p < (unsigned long long)k) {
      RItem it;
      it.s = (double)key;
      it.id = id;
      it.src = 0;
      it.alive = 1;
      it.is64 = 1;
      it.need64 = 0;
      it.pad = 0;
      out[p] = it;
    }
  }
}

__global__ void k_sel_write(const RItem *R, long long k, float *out_keys, long long *out_ids) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k; i += (long long)gridDim.x * blockDim.x) {
    out_keys[i] = (float)R[i].s;
    out_ids[i] = R[i].id;
  }
}

cudaError_t apx_sort_r(RItem *R, unsigned n_used, unsigned n_pow2, cudaStream_t st, const unsigned *n_dev = nullptr);

// Runs the selection with caller-provided scratch (state + a RItem buffer of n_pow2 >= k entries).
cudaError_t apx_topk_select_run(const float *keys, const long long *ids, long long n, long long k, float *out_keys,
                                long long *out_ids, SelState *S, RItem *R, unsigned n_pow2, cudaStream_t st) {
  const int grid = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 148 * 8));
  apx_count_launch();
  k_sel_init<<<1, 256, 0, st>>>(S, k);
  for (int stage = 0; stage < 2; ++stage) {
    const int passes = stage == 0 ? 4 : 8;
    for (int p = passes - 1; p >= 0; --p) {
      apx_count_launch();
      k_sel_hist<<<grid, 256, 0, st>>>(keys, ids, n, S, stage, 8 * p);
      apx_count_launch();
      k_sel_scan<<<1, 32, 0, st>>>(S, 8 * p, p == 0, stage);
    }
  }
  apx_count_launch();
  k_sel_compact<<<grid, 256, 0, st>>>(keys, ids, n, S, k, R);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = apx_sort_r(R, (unsigned)k, n_pow2, st);
  if (e != cudaSuccess) return e;
  apx_count_launch();
  k_sel_write<<<(unsigned)std::min<long long>((k + 255) / 256, 148 * 4), 256, 0, st>>>(R, k, out_keys, out_ids);
  return cudaGetLastError();
}

size_t apx_sel_state_bytes() { return sizeof(SelState); }

apex_status apx_fail(apex_status code, const char *msg);

extern "C" apex_status apex_topk_select(const float *keys, const int64_t *ids, int64_t n, int64_t k, float *out_keys,
                                        int64_t *out_ids, int64_t *n_out, void *cuda_stream) {
  if (n < 0 || k < 1 || !n_out || (n > 0 && (!keys || !ids || !out_keys || !out_ids)))
    return apx_fail(APEX_EINVAL, "topk_select: bad arguments");
  if (k > (1LL << 26)) return apx_fail(APEX_EINVAL, "topk_select: k above 2^26");
  *n_out = 0;
  if (n == 0) return APEX_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const long long ke = std::min<long long>(k, n);
  unsigned np = 2;
  while ((long long)np < ke) np <<= 1;
  SelState *S = nullptr;
  RItem *R = nullptr;
  if (cudaMalloc(&S, sizeof(SelState)) != cudaSuccess) return apx_fail(APEX_ENOMEM, "topk_select: cudaMalloc failed");
  if (cudaMalloc(&R, sizeof(RItem) * np) != cudaSuccess) {
    cudaFree(S);
    return apx_fail(APEX_ENOMEM, "topk_select: cudaMalloc failed");
  }
  cudaError_t e = apx_topk_select_run(keys, (const long long *)ids, n, ke, out_keys, (long long *)out_ids, S, R, np, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(S);
  cudaFree(R);
  if (e != cudaSuccess) return apx_fail(APEX_ECUDA, cudaGetErrorString(e));
  *n_out = ke;
  return APEX_OK;
}

// ------------------------------------------------------------------ variant without allocation
// Some callers cannot allocate device memory at the point where they need a selection: code
// that runs under a caller-owned memory pool or arena that forbids outside allocations, code
// inside a host callback or a real-time loop where cudaMalloc's implicit synchronization and
// latency are not acceptable, or plugins whose host framework owns every allocation. For them
// the scratch of apex_topk_select (selection state + sort buffer) lives in this file-scope
// device array instead, sized for k <= APEX_SELECT_NOALLOC_MAX_K. Every GPU that loads the
// library holds it until the process exits.
#define APX_SEL_STATE_SLOT 4096
static_assert(sizeof(SelState) <= APX_SEL_STATE_SLOT, "selection state exceeds its slot");
#define APX_NOALLOC_BYTES ((size_t)APX_SEL_STATE_SLOT + (size_t)APEX_SELECT_NOALLOC_MAX_K * sizeof(RItem))
static __device__ __align__(256) unsigned char g_select_scratch[APX_NOALLOC_BYTES];

#define APX_MAX_DEVICES 64
static void *g_select_scratch_dev[APX_MAX_DEVICES] = {nullptr};
static std::mutex g_select_scratch_mu;

extern "C" apex_status apex_topk_select_noalloc(const float *keys, const int64_t *ids, int64_t n, int64_t k,
                                                float *out_keys, int64_t *out_ids, int64_t *n_out, void *cuda_stream) {
  if (n < 0 || k < 1 || !n_out || (n > 0 && (!keys || !ids || !out_keys || !out_ids)))
    return apx_fail(APEX_EINVAL, "topk_select_noalloc: bad arguments");
  const long long ke = std::min<long long>(k, n);
  if (ke > APEX_SELECT_NOALLOC_MAX_K)
    return apx_fail(APEX_EINVAL, "topk_select_noalloc: min(k, n) exceeds the static scratch limit "
                                 "APEX_SELECT_NOALLOC_MAX_K (65536); use apex_topk_select");
  *n_out = 0;
  if (n == 0) return APEX_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= APX_MAX_DEVICES)
    return apx_fail(APEX_ECUDA, "topk_select_noalloc: no current CUDA device");
  void *base = nullptr;
  {
    // one-time set-up per device, with that device current: the device address of the array
    // (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> g(g_select_scratch_mu);
    if (!g_select_scratch_dev[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_select_scratch);
      if (e != cudaSuccess || !p)
        return apx_fail(APEX_ECUDA, "topk_select_noalloc: cudaGetSymbolAddress failed");
      g_select_scratch_dev[dev] = p;
    }
    base = g_select_scratch_dev[dev];
  }
  unsigned np = 2;
  while ((long long)np < ke) np <<= 1;
  SelState *S = reinterpret_cast<SelState *>(base);
  RItem *R = reinterpret_cast<RItem *>(static_cast<unsigned char *>(base) + APX_SEL_STATE_SLOT);
  // k_sel_init clears the selection state; the sort buffer is fully rewritten by each call
  cudaError_t e = apx_topk_select_run(keys, (const long long *)ids, n, ke, out_keys, (long long *)out_ids, S, R, np,
                                      (cudaStream_t)cuda_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return apx_fail(APEX_ECUDA, cudaGetErrorString(e));
  *n_out = ke;
  return APEX_OK;
}
