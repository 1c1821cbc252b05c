// k_fp32.cu -- FP32 "plain" path on the CUDA cores (SIMT FFMA), generic dense head.
//
// One CTA (256 threads) processes tiles of 128 compounds:
//   layer 1 (structure-exploiting, Eq. apex generalized to W_1): z_1 = sum_j P[t, j, s_j]
//     with P = W_1 u (+ b_1 on slot-1 rows) precomputed per synthon, then the activation;
//   layers 2..L: out = act(W_l a + b_l) as a register-tiled SIMT GEMM over the tile
//     (activations kept transposed in shared memory, W_l^T streamed in 16-row K-chunks);
//   epilogue: the queries (objective, boxes, admission) or a plain write of the outputs.
// Row sources: (a) enumeration work items of a LaunchPlan (inner block x outer run, see
// common.cuh), (b) a list of compound ids (candidate rescoring and calibration).
#include "common.cuh"

#define F32_AT_STRIDE 132   // floats per row of the transposed activation tile (128 + pad)
#define F32_KC 16           // K rows of W^T per stage

struct F32Smem {
  float AT[256][F32_AT_STRIDE];      // AT[k][row]
  float Wc[2][F32_KC][256];          // W^T chunk double buffer
};

__device__ __forceinline__ float f32_act(int act, float z) {
  if (act == APEX_ACT_RELU) return z > 0.f ? z : 0.f;
  if (act == APEX_ACT_SILU) return z / (1.0f + expf(-z));
  return z;
}

// Row sources of tile row r: the table rows to sum, validity and global id.
__device__ __forceinline__ int f32_row_sources(const DevTables &T, int mode, const RxnPlan *rp, long long q0, long long o,
                                               const long long *ids, long long id0, long long n_ids, int r,
                                               long long (&rows)[APEX_MAX_SLOTS], bool &valid, long long &id) {
  int nrows = 0;
  valid = false;
  id = -1;
  if (mode == 0) {
    const long long q = q0 + r;
    valid = q < rp->n_inner;
    if (valid) {
      long long rem = q;
      for (int j = rp->n_inner_slots - 1; j >= 0; --j) {
        const long long sz = rp->inner_size[j];
        rows[nrows++] = rp->inner_row[j] + rem % sz;
        rem /= sz;
      }
      if (rp->outer_row >= 0) rows[nrows++] = rp->outer_row + o;
      id = rp->id_first + q * rp->inner_stride + o * rp->outer_stride;
    }
  } else {
    const long long i = id0 + r;
    valid = i < n_ids;
    if (valid) {
      id = ids[i] & APX_ID_MASK;
      int lo = 0, hi = T.n_rx - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.id_first[mid] <= id) lo = mid; else hi = mid - 1;
      }
      const RxnPlan *p = T.rx + lo;
      long long rem = id - p->id_first;
      for (int j = p->n_slots - 1; j >= 0; --j) {
        const long long sz = p->slot_size[j];
        rows[nrows++] = p->slot_row[j] + rem % sz;
        rem /= sz;
      }
    }
  }
  return nrows;
}

// Writes z_1 (activated unless the head has a single layer) for the tile rows into AT.
// Each warp builds two rows at a time; lanes stride over the columns (coalesced 128 B loads),
// and every load of both rows is issued before the sums are formed.
__device__ void f32_build_layer1(F32Smem &S, const DevTables &T, int mode, const RxnPlan *rp, long long q0, long long o,
                                 const long long *ids, long long id0, long long n_ids, bool *row_valid,
                                 long long *row_id) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h1 = T.dims[1];
  const bool last = (T.n_layers == 1);
  for (int r0 = warp * 2; r0 < APX_TILE; r0 += 2 * (APX_SIMT_THREADS / 32)) {
    long long rows[2][APEX_MAX_SLOTS];
    int nrows[2];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      bool valid;
      long long id;
      nrows[rr] = f32_row_sources(T, mode, rp, q0, o, ids, id0, n_ids, r0 + rr, rows[rr], valid, id);
      if (lane == 0) {
        row_valid[r0 + rr] = valid;
        row_id[r0 + rr] = id;
      }
    }
    float z[2][8];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int i = 0; i < 8; ++i) z[rr][i] = 0.f;
#pragma unroll
    for (int j = 0; j < APEX_MAX_SLOTS; ++j)
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
        if (j < nrows[rr]) {
          const float *src = T.P32 + rows[rr][j] * h1;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = lane + 32 * i;
            if (c < h1) z[rr][i] += __ldg(src + c);
          }
        }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        if (c < h1) S.AT[c][r0 + rr] = last ? z[rr][i] : f32_act(T.act, z[rr][i]);
      }
  }
}

// out = act(W^T-chunked GEMM of AT) for layer l (1-based index into dims: K = dims[l], N = dims[l+1]).
__device__ void f32_layer(F32Smem &S, const DevTables &T, int l) {
  const int K = T.dims[l], N = T.dims[l + 1];
  const float *WT = T.WT[l];
  const float *B = T.B[l];
  const bool last = (l == T.n_layers - 1);
  const int t = threadIdx.x;
  const int rg = t >> 4, cg = t & 15;
  float acc[8][16];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[i][j] = 0.f;
  const int nk = (K + F32_KC - 1) / F32_KC;
  auto load_chunk = [&](int kc, int buf) {
    for (int e = t; e < F32_KC * N; e += APX_SIMT_THREADS) {
      const int kk = e / N, n = e % N;
      const int k = kc * F32_KC + kk;
      S.Wc[buf][kk][n] = (k < K) ? __ldg(WT + (long long)k * N + n) : 0.f;
    }
  };
  load_chunk(0, 0);
  __syncthreads();
  for (int kc = 0; kc < nk; ++kc) {
    const int buf = kc & 1;
    if (kc + 1 < nk) load_chunk(kc + 1, buf ^ 1);
    const int kmax = min(F32_KC, K - kc * F32_KC);
    for (int kk = 0; kk < kmax; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&S.AT[kc * F32_KC + kk][rg * 8]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&S.AT[kc * F32_KC + kk][rg * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float w[16];
#pragma unroll
      for (int jq = 0; jq < 4; ++jq) {  // thread cg owns columns 64 jq + 4 cg + e (conflict-free 16-byte reads)
        const float4 w4 = *reinterpret_cast<const float4 *>(&S.Wc[buf][kk][64 * jq + 4 * cg]);
        w[4 * jq + 0] = w4.x;
        w[4 * jq + 1] = w4.y;
        w[4 * jq + 2] = w4.z;
        w[4 * jq + 3] = w4.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();
  }
  // every thread has finished reading AT: overwrite it with this layer's output
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int n = 64 * (j >> 2) + 4 * cg + (j & 3);
    if (n < N) {
      const float bn = __ldg(B + n);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float z = acc[i][j] + bn;
        S.AT[n][rg * 8 + i] = last ? z : f32_act(T.act, z);
      }
    }
  }
  __syncthreads();
}

// mode 0: enumeration (LaunchPlan); mode 1: ids[0, n_ids) -> out[n_ids x n_out] (FP32 outputs)
__global__ void __launch_bounds__(APX_SIMT_THREADS, 1)
    k_fp32_head(const __grid_constant__ LaunchPlan L, const __grid_constant__ DevTables T, QuerySlot *slots,
                const long long *ids, long long n_ids, float *out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F32Smem &S = *reinterpret_cast<F32Smem *>(smem_raw);
  __shared__ bool row_valid[APX_TILE];
  __shared__ long long row_id[APX_TILE];
  const int mode = (ids != nullptr) ? 1 : 0;
  const int n_out = T.n_out;
  long long n_work = mode == 0 ? L.total_items : (n_ids + APX_TILE - 1) / APX_TILE;
  for (long long it = blockIdx.x; it < n_work; it += gridDim.x) {
    const RxnPlan *rp = nullptr;
    long long q0 = 0, o_begin = 0, o_end = 1;
    unsigned long long qmask = 0;
    if (mode == 0) {
      const int sg = apx_find_seg(L, it);
      const Segment &seg = L.seg[sg];
      rp = T.rx + seg.rxn;
      const long long local = seg.item_begin + (it - L.seg_first[sg]);
      const long long b = local / rp->n_oc, oc = local % rp->n_oc;
      q0 = b * APX_TILE;
      o_begin = oc * rp->L_o;
      o_end = min(o_begin + rp->L_o, rp->n_outer);
      qmask = seg.qmask;
    }
    for (long long o = o_begin; o < o_end; ++o) {
      f32_build_layer1(S, T, mode, rp, q0, o, ids, it * APX_TILE, n_ids, row_valid, row_id);
      __syncthreads();
      for (int l = 1; l < T.n_layers; ++l) f32_layer(S, T, l);
      if (threadIdx.x < APX_TILE) {
        const int r = threadIdx.x;
        float ov[APEX_MAX_OUTPUTS];
#pragma unroll
        for (int n = 0; n < APEX_MAX_OUTPUTS; ++n) ov[n] = (n < n_out) ? S.AT[n][r] : 0.f;
        const bool valid = row_valid[r];
        const long long id = row_id[r];
        if (mode == 1) {
          if (valid) {
#pragma unroll
            for (int n = 0; n < APEX_MAX_OUTPUTS; ++n)
              if (n < n_out) out[(it * APX_TILE + r) * n_out + n] = ov[n];
          }
        } else if (L.mode == 1) {
          if (valid && id >= L.dump_base && id < L.dump_base + L.dump_n) {
#pragma unroll
            for (int n = 0; n < APEX_MAX_OUTPUTS; ++n)
              if (n < n_out) L.dump[(id - L.dump_base) * n_out + n] = ov[n];
          }
        } else if (L.mode == 2) {
          const long long slot = (it * (long long)L.dump_lo + (o - o_begin)) * APX_TILE + r;
          if (slot < L.dump_n) {
            L.dump_ids[slot] = valid ? id : -1;
#pragma unroll
            for (int n = 0; n < APEX_MAX_OUTPUTS; ++n)
              if (n < n_out) L.dump[slot * n_out + n] = ov[n];
          }
        } else {
          apx_apply_queries<APEX_MAX_OUTPUTS>(slots, qmask, valid, id, ov);
        }
      }
      __syncthreads();
    }
  }
}

size_t apx_fp32_smem_bytes() { return sizeof(F32Smem); }

cudaError_t apx_launch_fp32(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, const long long *ids,
                            long long n_ids, float *out, int grid, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_fp32_head, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(F32Smem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (grid <= 0) return cudaSuccess;
  apx_count_launch();
  k_fp32_head<<<grid, APX_SIMT_THREADS, sizeof(F32Smem), st>>>(L, T, slots, ids, n_ids, out);
  return cudaGetLastError();
}
