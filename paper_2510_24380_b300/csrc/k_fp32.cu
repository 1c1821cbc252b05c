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

#define F32_KC 16           // K rows of W^T per stage

// TM tile rows: 128 for enumeration work items, 32 for id lists (small batches spread over SMs)
template <int TM>
struct F32Smem {
  float AT[256][TM + 4];             // AT[k][row], transposed activations of the tile
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
template <int TM>
__device__ void f32_build_layer1(F32Smem<TM> &S, const DevTables &T, int mode, const RxnPlan *rp, long long q0, long long o,
                                 const long long *ids, long long id0, long long n_ids, bool *row_valid,
                                 long long *row_id) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h1 = T.dims[1];
  const bool last = (T.n_layers == 1);
  for (int r0 = warp * 2; r0 < TM; r0 += 2 * (APX_SIMT_THREADS / 32)) {
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

// Two FP32 lanes in one 64-bit register (lane 0 in the low half). fma.rn.f32x2: each lane is an
// ordinary round-to-nearest fused multiply-add, so results equal two fmaf calls. Accumulators
// stay packed for the whole layer; operands that are adjacent in shared memory load as pairs.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2dup(float v) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ void f2unpack(f32x2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ void ffma2(f32x2 &c, f32x2 a, f32x2 b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(a), "l"(b));
}

// out = act(W^T-chunked GEMM of AT) for layer l (1-based index into dims: K = dims[l], N = dims[l+1]).
// Thread (rg, cg) owns 8 rows (rg) and CPT columns 4 CG jq + 4 cg + e (CG = 256 / CPT column
// groups; 16-byte conflict-free reads of W^T, broadcast reads of AT), two rows per packed FMA.
// CPT = 16 for 128-row tiles, 4 for 32-row tiles. Column groups past N are skipped. The next W^T
// chunk is fetched into registers before the current chunk is consumed and stored to shared
// memory after it, so its global-load latency overlaps the FMAs.
template <int TM>
__device__ void f32_layer(F32Smem<TM> &S, const DevTables &T, int l) {
  constexpr int RPT = 8;
  constexpr int RG = TM / RPT;                    // row groups: 16 (TM 128) or 4 (TM 32)
  constexpr int CG = APX_SIMT_THREADS / RG;       // column groups: 16 or 64
  constexpr int CPT = 256 / CG;                   // columns per thread: 16 or 4
  constexpr int JQ = CPT / 4;
  const int K = T.dims[l], N = T.dims[l + 1];
  const float *WT = T.WT[l];
  const float *B = T.B[l];
  const bool last = (l == T.n_layers - 1);
  const int t = threadIdx.x;
  const int rg = t / CG, cg = t % CG;
  const int jq_n = min(JQ, (N + 4 * CG - 1) / (4 * CG));  // column groups that hold outputs
  f32x2 acc[RPT / 2][CPT];  // rows (2i, 2i + 1) of column j
#pragma unroll
  for (int i = 0; i < RPT / 2; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = 0ull;
  const int nk = (K + F32_KC - 1) / F32_KC;
  float pre[F32_KC * 256 / APX_SIMT_THREADS];
  auto fetch = [&](int kc) {
#pragma unroll
    for (int q = 0; q < F32_KC * 256 / APX_SIMT_THREADS; ++q) {
      const int e = t + q * APX_SIMT_THREADS;
      const int kk = e >> 8, n = e & 255;
      const int k = kc * F32_KC + kk;
      pre[q] = (k < K && n < N) ? __ldg(WT + (long long)k * N + n) : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < F32_KC * 256 / APX_SIMT_THREADS; ++q) {
      const int e = t + q * APX_SIMT_THREADS;
      S.Wc[buf][e >> 8][e & 255] = pre[q];
    }
  };
  fetch(0);
  store(0);
  __syncthreads();
  for (int kc = 0; kc < nk; ++kc) {
    const int buf = kc & 1;
    if (kc + 1 < nk) fetch(kc + 1);
    const int kmax = min(F32_KC, K - kc * F32_KC);
    for (int kk = 0; kk < kmax; ++kk) {
      const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(&S.AT[kc * F32_KC + kk][rg * RPT]);
      const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(&S.AT[kc * F32_KC + kk][rg * RPT + 4]);
      const f32x2 a[RPT / 2] = {a0.x, a0.y, a1.x, a1.y};
#pragma unroll
      for (int jq = 0; jq < JQ; ++jq) {
        if (jq >= jq_n) break;  // uniform
        const float4 w4 = *reinterpret_cast<const float4 *>(&S.Wc[buf][kk][4 * CG * jq + 4 * cg]);
        const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const f32x2 wd = f2dup(w[e]);
#pragma unroll
          for (int i = 0; i < RPT / 2; ++i) ffma2(acc[i][4 * jq + e], a[i], wd);
        }
      }
    }
    if (kc + 1 < nk) store(buf ^ 1);  // the other buffer was last read before the previous barrier
    __syncthreads();
  }
  // every thread has finished reading AT: overwrite it with this layer's output
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int n = 4 * CG * (j >> 2) + 4 * cg + (j & 3);
    if (n < N) {
      const float bn = __ldg(B + n);
#pragma unroll
      for (int i = 0; i < RPT / 2; ++i) {
        float z0, z1;
        f2unpack(acc[i][j], z0, z1);
        z0 += bn;
        z1 += bn;
        S.AT[n][rg * RPT + 2 * i] = last ? z0 : f32_act(T.act, z0);
        S.AT[n][rg * RPT + 2 * i + 1] = last ? z1 : f32_act(T.act, z1);
      }
    }
  }
  __syncthreads();
}

// Last layer with at most 16 outputs (the usual head: a few objectives and properties): thread
// (row r, output group grp) accumulates OPG outputs over the whole K range in order, so every
// output is the same fmaf chain whatever the tile height (results do not depend on the id tile
// chosen by the autotuner); W^T of the layer is staged in shared memory (broadcast reads),
// reusing the W^T chunk buffers, instead of computing 256 padded columns.
template <int TM>
__device__ void f32_last_small(F32Smem<TM> &S, const DevTables &T, int l) {
  constexpr int NG = APX_SIMT_THREADS / TM;  // output groups: 2 (128-row tiles) or 8 (32-row tiles)
  constexpr int OPG = 16 / NG;               // outputs per group: 8 or 2
  const int K = T.dims[l], N = T.dims[l + 1];
  float *w = &S.Wc[0][0][0];  // [K][16]
  for (int e = threadIdx.x; e < K * 16; e += APX_SIMT_THREADS) {
    const int k = e >> 4, n = e & 15;
    w[e] = n < N ? __ldg(T.WT[l] + (long long)k * N + n) : 0.f;
  }
  __syncthreads();
  const int r = threadIdx.x % TM, grp = threadIdx.x / TM;
  f32x2 acc[OPG / 2];  // outputs (grp OPG + 2m, grp OPG + 2m + 1)
#pragma unroll
  for (int m = 0; m < OPG / 2; ++m) acc[m] = 0ull;
  for (int k = 0; k < K; ++k) {
    const f32x2 a = f2dup(S.AT[k][r]);
    const f32x2 *wk = reinterpret_cast<const f32x2 *>(w + k * 16 + grp * OPG);
#pragma unroll
    for (int m = 0; m < OPG / 2; ++m) ffma2(acc[m], a, wk[m]);
  }
  __syncthreads();  // every thread has read AT
#pragma unroll
  for (int m = 0; m < OPG / 2; ++m) {
    float z0, z1;
    f2unpack(acc[m], z0, z1);
    const int n = grp * OPG + 2 * m;
    if (n < N) S.AT[n][r] = z0 + __ldg(T.B[l] + n);
    if (n + 1 < N) S.AT[n + 1][r] = z1 + __ldg(T.B[l] + n + 1);
  }
  __syncthreads();
}

// mode 0: enumeration (LaunchPlan); mode 1: ids[0, n) -> out[n x n_out] (FP32 outputs), n = n_ids, or
// min(n_ids, *n_dev) when the list's length is a device count
template <int TM>
__global__ void __launch_bounds__(APX_SIMT_THREADS, 1)
    k_fp32_head(const __grid_constant__ LaunchPlan L, const __grid_constant__ DevTables T, QuerySlot *slots,
                const long long *ids, long long n_ids, float *out, const unsigned *n_dev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F32Smem<TM> &S = *reinterpret_cast<F32Smem<TM> *>(smem_raw);
  __shared__ bool row_valid[TM];
  __shared__ long long row_id[TM];
  const int mode = (ids != nullptr) ? 1 : 0;
  if (n_dev && (long long)*n_dev < n_ids) n_ids = *n_dev;  // id list sized on the device
  const int n_out = T.n_out;
  long long n_work = mode == 0 ? L.total_items : (n_ids + TM - 1) / TM;
  for (long long it = blockIdx.x; it < n_work; it += gridDim.x) {
    const RxnPlan *rp = nullptr;
    long long q0 = 0, o_begin = 0, o_end = 1, tile0 = 0;
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
      // launch tile of outer index o_begin (mode-2 dump layout shared with the tensor-core kernel)
      tile0 = L.seg_tile_first[sg] + apx_tiles_before(*rp, local) - apx_tiles_before(*rp, seg.item_begin);
    }
    for (long long o = o_begin; o < o_end; ++o) {
      f32_build_layer1<TM>(S, T, mode, rp, q0, o, ids, it * TM, n_ids, row_valid, row_id);
      __syncthreads();
      for (int l = 1; l < T.n_layers; ++l) {
        if (l == T.n_layers - 1 && T.dims[l + 1] <= 16)
          f32_last_small<TM>(S, T, l);
        else
          f32_layer<TM>(S, T, l);
      }
      if (threadIdx.x < TM) {
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
              if (n < n_out) out[(it * TM + r) * n_out + n] = ov[n];
          }
        } else if (L.mode == 1) {
          if (valid && id >= L.dump_base && id < L.dump_base + L.dump_n) {
#pragma unroll
            for (int n = 0; n < APEX_MAX_OUTPUTS; ++n)
              if (n < n_out) L.dump[(id - L.dump_base) * n_out + n] = ov[n];
          }
        } else if (L.mode == 2) {
          const long long slot = (tile0 + (o - o_begin)) * APX_TILE + r;
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

size_t apx_fp32_smem_bytes() { return sizeof(F32Smem<128>); }

// Enumeration (ids == nullptr) runs 128-row tiles; id lists run id_tile-row tiles (32 or 128,
// chosen by the autotuner), min(tiles, 148 * 2) CTAs.
cudaError_t apx_launch_fp32(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, const long long *ids,
                            long long n_ids, float *out, int grid, cudaStream_t st, int id_tile, const unsigned *n_dev) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_fp32_head<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(F32Smem<128>));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fp32_head<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(F32Smem<32>));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (ids == nullptr) {
    if (grid <= 0) return cudaSuccess;
    apx_count_launch();
    k_fp32_head<128><<<grid, APX_SIMT_THREADS, sizeof(F32Smem<128>), st>>>(L, T, slots, ids, n_ids, out, n_dev);
  } else if (id_tile == 128) {
    const long long tiles = (n_ids + 127) / 128;
    if (tiles <= 0) return cudaSuccess;
    const int g = (int)(tiles < 148 * 2 ? tiles : 148 * 2);
    apx_count_launch();
    k_fp32_head<128><<<g, APX_SIMT_THREADS, sizeof(F32Smem<128>), st>>>(L, T, slots, ids, n_ids, out, n_dev);
  } else {
    const long long tiles = (n_ids + 31) / 32;
    if (tiles <= 0) return cudaSuccess;
    const int g = (int)(tiles < 148 * 2 ? tiles : 148 * 2);
    apx_count_launch();
    k_fp32_head<32><<<g, APX_SIMT_THREADS, sizeof(F32Smem<32>), st>>>(L, T, slots, ids, n_ids, out, n_dev);
  }
  return cudaGetLastError();
}
