// k_fp64.cu -- FP64 rescoring in the plain (unfactorized) order: g = sum_j u_{t,j,s_j}
// (Eq. factorizer), then every layer of the head in double precision. Used only for the
// compounds of the top-k boundary band and near-ties (the exact ordering of Sec. 3's problem),
// and for calibration. A CTA scores F64_CPB compounds at once: threads own output units, and
// every weight element loaded from memory feeds F64_CPB fused multiply-adds.
#include <algorithm>
#include "common.cuh"

#define F64_THREADS 256
#define F64_CPB 4

__device__ __forceinline__ double f64_act(int act, double z) {
  if (act == APEX_ACT_RELU) return z > 0.0 ? z : 0.0;
  if (act == APEX_ACT_SILU) return z / (1.0 + exp(-z));
  return z;
}

// ids: [n] (bit 62 ignored); out: [n x n_out] doubles
__global__ void __launch_bounds__(F64_THREADS) k_fp64_score(const __grid_constant__ DevTables T, const long long *ids,
                                                            long long n, double *out) {
  extern __shared__ double sh[];          // x: [F64_CPB][d_max], y: [F64_CPB][256]
  __shared__ long long rows[F64_CPB][APEX_MAX_SLOTS];
  __shared__ int nrows[F64_CPB];
  const int dmax = max(T.d, 256);
  double *x = sh;
  double *y = sh + F64_CPB * dmax;
  for (long long g0 = (long long)blockIdx.x * F64_CPB; g0 < n; g0 += (long long)gridDim.x * F64_CPB) {
    if (threadIdx.x < F64_CPB) {
      const int c = threadIdx.x;
      const long long i = g0 + c;
      int cnt = 0;
      if (i < n) {
        const long long id = ids[i] & APX_ID_MASK;
        int lo = 0, hi = T.n_rx - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (T.id_first[mid] <= id) lo = mid; else hi = mid - 1;
        }
        const RxnPlan *p = T.rx + lo;
        long long rem = id - p->id_first;
        for (int j = p->n_slots - 1; j >= 0; --j) {
          rows[c][j] = p->slot_row[j] + rem % p->slot_size[j];
          rem /= p->slot_size[j];
        }
        cnt = p->n_slots;
      }
      nrows[c] = cnt;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < F64_CPB * T.d; e += F64_THREADS) {
      const int c = e / T.d, col = e % T.d;
      double g = 0.0;
      for (int j = 0; j < nrows[c]; ++j) g += (double)__ldg(T.U + rows[c][j] * T.d + col);
      x[c * dmax + col] = g;
    }
    __syncthreads();
    for (int l = 0; l < T.n_layers; ++l) {
      const int K = T.dims[l], N = T.dims[l + 1];
      const double *WT = T.WT64[l];
      const bool last = (l == T.n_layers - 1);
      for (int nn = threadIdx.x; nn < N; nn += F64_THREADS) {
        double z[F64_CPB];
#pragma unroll
        for (int c = 0; c < F64_CPB; ++c) z[c] = T.B64[l][nn];
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
          const double w = WT[(long long)k * N + nn];
#pragma unroll
          for (int c = 0; c < F64_CPB; ++c) z[c] = fma(w, x[c * dmax + k], z[c]);
        }
#pragma unroll
        for (int c = 0; c < F64_CPB; ++c) y[c * 256 + nn] = last ? z[c] : f64_act(T.act, z[c]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < F64_CPB * N; e += F64_THREADS) {
        const int c = e / N, nn = e % N;
        x[c * dmax + nn] = y[c * 256 + nn];
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < F64_CPB * T.n_out; e += F64_THREADS) {
      const int c = e / T.n_out, nn = e % T.n_out;
      if (g0 + c < n) out[(g0 + c) * T.n_out + nn] = x[c * dmax + nn];
    }
    __syncthreads();
  }
}

cudaError_t apx_launch_fp64(const DevTables &T, const long long *ids, long long n, double *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int dmax = std::max(T.d, 256);
  const size_t smem = sizeof(double) * F64_CPB * (dmax + 256);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_fp64_score, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * F64_CPB * (1024 + 256)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long blocks = (n + F64_CPB - 1) / F64_CPB;
  const int grid = (int)std::min<long long>(blocks, 148 * 8);
  apx_count_launch();
  k_fp64_score<<<grid, F64_THREADS, smem, st>>>(T, ids, n, out);
  return cudaGetLastError();
}
