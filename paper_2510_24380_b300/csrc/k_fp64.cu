// k_fp64.cu -- FP64 rescoring in the plain (unfactorized) order: g = sum_j u_{t,j,s_j}
// (Eq. factorizer), then every layer of the head in double precision. Used only for the
// compounds of the top-k boundary band and ties (Sec. 3 problem, final ordering), and for
// calibration. One CTA per compound, threads over the output units of each layer.
#include "common.cuh"

#define F64_THREADS 256

__device__ __forceinline__ double f64_act(int act, double z) {
  if (act == APEX_ACT_RELU) return z > 0.0 ? z : 0.0;
  if (act == APEX_ACT_SILU) return z / (1.0 + exp(-z));
  return z;
}

// ids: [n] (bit 62 ignored); out: [n x n_out] doubles
__global__ void __launch_bounds__(F64_THREADS) k_fp64_score(const __grid_constant__ DevTables T, const long long *ids,
                                                            long long n, double *out) {
  __shared__ double x[1024];   // d <= 1024, hidden widths <= 256
  __shared__ double y[256];
  __shared__ long long rows[APEX_MAX_SLOTS];
  __shared__ int nrows;
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    if (threadIdx.x == 0) {
      const long long id = ids[i] & APX_ID_MASK;
      int lo = 0, hi = T.n_rx - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.id_first[mid] <= id) lo = mid; else hi = mid - 1;
      }
      const RxnPlan *p = T.rx + lo;
      long long rem = id - p->id_first;
      int c = 0;
      for (int j = p->n_slots - 1; j >= 0; --j) {
        rows[j] = p->slot_row[j] + rem % p->slot_size[j];
        rem /= p->slot_size[j];
        ++c;
      }
      nrows = c;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < T.d; c += F64_THREADS) {
      double g = 0.0;
      for (int j = 0; j < nrows; ++j) g += (double)__ldg(T.U + rows[j] * T.d + c);
      x[c] = g;
    }
    __syncthreads();
    for (int l = 0; l < T.n_layers; ++l) {
      const int K = T.dims[l], N = T.dims[l + 1];
      const double *WT = T.WT64[l];
      for (int nn = threadIdx.x; nn < N; nn += F64_THREADS) {
        double z = T.B64[l][nn];
        for (int k = 0; k < K; ++k) z = fma(WT[(long long)k * N + nn], x[k], z);
        y[nn] = (l == T.n_layers - 1) ? z : f64_act(T.act, z);
      }
      __syncthreads();
      for (int nn = threadIdx.x; nn < N; nn += F64_THREADS) x[nn] = y[nn];
      __syncthreads();
    }
    for (int nn = threadIdx.x; nn < T.n_out; nn += F64_THREADS) out[i * T.n_out + nn] = x[nn];
    __syncthreads();
  }
}

cudaError_t apx_launch_fp64(const DevTables &T, const long long *ids, long long n, double *out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)(n < 148 * 16 ? n : 148 * 16);
  apx_count_launch();
  k_fp64_score<<<grid, F64_THREADS, 0, st>>>(T, ids, n, out);
  return cudaGetLastError();
}
