// k_fp64.cu -- FP64 rescoring in the plain (unfactorized) order: g = sum_j u_{t,j,s_j}
// (Eq. factorizer), then every layer of the head in double precision. Used only for the
// compounds of the top-k boundary band and near bounds (the exact ordering of Sec. 3's
// problem), for calibration and for apex_score_ids.
//
// FP64 runs at a small fraction of the FP32 rate on this part, and the rescored sets are small
// (usually a few to a few hundred compounds), so latency matters more than reuse: one compound
// is spread over a cluster of 8 CTAs (8 SMs). In every layer CTA r computes its eighth of the
// output units (8 warps split K, lanes own consecutive units, so weight reads are coalesced)
// and writes them into the input buffer of all 8 CTAs through distributed shared memory; a
// cluster barrier separates the layers. The cluster barrier is a hardware barrier over CTAs
// that are co-scheduled by construction, so it needs no timeout.
#include <algorithm>
#include <cooperative_groups.h>
#include "common.cuh"

namespace cg = cooperative_groups;

#define F64_CLUSTER 8
#define F64_THREADS 256
#define F64_WARPS (F64_THREADS / 32)

__device__ __forceinline__ double f64_act(int act, double z) {
  if (act == APEX_ACT_RELU) return z > 0.0 ? z : 0.0;
  if (act == APEX_ACT_SILU) return z / (1.0 + exp(-z));
  return z;
}

// ids: [n] (bit 62 ignored); out: [n x n_out] doubles; n = min(n_max, *n_dev) when n_dev is set
__global__ void __cluster_dims__(F64_CLUSTER, 1, 1) __launch_bounds__(F64_THREADS)
    k_fp64_score(const __grid_constant__ DevTables T, const long long *ids, long long n_max, const unsigned *n_dev,
                 double *out) {
  cg::cluster_group cluster = cg::this_cluster();
  const long long n = n_dev ? (long long)min((unsigned long long)n_max, (unsigned long long)*n_dev) : n_max;
  extern __shared__ double sh[];  // x[2][dmax] (layer inputs, double buffered), part[F64_WARPS][32]
  __shared__ long long rows[APEX_MAX_SLOTS];
  __shared__ int nrows;
  const int dmax = max(T.d, 256);
  double *xb[2] = {sh, sh + dmax};
  double *part = sh + 2 * dmax;
  const unsigned rank = cluster.block_rank();
  const long long cid = blockIdx.x / F64_CLUSTER, n_cl = gridDim.x / F64_CLUSTER;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long i = cid; i < n; i += n_cl) {  // uniform within a cluster
    if (threadIdx.x == 0) {
      const long long id = ids[i] & APX_ID_MASK;
      int lo = 0, hi = T.n_rx - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.id_first[mid] <= id) lo = mid; else hi = mid - 1;
      }
      const RxnPlan *p = T.rx + lo;
      long long rem = id - p->id_first;
      for (int j = p->n_slots - 1; j >= 0; --j) {
        rows[j] = p->slot_row[j] + rem % p->slot_size[j];
        rem /= p->slot_size[j];
      }
      nrows = p->n_slots;
    }
    __syncthreads();
    // g = sum of the compound's synthon embeddings (every CTA keeps its own copy)
    for (int col = threadIdx.x; col < T.d; col += F64_THREADS) {
      double g = 0.0;
      for (int j = 0; j < nrows; ++j) g += (double)__ldg(T.U + rows[j] * T.d + col);
      xb[0][col] = g;
    }
    __syncthreads();
    for (int l = 0; l < T.n_layers; ++l) {
      const int K = T.dims[l], N = T.dims[l + 1];
      const int per = (N + F64_CLUSTER - 1) / F64_CLUSTER;  // <= 32 output units per CTA
      const int nn = (int)rank * per + lane;
      const bool mine = lane < per && nn < N;
      const double *x = xb[l & 1];
      const double *WT = T.WT64[l];
      double z = 0.0;
      if (mine)
        for (int k = warp; k < K; k += F64_WARPS) z = fma(WT[(long long)k * N + nn], x[k], z);
      part[warp * 32 + lane] = z;
      __syncthreads();
      if (warp == 0 && mine) {
        double s = T.B64[l][nn];
#pragma unroll
        for (int w = 0; w < F64_WARPS; ++w) s += part[w * 32 + lane];
        if (l == T.n_layers - 1) {
          out[i * T.n_out + nn] = s;
        } else {
          const double y = f64_act(T.act, s);
          for (unsigned r = 0; r < F64_CLUSTER; ++r) cluster.map_shared_rank(xb[(l + 1) & 1], r)[nn] = y;
        }
      }
      cluster.sync();  // this layer's outputs are in every CTA; its inputs are no longer read
    }
  }
}

// n_dev (optional): device count, at most n
cudaError_t apx_launch_fp64(const DevTables &T, const long long *ids, long long n, double *out, cudaStream_t st,
                            const unsigned *n_dev) {
  if (n <= 0) return cudaSuccess;
  const int dmax = std::max(T.d, 256);
  const size_t smem = sizeof(double) * (2 * dmax + F64_WARPS * 32);
  const long long clusters = std::min<long long>(n, 148);
  apx_count_launch();
  k_fp64_score<<<(unsigned)(clusters * F64_CLUSTER), F64_THREADS, smem, st>>>(T, ids, n, n_dev, out);
  return cudaGetLastError();
}
