// k_prep.cu -- per-library precompute, run once at load (the "cache the synthon contributions"
// step of Sec. 3.3 and App. A.1, generalized from a row vector w_i to the matrix W_1):
//   P32[r] = W_1 u_r (+ b_1 when row r belongs to a reaction's first slot)   FP32
//   P16[r] = bf16(scale * P32[r])                                           tensor-core path
// so that the first layer of any compound is the plain sum of its slots' P rows.
#include <cuda_bf16.h>
#include <algorithm>
#include "common.cuh"

#define PREP_TM 64
#define PREP_TN 64
#define PREP_TK 16

// P[rows x N] = U[rows x K] * W^T (W: [N x K]) + bias[n] * bias_row[r]
__global__ void __launch_bounds__(256) k_p32(const float *__restrict__ U, const float *__restrict__ W,
                                             const float *__restrict__ bias, const unsigned char *__restrict__ bias_row,
                                             long long rows, int K, int N, float *__restrict__ P) {
  __shared__ float As[PREP_TK][PREP_TM + 4];
  __shared__ float Bs[PREP_TK][PREP_TN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int n0 = blockIdx.y * PREP_TN;
  for (long long r0 = (long long)blockIdx.x * PREP_TM; r0 < rows; r0 += (long long)gridDim.x * PREP_TM) {
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += PREP_TK) {
      for (int e = threadIdx.x; e < PREP_TK * PREP_TM; e += 256) {
        const int kk = e % PREP_TK, m = e / PREP_TK;
        const long long r = r0 + m;
        As[kk][m] = (r < rows && k0 + kk < K) ? U[r * K + k0 + kk] : 0.f;
      }
      for (int e = threadIdx.x; e < PREP_TK * PREP_TN; e += 256) {
        const int kk = e % PREP_TK, n = e / PREP_TK;
        Bs[kk][n] = (n0 + n < N && k0 + kk < K) ? W[(long long)(n0 + n) * K + k0 + kk] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < PREP_TK; ++kk) {
        float a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long r = r0 + ty * 4 + i;
      if (r >= rows) continue;
      const float br = bias_row[r] ? 1.f : 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx * 4 + j;
        if (n < N) P[r * N + n] = acc[i][j] + br * bias[n];
      }
    }
  }
}

__global__ void k_p16(const float *__restrict__ P32, long long n, float scale, __nv_bfloat16 *__restrict__ P16) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    P16[i] = __float2bfloat16_rn(scale * P32[i]);
}

cudaError_t apx_launch_prep(const float *U, const float *W1, const float *b1, const unsigned char *bias_row,
                            long long rows, int K, int N, float *P32, cudaStream_t st) {
  dim3 grid((unsigned)std::min<long long>((rows + PREP_TM - 1) / PREP_TM, 65535), (N + PREP_TN - 1) / PREP_TN);
  apx_count_launch();
  k_p32<<<grid, 256, 0, st>>>(U, W1, b1, bias_row, rows, K, N, P32);
  return cudaGetLastError();
}

cudaError_t apx_launch_p16(const float *P32, long long n, float scale, void *P16, cudaStream_t st) {
  apx_count_launch();
  k_p16<<<148 * 8, 256, 0, st>>>(P32, n, scale, reinterpret_cast<__nv_bfloat16 *>(P16));
  return cudaGetLastError();
}
