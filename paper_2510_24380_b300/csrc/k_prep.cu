// k_prep.cu -- per-library precompute, run once at load (the "cache the synthon contributions"
// step of Sec. 3.3 and App. A.1, generalized from a row vector w_i to the matrix W_1):
//   P32[r] = W_1 u_r (+ b_1 when row r belongs to a reaction's first slot)   FP32
//   P16[r] = bf16(scale * P32[r])                                           tensor-core path
// so that the first layer of any compound is the plain sum of its slots' P rows.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
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

__global__ void k_p16(const float *__restrict__ P32, long long n, float scale, int fmt, unsigned short *__restrict__ P16) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = scale * P32[i];
    P16[i] = fmt == 0 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
  }
}

// SW128 K-major shared-memory image of W [rows_used x 256] (float, already scaled), padded to
// rows rows: four 64-column chunks of rows x 128 B, 8-row atoms of 1024 B, 16-byte pieces
// XOR-swizzled by (row mod 8); 16-bit elements in the given format.
__global__ void k_sw128_image(const float *__restrict__ W, int rows_used, int rows, int fmt, unsigned char *img) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * 256; e += gridDim.x * blockDim.x) {
    const int n = e >> 8, k = e & 255;
    const float v = n < rows_used ? W[(size_t)n * 256 + k] : 0.f;
    const unsigned short b = fmt == 0 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
    const int kc = k >> 6, kin = k & 63, piece = kin >> 3, el = kin & 7;
    const size_t off = (size_t)kc * rows * 128 + (size_t)(n >> 3) * 1024 + (size_t)(n & 7) * 128 +
                       (size_t)((piece ^ (n & 7)) * 16) + (size_t)el * 2;
    *reinterpret_cast<unsigned short *>(img + off) = b;
  }
}

// FP8 (e4m3) SW128 K-major image of W [rows_used x 256] with one scale per row: element
// e4m3(W[n][k] / scale[n]) (round to nearest even, saturating); 128 K elements per 128-byte row,
// two K chunks of rows x 128 B, 8-row atoms of 1024 B, 16-byte pieces XOR-swizzled by (row mod 8).
__global__ void k_sw128_image_e4m3(const float *__restrict__ W, const float *__restrict__ scale, int rows_used, int rows,
                                   unsigned char *img) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * 256; e += gridDim.x * blockDim.x) {
    const int n = e >> 8, k = e & 255;
    const float v = n < rows_used ? W[(size_t)n * 256 + k] / scale[n] : 0.f;
    const __nv_fp8_storage_t b = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    const int kc = k >> 7, kin = k & 127, piece = kin >> 4, el = kin & 15;
    const size_t off = (size_t)kc * rows * 128 + (size_t)(n >> 3) * 1024 + (size_t)(n & 7) * 128 +
                       (size_t)((piece ^ (n & 7)) * 16) + (size_t)el;
    img[off] = (unsigned char)b;
  }
}

// Per-slot column extremes of P (FP32): mx[j][n] = max over the slot's rows r of P[r][n], mn likewise.
// One block per slot, one thread per column (rows read in order, coalesced).
__global__ void k_slot_extremes(const float *__restrict__ P, const long long *__restrict__ row_first, int N,
                                float *__restrict__ mx, float *__restrict__ mn) {
  const int j = blockIdx.x;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    float a = -INFINITY, b = INFINITY;
    for (long long r = row_first[j]; r < row_first[j + 1]; ++r) {
      const float v = P[r * N + n];
      a = fmaxf(a, v);
      b = fminf(b, v);
    }
    mx[(size_t)j * N + n] = a;
    mn[(size_t)j * N + n] = b;
  }
}

cudaError_t apx_launch_slot_extremes(const float *P, const long long *row_first, int n_slots, int N, float *mx,
                                     float *mn, cudaStream_t st) {
  if (n_slots <= 0) return cudaSuccess;
  apx_count_launch();
  k_slot_extremes<<<n_slots, 256, 0, st>>>(P, row_first, N, mx, mn);
  return cudaGetLastError();
}

cudaError_t apx_launch_image_e4m3(const float *W, const float *scale, int rows_used, int rows, void *img,
                                  cudaStream_t st) {
  apx_count_launch();
  k_sw128_image_e4m3<<<(rows * 256 + 255) / 256, 256, 0, st>>>(W, scale, rows_used, rows, (unsigned char *)img);
  return cudaGetLastError();
}

cudaError_t apx_launch_image(const float *W, int rows_used, int rows, int fmt, void *img, cudaStream_t st) {
  apx_count_launch();
  k_sw128_image<<<(rows * 256 + 255) / 256, 256, 0, st>>>(W, rows_used, rows, fmt, (unsigned char *)img);
  return cudaGetLastError();
}

cudaError_t apx_launch_prep(const float *U, const float *W1, const float *b1, const unsigned char *bias_row,
                            long long rows, int K, int N, float *P32, cudaStream_t st) {
  dim3 grid((unsigned)std::min<long long>((rows + PREP_TM - 1) / PREP_TM, 65535), (N + PREP_TN - 1) / PREP_TN);
  apx_count_launch();
  k_p32<<<grid, 256, 0, st>>>(U, W1, b1, bias_row, rows, K, N, P32);
  return cudaGetLastError();
}

cudaError_t apx_launch_p16(const float *P32, long long n, float scale, int fmt, void *P16, cudaStream_t st) {
  apx_count_launch();
  k_p16<<<148 * 8, 256, 0, st>>>(P32, n, scale, fmt, reinterpret_cast<unsigned short *>(P16));
  return cudaGetLastError();
}
