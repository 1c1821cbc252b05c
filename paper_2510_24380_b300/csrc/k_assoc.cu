// k_assoc.cu -- associative embeddings of Eq. assoc_embeds, u_{r,s} = K_r v_s: one key matrix
// K_r (d x d_u) per R-group slot, one value vector v_s (d_u) per synthon row, rows slot-major.
// A grouped FP32 GEMM run once per library (its cost is O(|S|), Sec. 3.3): CTA = 64 rows of one
// slot x 64 output columns; the slot's key tile and the value rows are staged through shared
// memory in 32-wide K chunks, each thread accumulates a 4 x 4 block in registers.
#include <algorithm>
#include "common.cuh"

#define AS_ROWS 64
#define AS_COLS 64
#define AS_KC 32

// blocks: every (slot, 64-row block) pair, listed by the host as (slot, first row, rows)
struct AssocBlock {
  int slot;
  int rows;
  long long row0;
};

__global__ void __launch_bounds__(256) k_assoc(const AssocBlock *blocks, int d, int d_u, const float *__restrict__ K,
                                               const float *__restrict__ V, float *__restrict__ U) {
  __shared__ float sv[AS_KC][AS_ROWS + 1];  // value rows, transposed: sv[k][row]
  __shared__ float sk[AS_KC][AS_COLS + 1];  // key tile, transposed: sk[k][col]
  const AssocBlock B = blocks[blockIdx.x];
  const int c0 = blockIdx.y * AS_COLS;
  const int t = threadIdx.x, tr = t >> 4, tc = t & 15;  // 16 x 16 threads, 4 x 4 outputs each
  const float *Kr = K + (size_t)B.slot * d * d_u;
  float acc[4][4] = {{0.f}};
  for (int k0 = 0; k0 < d_u; k0 += AS_KC) {
    for (int e = t; e < AS_KC * AS_ROWS; e += 256) {
      const int kk = e % AS_KC, rr = e / AS_KC;
      sv[kk][rr] = (rr < B.rows && k0 + kk < d_u) ? V[(size_t)(B.row0 + rr) * d_u + k0 + kk] : 0.f;
    }
    for (int e = t; e < AS_KC * AS_COLS; e += 256) {
      const int kk = e % AS_KC, cc = e / AS_KC;
      sk[kk][cc] = (c0 + cc < d && k0 + kk < d_u) ? Kr[(size_t)(c0 + cc) * d_u + k0 + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < AS_KC; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sv[kk][tr * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sk[kk][tc * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = tr * 4 + i;
    if (r >= B.rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tc * 4 + j;
      if (c < d) U[(size_t)(B.row0 + r) * d + c] = acc[i][j];
    }
  }
}

cudaError_t apx_launch_assoc(const void *blocks, int n_blocks, int d, int d_u, const float *K, const float *V, float *U,
                             cudaStream_t st) {
  if (n_blocks <= 0) return cudaSuccess;
  apx_count_launch();
  dim3 grid((unsigned)n_blocks, (unsigned)((d + AS_COLS - 1) / AS_COLS));
  k_assoc<<<grid, 256, 0, st>>>(reinterpret_cast<const AssocBlock *>(blocks), d, d_u, K, V, U);
  return cudaGetLastError();
}

// host helper: the (slot, 64-row block) list of a library's slots
int apx_assoc_blocks(long long n_slots_total, const int64_t *slot_sizes, void *out, int capacity) {
  AssocBlock *b = reinterpret_cast<AssocBlock *>(out);
  int n = 0;
  long long row = 0;
  for (long long s = 0; s < n_slots_total; ++s) {
    for (long long r = 0; r < slot_sizes[s]; r += AS_ROWS) {
      if (n < capacity) {
        b[n].slot = (int)s;
        b[n].rows = (int)std::min<long long>(AS_ROWS, slot_sizes[s] - r);
        b[n].row0 = row + r;
      }
      ++n;
    }
    row += slot_sizes[s];
  }
  return n;
}
size_t apx_assoc_block_bytes() { return sizeof(AssocBlock); }
