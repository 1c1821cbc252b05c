// k_linear.cu -- the paper's own fast path for a linear surrogate head (Eq. surrogate, Eq. apex):
// with o = W g + b and g = sum_j u_{t,j,s_j}, every output is a sum of per-synthon scalars,
// P[row] = W u_row (+ b on slot-1 rows), so a compound costs n_slots additions per output
// instead of a dense layer. The objective folds further: f = sum_i w_i o_i = f_inner + f_outer,
// with f_inner formed once per tile row (the row's inner-slot synthons) and f_outer once per
// outer synthon, so scoring a compound against a query's admission threshold is one addition
// and one comparison; the constraint outputs are summed only for the compounds that pass.
//
// Work: the tiles of the launch (128 inner rows x one outer synthon), an equal contiguous share
// per CTA, walked in runs that share their inner block. Thread r owns inner row q0 + r; the
// outer synthons of a run are staged through shared memory 128 at a time, with the query's
// objective and constrained outputs already folded per synthon.
#include "common.cuh"

#define LIN_THREADS 128

__global__ void __launch_bounds__(LIN_THREADS) k_linear(const __grid_constant__ LaunchPlan L,
                                                        const __grid_constant__ DevTables T, QuerySlot *slots) {
  __shared__ float s_f[LIN_THREADS];                          // f_outer of the chunk's outer synthons
  __shared__ float s_c[APEX_MAX_CONSTRAINTS][LIN_THREADS];    // their constrained outputs
  const int r = threadIdx.x, lane = r & 31;
  const int n_out = T.n_out;
  const long long t_begin = (long long)blockIdx.x * L.total_tiles / gridDim.x;
  const long long t_end = (long long)(blockIdx.x + 1) * L.total_tiles / gridDim.x;
  for (long long tile = t_begin; tile < t_end;) {
    const TileRun I = apx_tile_run(L, T.rx, tile, t_end);
    tile += I.o_end - I.o_begin;
    const RxnPlan *rp = I.rp;
    const long long q = I.q0 + r;
    const bool valid = q < rp->n_inner;
    // this row's inner-slot sums of every output
    float vi[APEX_MAX_OUTPUTS];
#pragma unroll
    for (int i = 0; i < APEX_MAX_OUTPUTS; ++i) vi[i] = 0.f;
    if (valid) {
      long long rem = q;
      for (int sl = rp->n_inner_slots - 1; sl >= 0; --sl) {
        const long long sz = rp->inner_size[sl];
        const float *src = T.P32 + (rp->inner_row[sl] + rem % sz) * n_out;
        rem /= sz;
#pragma unroll
        for (int i = 0; i < APEX_MAX_OUTPUTS; ++i)
          if (i < n_out) vi[i] += __ldg(src + i);
      }
    }
    const long long id_row = rp->id_first + q * rp->inner_stride;
    for (unsigned long long qm = I.qmask; qm; qm &= qm - 1) {
      QuerySlot *Q = slots + (__ffsll((long long)qm) - 1);
      const int n_obj = Q->n_obj, m = Q->n_cons;
      const float admit = *((volatile float *)&Q->admit);
      float fi = 0.f;
#pragma unroll
      for (int i = 0; i < APEX_MAX_OBJECTIVES && i < APEX_MAX_OUTPUTS; ++i)
        if (i < n_obj) fi = fmaf(__ldg(&Q->w[i]), vi[i], fi);
      for (long long o0 = I.o_begin; o0 < I.o_end; o0 += LIN_THREADS) {
        const int n_chunk = (int)min((long long)LIN_THREADS, I.o_end - o0);
        __syncthreads();  // the previous chunk's values are no longer read
        if (r < n_chunk) {
          float fo = 0.f;
          if (rp->outer_row >= 0) {
            const float *src = T.P32 + (rp->outer_row + o0 + r) * n_out;
            for (int i = 0; i < n_obj; ++i) fo = fmaf(__ldg(&Q->w[i]), __ldg(src + i), fo);
            for (int c = 0; c < m; ++c) s_c[c][r] = __ldg(src + Q->cons_idx[c]);
          } else {
            for (int c = 0; c < m; ++c) s_c[c][r] = 0.f;
          }
          s_f[r] = fo;
        }
        __syncthreads();
        for (int j = 0; j < n_chunk; ++j) {
          const float f = fi + s_f[j];
          bool pass = valid && f >= admit;
          if (__ballot_sync(0xffffffffu, pass) == 0u) continue;
          bool sure = true;
          for (int c = 0; c < m; ++c) {
            const int p = Q->cons_idx[c];
            float v = s_c[c][j];
#pragma unroll
            for (int i = 0; i < APEX_MAX_OUTPUTS; ++i)
              if (i == p) v += vi[i];
            pass = pass && v >= Q->lo_w[c] && v <= Q->hi_w[c];
            sure = sure && v >= Q->lo_s[c] && v <= Q->hi_s[c];
          }
          const unsigned pos = apx_warp_reserve(&Q->count, pass);
          if (pass) {
            if (pos < Q->cap) {
              Q->keys[pos] = f;
              Q->ids[pos] = (id_row + (o0 + j) * rp->outer_stride) | (sure ? 0LL : APX_UNSURE_BIT);
            } else {
              apx_note_dropped(Q, f);
            }
          }
        }
      }
    }
    (void)lane;
  }
}

cudaError_t apx_launch_linear(const LaunchPlan &L, const DevTables &T, QuerySlot *slots, int n_sm, cudaStream_t st) {
  if (L.total_tiles <= 0) return cudaSuccess;
  const long long g = L.total_tiles < (long long)n_sm * 8 ? L.total_tiles : (long long)n_sm * 8;
  apx_count_launch();
  k_linear<<<(unsigned)g, LIN_THREADS, 0, st>>>(L, T, slots);
  return cudaGetLastError();
}
