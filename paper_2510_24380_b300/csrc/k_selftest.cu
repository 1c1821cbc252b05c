// k_selftest.cu -- self-test of the bounded waits that every kernel of this library uses: one
// thread waits, with a caller-chosen limit, on an mbarrier phase that nothing completes. The wait
// must give up after the limit, record APX_ERR_TIMEOUT in the status word and return, leaving the
// CUDA context usable; nothing faults, traps or hangs.
#include "common.cuh"
#include "tc_sync.cuh"

__global__ void k_wait_selftest(int *err, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&bar), 1);  // phase 0 completes after one arrival, and none is made
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(smem_u32(&bar), 0, &abort_flag, err, limit_ns);
  __syncthreads();
}

cudaError_t apx_launch_wait_selftest(int *err, unsigned long long limit_ns, cudaStream_t st) {
  apx_count_launch();
  k_wait_selftest<<<1, 32, 0, st>>>(err, limit_ns);
  return cudaGetLastError();
}
