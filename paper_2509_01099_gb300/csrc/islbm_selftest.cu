// Self-test of the bounded waits used by the pipelined step kernels: a CTA
// waits on an mbarrier that nothing arrives at, gives up after the wait
// limit (one second of the global timer), raises the device error flag and
// returns.  The host sees
// ISLBM_ERR_TIMEOUT and the context stays usable.  The paper has no
// counterpart.
#include "islbm_internal.h"
#include "islbm_tma.cuh"

namespace islbm {
namespace {

__global__ void k_wait_never(int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // nothing arrives: phase 0 never completes
  const bool ok = mbar_wait(&bar, 0);
  if (!__syncthreads_or(!ok)) return;
  if (threadIdx.x == 0) atomicExch(err, 1);
}

// The abort flag of the barrier-free pipelined loops: warp 0 waits on an
// mbarrier that nothing arrives at until its limit and then raises the CTA's
// abort flag; the other warps make three waits on another such mbarrier with
// mbar_wait_or_abort.  Without the flag they would take three limits; with it
// the first ends at about one limit and the other two at once.  out[0]: the
// failed waits of warp 1 (3 expected), out[1]: their total time in ms.
__global__ void k_wait_abort(int* err, int* out) {
  __shared__ uint64_t bar[2];
  __shared__ int abort_flag;
  volatile int* abort = &abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = mbar_wait(&bar[0], 0);   // nothing arrives: gives up at the limit
    if (!ok && threadIdx.x == 0) {
      atomicExch(err, 1);
      *abort = 1;
    }
  } else {
    const unsigned long long t0 = global_ns();
    int failed = 0;
    for (int i = 0; i < 3; ++i) failed += mbar_wait_or_abort(&bar[1], 0, abort) ? 0 : 1;
    const unsigned long long dt = global_ns() - t0;
    if (threadIdx.x == 32) {
      out[0] = failed;
      out[1] = (int)(dt / 1000000ull);
    }
  }
}

}  // namespace
}  // namespace islbm

extern "C" islbm_status islbm_selftest_wait_timeout(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* d = nullptr;
  const islbm::DevAllocator mem = islbm::current_allocator();
  if (islbm::dev_alloc(mem, reinterpret_cast<void**>(&d), sizeof(int), st) != cudaSuccess)
    return ISLBM_ERR_OOM;
  int flag = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    islbm::k_wait_never<<<1, 64, 0, st>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  islbm::dev_free(mem, d, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ISLBM_ERR_CUDA;
  return flag ? ISLBM_ERR_TIMEOUT : ISLBM_OK;
}

extern "C" islbm_status islbm_selftest_wait_abort(void* stream, int* failed_waits, int* ms) {
  if (!failed_waits || !ms) return ISLBM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* d = nullptr;
  const islbm::DevAllocator mem = islbm::current_allocator();
  if (islbm::dev_alloc(mem, reinterpret_cast<void**>(&d), 3 * sizeof(int), st) != cudaSuccess)
    return ISLBM_ERR_OOM;
  int h[3] = {0, 0, 0};
  cudaError_t e = cudaMemsetAsync(d, 0, 3 * sizeof(int), st);
  if (e == cudaSuccess) {
    islbm::k_wait_abort<<<1, 256, 0, st>>>(d, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 3 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  islbm::dev_free(mem, d, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ISLBM_ERR_CUDA;
  *failed_waits = h[1];
  *ms = h[2];
  return h[0] ? ISLBM_ERR_TIMEOUT : ISLBM_OK;
}
