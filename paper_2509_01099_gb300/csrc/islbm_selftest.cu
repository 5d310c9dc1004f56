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
