// Check of the bounded mbarrier wait of mbarrier.cuh: a single CTA waits on
// a barrier that nothing arrives at, with the library's wait function and a
// caller-chosen limit; the wait must give up and report it.  This exercises
// failure detection without any GPU fault or hang.
#include "../../include/amr.h"
#include "amr_internal.h"
#include "mbarrier.cuh"

namespace amr {

static __device__ int32_t g_probe_flag;

__global__ void k_wait_probe(long long limit_cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_addr(&bar), 0u, limit_cycles);
  __syncthreads();
  if (threadIdx.x == 0) {
    g_probe_flag = ok ? 0 : 1;
    mbar_inval(smem_addr(&bar));
  }
}

}  // namespace amr

extern "C" int amr_check_bounded_wait(long long limit_cycles, void* stream) {
  using namespace amr;
  if (limit_cycles <= 0 || limit_cycles > (1ll << 32)) {
    set_error("limit_cycles must be in (0, 2^32]");
    return AMR_E_INVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t zero = -1;
  AMR_CUDA(cudaMemcpyToSymbolAsync(g_probe_flag, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s));
  k_wait_probe<<<1, 32, 0, s>>>(limit_cycles);
  AMR_CUDA(cudaGetLastError());
  int32_t flag = -1;
  AMR_CUDA(cudaMemcpyFromSymbolAsync(&flag, g_probe_flag, sizeof(flag), 0, cudaMemcpyDeviceToHost, s));
  AMR_CUDA(cudaStreamSynchronize(s));
  if (flag == 1) {
    set_error("bounded wait gave up as expected");
    return AMR_E_TIMEOUT;
  }
  return flag == 0 ? AMR_OK : AMR_E_CUDA;
}
