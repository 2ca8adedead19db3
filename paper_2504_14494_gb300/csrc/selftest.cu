// Failure-detection self-test of the bounded device waits.  Every wait of
// the tensor-core kernels on an mbarrier gives up after a cycle budget,
// raises the timeout bit of the status word and lets the kernel release its
// resources and return.  This kernel exercises exactly that path on a barrier
// that nothing ever arrives on, with a short budget; nothing traps or hangs.
#include "common.cuh"
#include "umma.cuh"

namespace lbmgnn {

__global__ void wait_timeout_kernel(long long max_cycles, unsigned* stw, int* gave_up) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, max_cycles);  // no arrival: must give up
  if (__syncthreads_or(!ok) && threadIdx.x == 0) {
    raise_status(stw, ST_TIMEOUT);
    if (gave_up) *gave_up = 1;
  }
}

}  // namespace lbmgnn

extern "C" int lbm_selftest_wait_timeout(long long max_cycles, void* stream) {
  using namespace lbmgnn;
  if (max_cycles < 1 || max_cycles > 2000000000LL) return LBM_ERR_ARG;
  unsigned* stw = status_word();
  if (!stw) return LBM_ERR_CUDA;
  wait_timeout_kernel<<<1, 64, 0, static_cast<cudaStream_t>(stream)>>>(max_cycles, stw, nullptr);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
