// Issue-rate microbenchmark of the tensor cores: cycles per tcgen05.mma
// (M = 128, K = 16, BF16 operands from shared memory, FP32 accumulator) for
// several N, one or two CTAs per SM, one issuing thread per CTA (512 MMAs
// into one accumulator, one commit, a bounded mbarrier wait).
#include <cstdio>
#include <cstdint>
#include "umma.cuh"
using namespace lbmgnn;

__global__ void probe(int N, int reps, long long* out, int ctas_per_sm_unused) {
  extern __shared__ uint8_t raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t bar;
  __shared__ uint32_t tm;
  // A: 128 rows x 128 B (16 KB), B: 256 rows x 128 B (32 KB), zero-filled
  for (int i = threadIdx.x; i < (16384 + 32768) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  if (threadIdx.x < 32) tmem_alloc(&tm, 256);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  long long t0 = 0, t1 = 0;
  bool ok = true;
  if (threadIdx.x == 0) {
    const uint32_t id = idesc_bf16(128, N);
    const uint64_t ad = sw128_desc(smem_u32(sm));
    const uint64_t bd = sw128_desc(smem_u32(sm + 16384));
    // warm-up
    umma_bf16(tm, ad, bd, id, 0u);
    umma_commit(&bar);
    ok = mbar_wait(&bar, 0, 200000000LL);
    tc_fence_after();
    t0 = clock64();
    for (int r = 0; r < reps; ++r) umma_bf16(tm, ad, bd, id, r > 0 ? 1u : 0u);
    umma_commit(&bar);
    ok = ok && mbar_wait(&bar, 1, 200000000LL);
    t1 = clock64();
    out[blockIdx.x * 2] = ok ? (t1 - t0) : -1;
    out[blockIdx.x * 2 + 1] = reps;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tmem_dealloc(tm, 256);
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, 50176);
  long long* d;
  cudaMalloc(&d, sizeof(long long) * 2 * 4 * 200);
  long long h[2 * 4 * 200];
  const int Ns[] = {16, 32, 64, 128, 256};
  for (int per = 1; per <= 2; ++per) {
    for (int N : Ns) {
      const int grid = sms * per;
      probe<<<grid, 128, 50176>>>(N, 512, d, per);
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
      cudaMemcpy(h, d, sizeof(long long) * 2 * grid, cudaMemcpyDeviceToHost);
      double s = 0; int n = 0;
      for (int i = 0; i < grid; ++i) if (h[2 * i] > 0) { s += (double)h[2 * i] / h[2 * i + 1]; ++n; }
      printf("ctas/SM %d  N %3d  cycles per MMA (M=128,K=16) %.1f  (flop/clk/SM %.0f)\n", per, N,
             s / n, per * 2.0 * 128 * N * 16 / (s / n));
    }
  }
  cudaFree(d);
  return 0;
}
