// Issue-rate microbenchmark of the packed-FP16 arithmetic the message
// passing of the GNN-enhanced collision runs on (the elementwise bound of the
// message-passing round kernel): warp instructions per SM clock of
//   HFMA2               (fma.rn.f16x2)
//   tanh.approx.f16x2   (the MUFU unit)
//   one edge message on a pair of features: z = (A + c) + B, u = z (c0 + c1
//   z^2), acc += z + z tanh(u) -- 7 packed-FP16 operations and one tanh,
//   i.e. two edge-feature GELUs -- timed as a whole.
// Each thread runs 8 independent chains; 8 CTAs of 256 threads per SM; the
// cycles of each CTA come from clock64(); results are written out so that
// nothing is optimised away.  Prints one JSON line.
#include <cuda_fp16.h>
#include <cstdint>
#include <cstdio>

constexpr int CH = 8;

__device__ __forceinline__ __half2 tanh_h2(__half2 x) {
  uint32_t y;
  asm volatile("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<uint32_t*>(&x)));
  return *reinterpret_cast<__half2*>(&y);
}

template <int KIND>
__global__ void __launch_bounds__(256) rate(int iters, float seed, long long* cycles, float* sink) {
  __half2 acc[CH], z[CH];
  for (int c = 0; c < CH; ++c) {
    acc[c] = __float2half2_rn(seed * (c + 1) + threadIdx.x * 1e-3f);
    z[c] = __float2half2_rn(0.25f + 0.01f * c);
  }
  const __half2 a = __float2half2_rn(0.999f), b = __float2half2_rn(1e-3f);
  const __half2 c0 = __float2half2_rn(0.7978845608028654f);
  const __half2 c1 = __float2half2_rn(0.0356774081363001f);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (KIND == 0) {
        acc[c] = __hfma2(acc[c], a, b);
      } else if (KIND == 1) {
        acc[c] = tanh_h2(acc[c]);
      } else {
        const __half2 zz = __hadd2(__hadd2(z[c], b), acc[c]);
        const __half2 u = __hmul2(zz, __hfma2(c1, __hmul2(zz, zz), c0));
        acc[c] = __hadd2(acc[c], __hfma2(zz, tanh_h2(u), zz));
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
  for (int c = 0; c < CH; ++c) s += __low2float(acc[c]) + __high2float(acc[c]);
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

int main() {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = 8, grid = sms * per_sm, iters = 4096;
  long long* dc;
  float* ds;
  cudaMalloc(&dc, sizeof(long long) * grid);
  cudaMalloc(&ds, sizeof(float) * grid * 256);
  long long* hc = new long long[grid];
  const char* names[3] = {"hfma2", "tanh_f16x2", "edge_message_pair"};
  // instructions per chain iteration (warp instructions per warp)
  const double per_iter[3] = {1.0, 1.0, 8.0};
  printf("{\"sms\": %d", sms);
  for (int kind = 0; kind < 3; ++kind) {
    for (int rep = 0; rep < 2; ++rep) {  // first run warms up
      if (kind == 0) rate<0><<<grid, 256>>>(iters, 0.5f, dc, ds);
      if (kind == 1) rate<1><<<grid, 256>>>(iters, 0.5f, dc, ds);
      if (kind == 2) rate<2><<<grid, 256>>>(iters, 0.5f, dc, ds);
      if (cudaDeviceSynchronize() != cudaSuccess) {
        printf(", \"error\": \"%s\"}\n", cudaGetErrorString(cudaGetLastError()));
        return 1;
      }
    }
    cudaMemcpy(hc, dc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    double mx = 0;
    for (int i = 0; i < grid; ++i) mx = hc[i] > mx ? hc[i] : mx;
    // all CTAs of an SM run concurrently: warp instructions of one SM / the
    // longest CTA's cycles
    const double winstr = (double)per_sm * 8 * iters * CH * per_iter[kind];
    printf(", \"%s_warp_instr_per_clk_per_sm\": %.3f", names[kind], winstr / mx);
    if (kind == 2)
      printf(", \"edge_feature_gelus_per_clk_per_sm\": %.2f",
             (double)per_sm * 8 * 32 * iters * CH * 2 / mx);
  }
  printf("}\n");
  cudaFree(dc);
  cudaFree(ds);
  delete[] hc;
  return 0;
}
