// Per-instance weights of the training loss (this library's training option;
// the paper's Eq. 4 is the plain mean over nodes x 9).
//
// For every lattice b of a stack of training pairs (f_in: coarse state at
// step n, f_target: at n + 1) the one-step residual of the plain method,
//   D_b = mean over the lattice's nodes x 9 of (BGK(stream(f_in)) - f_target)^2,
// measures how far the method without the network is from the refined
// solution on that instance.  The weight w_b = mean_c(D_c) / D_b (capped at
// WMAX) makes each instance count by its error relative to BGK's, so that
// pairs of the developed flow weigh as much as the start-up transient, whose
// residuals are ~1e3 larger.  With these weights the weighted loss of the
// zero network equals the plain Eq. 4 loss.
//
// Three deterministic passes: per (lattice, chunk) partial sums in FP64, one
// fixed-order sum per lattice, and the mean and weights in one CTA.
#include "common.cuh"
#include "gnn.cuh"
#include "gnn_launch.h"

namespace lbmgnn {

constexpr int PW_CHUNKS = 64;       // blocks per lattice (at most)
constexpr float PW_WMAX = 1.0e4f;   // cap of a weight

// Block (chunk, b): squared BGK residual summed over its share of lattice b.
__global__ void __launch_bounds__(256) pair_residual_kernel(
    const float* __restrict__ f_in, const float* __restrict__ tgt, Shape s, float tau0,
    const float* __restrict__ taus, double* __restrict__ part, int chunks, unsigned* stw) {
  const int b = blockIdx.y;
  const int64_t M = (int64_t)s.nx * s.ny, lat = (int64_t)b * M;
  const float omega = 1.0f / (taus ? __ldg(taus + b) : tau0);
  double acc = 0.0;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M;
       m += (int64_t)chunks * blockDim.x) {
    const int y = (int)(m / s.nx), x = (int)(m - (int64_t)y * s.nx);
    const int xm = x == 0 ? s.nx - 1 : x - 1, xp = x == s.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? s.ny - 1 : y - 1, yp = y == s.ny - 1 ? 0 : y + 1;
    float f[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {  // pull from x - e_q
      const int sx = ex(q) > 0 ? xm : (ex(q) < 0 ? xp : x);
      const int sy = ey(q) > 0 ? ym : (ey(q) < 0 ? yp : y);
      f[q] = __ldg(f_in + q * s.ps + checked(lat + (int64_t)sy * s.nx + sx, 0, s.nb * M, stw));
    }
    bgk_collide(f, omega);
    float r2 = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float r = f[q] - __ldg(tgt + q * s.ps + lat + m);
      r2 = fmaf(r, r, r2);
    }
    acc += (double)r2;
  }
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    part[(int64_t)b * chunks + blockIdx.x] = t;
  }
}

// One CTA: D_b (fixed-order sum of the partials, / (9 M)), their mean, and
// w_b = mean / D_b capped at PW_WMAX (a lattice with D_b = 0 gets the cap).
__global__ void __launch_bounds__(256) pair_weights_kernel(const double* __restrict__ part,
                                                           int chunks, int nb, double count,
                                                           double* __restrict__ resid,
                                                           float* __restrict__ w) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < chunks; ++c) t += part[(int64_t)b * chunks + c];
    resid[b] = t / count;
    acc += t / count;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  const double mean = red[0] / nb;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double d = resid[b];
    w[b] = (d * PW_WMAX > mean) ? (float)(mean / d) : PW_WMAX;
  }
}

int64_t pair_weights_ws(const Shape& s) {
  return (int64_t)s.nb * PW_CHUNKS * 8 + (int64_t)s.nb * 8 + 256;
}

cudaError_t launch_pair_weights(const float* f_in, const float* tgt, const Shape& s, float tau,
                                const float* taus, float* w, void* ws, cudaStream_t st) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  const int64_t M = (int64_t)s.nx * s.ny;
  const int64_t want = (M + 2047) / 2048;
  const int chunks = (int)(want < PW_CHUNKS ? want : PW_CHUNKS);
  double* part = static_cast<double*>(ws);
  double* resid = part + (int64_t)s.nb * PW_CHUNKS;
  pair_residual_kernel<<<dim3(chunks, s.nb), 256, 0, st>>>(f_in, tgt, s, tau, taus, part, chunks,
                                                           stw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  pair_weights_kernel<<<1, 256, 0, st>>>(part, chunks, s.nb, 9.0 * (double)M, resid, w);
  return cudaGetLastError();
}

}  // namespace lbmgnn
