// Channel (Poiseuille) flow, paper Sec. 3.1 Eq. 5: the BGK step with walls
// and a body force.  The paper names "Apply Boundary Conditions" (Fig. 1)
// without a scheme; this library uses halfway bounce-back walls at
// y = -1/2 and y = ny - 1/2 of every lattice (periodic in x) and Guo's
// forcing for a force (G, 0) per unit volume:
//   u = (sum f_i e_i + F/2) / rho,
//   f*_i = f_i - (f_i - f_i^eq)/tau + (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i].F
// In pull form the bounce-back reads f_i(x, y) = f*_opp(i)(x, y) whenever
// (x - e_ix, y - e_iy) lies outside the channel.
#include "common.cuh"
#include "launch.h"

namespace lbmgnn {

__device__ __forceinline__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}

template <bool TOTALS>
__global__ void __launch_bounds__(256) channel_step_kernel(const float* __restrict__ fin,
                                                           float* __restrict__ fout, Shape s,
                                                           float tau, const float* __restrict__ taus,
                                                           float gx, double* __restrict__ totals,
                                                           unsigned* stw) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = n < N;
  const int64_t nn = on ? n : N - 1;
  const int x = (int)(nn % s.nx);
  const int64_t row = nn / s.nx;
  const int b = (int)(row / s.ny);
  const int y = (int)(row - (int64_t)b * s.ny);
  const int64_t lat = (int64_t)b * s.ny * s.nx;
  float f[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int ys = y - ey(q);
    if (ys < 0 || ys >= s.ny) {
      f[q] = __ldg(fin + opp(q) * s.ps + nn);  // halfway bounce-back
    } else {
      int xs = x - ex(q);
      xs = xs < 0 ? xs + s.nx : (xs >= s.nx ? xs - s.nx : xs);
      f[q] = __ldg(fin + q * s.ps +
                   checked(lat + (int64_t)ys * s.nx + xs, 0, (int64_t)s.nb * s.ny * s.nx, stw));
    }
  }
  const float t = taus ? __ldg(taus + b) : tau;
  const float rho = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
  const float jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
  const float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const float inv = 1.0f / rho;
  const Moments m{rho, (jx + 0.5f * gx) * inv, jy * inv};
  const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
  const float omega = 1.0f / t, pre = 1.0f - 0.5f * omega;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float eu = float(ex(q)) * m.ux + float(ey(q)) * m.uy;
    const float src = pre * wq(q) * (3.0f * (float(ex(q)) - m.ux) + 9.0f * eu * float(ex(q))) * gx;
    f[q] = f[q] - omega * (f[q] - feq_i(q, m, usq15)) + src;
  }
  if (on) {
#pragma unroll
    for (int q = 0; q < Q; ++q) fout[q * s.ps + nn] = f[q];
  }
  if constexpr (TOTALS) {
    double tt[5] = {0, 0, 0, 0, 0};
    if (on) {
      bool finite = true;
#pragma unroll
      for (int q = 0; q < Q; ++q) finite &= isfinite(f[q]);
      if (finite) {
        double r = 0.0, px = 0.0, py = 0.0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          r += f[q];
          if (ex(q)) px += ex(q) * (double)f[q];
          if (ey(q)) py += ey(q) * (double)f[q];
        }
        tt[0] = r;
        tt[1] = px;
        tt[2] = py;
        tt[3] = 0.5 * (px * px + py * py) / r;
      } else {
        tt[4] = 1.0;
      }
    }
    if (tt[4] != 0.0) raise_status(stw, ST_NONFINITE);
    __shared__ double red[8][5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tt[k] += __shfl_xor_sync(0xffffffffu, tt[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k) red[threadIdx.x >> 5][k] = tt[k];
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      double acc = 0.0;
      for (int i = 0; i < 8; ++i) acc += red[i][threadIdx.x];
      if (acc != 0.0) atomicAdd(totals + threadIdx.x, acc);
    }
  }
}

cudaError_t launch_channel_step(const float* fin, float* fout, const Shape& s, float tau,
                                const float* taus, float gx, double* totals, cudaStream_t st) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  unsigned* stw = status_word();
  if (totals && !stw) return cudaErrorInvalidDevice;
  const unsigned blocks = (unsigned)((N + 255) / 256);
  if (totals)
    channel_step_kernel<true><<<blocks, 256, 0, st>>>(fin, fout, s, tau, taus, gx, totals, stw);
  else
    channel_step_kernel<false><<<blocks, 256, 0, st>>>(fin, fout, s, tau, taus, gx, totals, stw);
  return cudaGetLastError();
}

}  // namespace lbmgnn
