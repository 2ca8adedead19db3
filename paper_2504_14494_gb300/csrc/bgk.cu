// D2Q9 BGK kernels: Taylor-Green initial state, the fused pull-stream +
// moments + equilibrium + BGK relaxation step, and the moments/totals pass.
//
// Paper: Sec. 2.1 Eq. 1 (BGK), Eq. 2 (equilibrium), Fig. 1 (loop order),
// Sec. 3.2 (Taylor-Green vortex).
//
// The step is HBM-bound: 9 FP32 loads and 9 FP32 stores per node (72 B).
// The fast kernel gives each warp 128 consecutive nodes of one row (4 per
// lane, 16-byte vector loads and stores).  The x +- 1 shifted planes reuse
// the aligned vector of the lane and take the one missing value from the
// neighbouring lane by a shuffle; the warp's edge lanes fetch it with a
// scalar load (which also implements the periodic wrap).  Row wrap is a select.
#include <atomic>

#include "common.cuh"
#include "launch.h"

namespace lbmgnn {

__device__ unsigned g_status = 0;

unsigned* status_word() {
  // per-device cache of the symbol's address (host threads may race on the
  // first call: both store the same address)
  static std::atomic<unsigned*> addr[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  unsigned* a = addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    a = static_cast<unsigned*>(p);
    addr[dev].store(a, std::memory_order_release);
  }
  return a;
}

// ---------------------------------------------------------------------------
// Fast step: nx % 4 == 0, plane stride % 4 == 0, 16-byte aligned buffers.
template <bool TOTALS>
__global__ void __launch_bounds__(128) bgk_step_x4(const float* __restrict__ fin,
                                                   float* __restrict__ fout, Shape s, float tau,
                                                   const float* __restrict__ taus,
                                                   double* __restrict__ totals, unsigned* stw,
                                                   int64_t row0, int64_t row1) {
  // Rows row0 .. row1-1 of the nb*ny lattice rows are updated.
  const int lane = threadIdx.x & 31;
  const int64_t wid = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int nchunk = (s.nx + 127) >> 7;
  int64_t row = row0 + wid / nchunk;
  const int chunk = (int)(wid % nchunk);
  const bool warp_on = row < row1;
  if (!warp_on) row = row1 - 1;
  const int x0 = chunk * 128 + lane * 4;
  const bool on = warp_on && x0 < s.nx;
  const int xl = on ? x0 : s.nx - 4;  // in-range position for idle lanes
  const int b = (int)(row / s.ny);
  const int y = (int)(row - (int64_t)b * s.ny);
  const int64_t lat = (int64_t)b * s.ny * s.nx;
  const int ym = (y == 0) ? s.ny - 1 : y - 1;
  const int yp = (y == s.ny - 1) ? 0 : y + 1;
  const int64_t r0 = lat + (int64_t)y * s.nx;
  const int64_t rm = lat + (int64_t)ym * s.nx;  // source row of e_y = +1
  const int64_t rp = lat + (int64_t)yp * s.nx;  // source row of e_y = -1
  const int xm = (xl == 0) ? s.nx - 1 : xl - 1;          // source of e_x = +1 (lane edge)
  const int xr = (xl + 4 >= s.nx) ? xl + 4 - s.nx : xl + 4;  // source of e_x = -1 (lane edge)
  const bool need_l = (lane == 0);
  const bool need_r = (lane == 31) || (xl + 4 >= s.nx);
  const int64_t ps = s.ps;

  const int64_t nn4 = (int64_t)s.nb * s.ny * s.nx - 3;  // last valid start of a 4-vector
  const int64_t nn1 = nn4 + 3;
  auto v4 = [&](int q, int64_t r) {
    return __ldg(reinterpret_cast<const float4*>(fin + q * ps + checked(r + xl, 0, nn4, stw)));
  };
  const float4 c0 = v4(0, r0), c1 = v4(1, r0), c2 = v4(2, rm), c3 = v4(3, r0), c4 = v4(4, rp);
  const float4 c5 = v4(5, rm), c6 = v4(6, rm), c7 = v4(7, rp), c8 = v4(8, rp);
  // lane-edge scalars (predicated loads)
  float l1 = 0.f, l5 = 0.f, l8 = 0.f, e3 = 0.f, e6 = 0.f, e7 = 0.f;
  if (need_l) {
    l1 = __ldg(fin + 1 * ps + checked(r0 + xm, 0, nn1, stw));
    l5 = __ldg(fin + 5 * ps + checked(rm + xm, 0, nn1, stw));
    l8 = __ldg(fin + 8 * ps + checked(rp + xm, 0, nn1, stw));
  }
  if (need_r) {
    e3 = __ldg(fin + 3 * ps + checked(r0 + xr, 0, nn1, stw));
    e6 = __ldg(fin + 6 * ps + checked(rm + xr, 0, nn1, stw));
    e7 = __ldg(fin + 7 * ps + checked(rp + xr, 0, nn1, stw));
  }
  const float s1 = __shfl_up_sync(0xffffffffu, c1.w, 1);
  const float s5 = __shfl_up_sync(0xffffffffu, c5.w, 1);
  const float s8 = __shfl_up_sync(0xffffffffu, c8.w, 1);
  const float s3 = __shfl_down_sync(0xffffffffu, c3.x, 1);
  const float s6 = __shfl_down_sync(0xffffffffu, c6.x, 1);
  const float s7 = __shfl_down_sync(0xffffffffu, c7.x, 1);
  if (!need_l) { l1 = s1; l5 = s5; l8 = s8; }
  if (!need_r) { e3 = s3; e6 = s6; e7 = s7; }

  float f[4][Q] = {
      {c0.x, l1, c2.x, c3.y, c4.x, l5, c6.y, c7.y, l8},
      {c0.y, c1.x, c2.y, c3.z, c4.y, c5.x, c6.z, c7.z, c8.x},
      {c0.z, c1.y, c2.z, c3.w, c4.z, c5.y, c6.w, c7.w, c8.y},
      {c0.w, c1.z, c2.w, e3, c4.w, c5.z, e6, e7, c8.z}};
  const float omega = 1.0f / (taus ? __ldg(taus + b) : tau);
#pragma unroll
  for (int j = 0; j < 4; ++j) bgk_collide(f[j], omega);
  if (on) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      *reinterpret_cast<float4*>(fout + q * ps + r0 + x0) =
          make_float4(f[0][q], f[1][q], f[2][q], f[3][q]);
    }
  }
  if constexpr (TOTALS) {
    NodeTotals t;
    if (on) {
#pragma unroll
      for (int j = 0; j < 4; ++j) t.add(f[j]);
    }
    if (t.bad) raise_status(stw, ST_NONFINITE);
    t.flush<128>(totals);
  }
}

// General step: any nx, ny, stride, alignment.  One thread per node.
template <bool TOTALS>
__global__ void __launch_bounds__(256) bgk_step_any(const float* __restrict__ fin,
                                                    float* __restrict__ fout, Shape s, float tau,
                                                    const float* __restrict__ taus,
                                                    double* __restrict__ totals, unsigned* stw,
                                                    int64_t row0, int64_t row1) {
  // Nodes of rows row0 .. row1-1 of the nb*ny lattice rows are updated.
  const int64_t N = row1 * s.nx;
  const int64_t n = row0 * s.nx + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
    int xs = x - ex(q), ys = y - ey(q);
    xs = xs < 0 ? xs + s.nx : (xs >= s.nx ? xs - s.nx : xs);
    ys = ys < 0 ? ys + s.ny : (ys >= s.ny ? ys - s.ny : ys);
    f[q] = __ldg(fin + q * s.ps + checked(lat + (int64_t)ys * s.nx + xs, 0, N, stw));
  }
  bgk_collide(f, 1.0f / (taus ? __ldg(taus + b) : tau));
  if (on) {
#pragma unroll
    for (int q = 0; q < Q; ++q) fout[q * s.ps + nn] = f[q];
  }
  if constexpr (TOTALS) {
    NodeTotals t;
    if (on) t.add(f);
    if (t.bad) raise_status(stw, ST_NONFINITE);
    t.flush<256>(totals);
  }
}

// ---------------------------------------------------------------------------
// Moments of a stored state and FP64 totals.
__global__ void __launch_bounds__(256) moments_kernel(const float* __restrict__ f, Shape s,
                                                      float* __restrict__ rho,
                                                      float* __restrict__ ux,
                                                      float* __restrict__ uy,
                                                      double* __restrict__ totals, unsigned* stw) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = n < N;
  const int64_t nn = on ? n : N - 1;
  float v[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) v[q] = __ldg(f + q * s.ps + nn);
  const Moments m = moments9(v);
  if (on) {
    if (rho) rho[nn] = m.rho;
    if (ux) ux[nn] = m.ux;
    if (uy) uy[nn] = m.uy;
  }
  if (totals) {
    NodeTotals t;
    if (on) t.add(v);
    if (t.bad) raise_status(stw, ST_NONFINITE);
    t.flush<256>(totals);
  }
}

// Taylor-Green initial state, FP64 arithmetic, FP32 store.
__global__ void __launch_bounds__(256) tgv_init_kernel(float* __restrict__ f, Shape s, double rho0,
                                                       double u0, double kx, double ky, int pc) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % s.nx);
  const int y = (int)((n / s.nx) % s.ny);
  double sx, cx, sy, cy;
  sincos(kx * x, &sx, &cx);
  sincos(ky * y, &sy, &cy);
  const double ux = u0 * cx * sy;
  const double uy = -u0 * sx * cy;
  double rho = rho0;
  if (pc) rho = rho0 * (1.0 - 0.75 * u0 * u0 * ((cx * cx - sx * sx) + (cy * cy - sy * sy)));
  const double usq = ux * ux + uy * uy;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const double eu = ex(q) * ux + ey(q) * uy;
    const double w = q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    f[q * s.ps + n] = (float)(w * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
  }
}

// ---------------------------------------------------------------------------
// Launchers
static inline bool x4_ok(const float* a, const float* b, const Shape& s) {
  return (s.nx % 4 == 0) && (s.ps % 4 == 0) && ((uintptr_t)a % 16 == 0) &&
         ((uintptr_t)b % 16 == 0);
}

cudaError_t launch_bgk_step_rows(const float* fin, float* fout, const Shape& s, float tau,
                                 const float* taus, double* totals, int64_t row0, int64_t row1,
                                 cudaStream_t st) {
  if (row0 < 0 || row1 > (int64_t)s.nb * s.ny || row0 >= row1) return cudaErrorInvalidValue;
  unsigned* stw = status_word();
  if (totals && !stw) return cudaErrorInvalidDevice;
  const int64_t rows = row1 - row0;
  if (x4_ok(fin, fout, s)) {
    const int64_t warps = rows * ((s.nx + 127) / 128);
    const unsigned blocks = (unsigned)((warps + 3) / 4);
    if (totals)
      bgk_step_x4<true><<<blocks, 128, 0, st>>>(fin, fout, s, tau, taus, totals, stw, row0, row1);
    else
      bgk_step_x4<false><<<blocks, 128, 0, st>>>(fin, fout, s, tau, taus, totals, stw, row0,
                                                 row1);
  } else {
    const unsigned blocks = (unsigned)((rows * s.nx + 255) / 256);
    if (totals)
      bgk_step_any<true><<<blocks, 256, 0, st>>>(fin, fout, s, tau, taus, totals, stw, row0,
                                                 row1);
    else
      bgk_step_any<false><<<blocks, 256, 0, st>>>(fin, fout, s, tau, taus, totals, stw, row0,
                                                  row1);
  }
  return cudaGetLastError();
}

cudaError_t launch_bgk_step(const float* fin, float* fout, const Shape& s, float tau,
                            const float* taus, double* totals, cudaStream_t st) {
  return launch_bgk_step_rows(fin, fout, s, tau, taus, totals, 0, (int64_t)s.nb * s.ny, st);
}

cudaError_t launch_moments(const float* f, const Shape& s, float* rho, float* ux, float* uy,
                           double* totals, cudaStream_t st) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  unsigned* stw = status_word();
  if (totals && !stw) return cudaErrorInvalidDevice;
  moments_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(f, s, rho, ux, uy, totals, stw);
  return cudaGetLastError();
}

cudaError_t launch_tgv_init(float* f, const Shape& s, double rho0, double u0, double kx,
                            double ky, int pc, cudaStream_t st) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  tgv_init_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(f, s, rho0, u0, kx, ky, pc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Streaming only (pull with periodic wrap): f_out_i(x) = f_in_i(x - e_i).
__global__ void __launch_bounds__(256) stream_kernel(const float* __restrict__ fin,
                                                     float* __restrict__ fout, Shape s) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % s.nx);
  const int64_t row = n / s.nx;
  const int b = (int)(row / s.ny);
  const int y = (int)(row - (int64_t)b * s.ny);
  const int64_t lat = (int64_t)b * s.ny * s.nx;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int xs = x - ex(q), ys = y - ey(q);
    xs = xs < 0 ? xs + s.nx : (xs >= s.nx ? xs - s.nx : xs);
    ys = ys < 0 ? ys + s.ny : (ys >= s.ny ? ys - s.ny : ys);
    fout[q * s.ps + n] = __ldg(fin + q * s.ps + lat + (int64_t)ys * s.nx + xs);
  }
}

// Restriction of an m-times refined post-collision state to the coarse
// lattice: inject rho, u of fine node (m X, m Y); rescale the non-equilibrium
// part, f_neq_c = m (tau_c / tau_f) (f*_f - f^eq) / (1 - 1/tau_f);
// f*_c = f^eq + (1 - 1/tau_c) f_neq_c.
__global__ void __launch_bounds__(256) restrict_kernel(const float* __restrict__ ff, Shape fs,
                                                       float* __restrict__ fc, Shape cs, int m,
                                                       float tau_f, const float* __restrict__ taus_f,
                                                       float tau_c, const float* __restrict__ taus_c) {
  const int64_t N = (int64_t)cs.nb * cs.ny * cs.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int X = (int)(n % cs.nx);
  const int64_t row = n / cs.nx;
  const int b = (int)(row / cs.ny);
  const int Y = (int)(row - (int64_t)b * cs.ny);
  const int64_t src = ((int64_t)b * fs.ny + (int64_t)m * Y) * fs.nx + (int64_t)m * X;
  float f[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) f[q] = __ldg(ff + q * fs.ps + src);
  const float tf = taus_f ? __ldg(taus_f + b) : tau_f;
  const float tc = taus_c ? __ldg(taus_c + b) : tau_c;
  const Moments mm = moments9(f);
  const float usq15 = 1.5f * (mm.ux * mm.ux + mm.uy * mm.uy);
  const float scale = (1.0f - 1.0f / tc) * (float)m * (tc / tf) / (1.0f - 1.0f / tf);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float fe = feq_i(q, mm, usq15);
    fc[q * cs.ps + n] = fe + scale * (f[q] - fe);
  }
}

// Taylor-Green initial state with per-lattice parameters p[b] = (rho0, u0, kx, ky).
__global__ void __launch_bounds__(256) tgv_init_batch_kernel(float* __restrict__ f, Shape s,
                                                             const double* __restrict__ prm,
                                                             int pc) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int x = (int)(n % s.nx);
  const int64_t row = n / s.nx;
  const int b = (int)(row / s.ny);
  const int y = (int)(row - (int64_t)b * s.ny);
  const double rho0 = prm[4 * b], u0 = prm[4 * b + 1], kx = prm[4 * b + 2], ky = prm[4 * b + 3];
  double sx, cx, sy, cy;
  sincos(kx * x, &sx, &cx);
  sincos(ky * y, &sy, &cy);
  const double ux = u0 * cx * sy;
  const double uy = -u0 * sx * cy;
  double rho = rho0;
  if (pc) rho = rho0 * (1.0 - 0.75 * u0 * u0 * ((cx * cx - sx * sx) + (cy * cy - sy * sy)));
  const double usq = ux * ux + uy * uy;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const double eu = ex(q) * ux + ey(q) * uy;
    const double w = q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    f[q * s.ps + n] = (float)(w * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
  }
}

cudaError_t launch_stream(const float* fin, float* fout, const Shape& s, cudaStream_t st) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  stream_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(fin, fout, s);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const float* ff, const Shape& fs, float* fc, const Shape& cs, int m,
                            float tau_f, const float* taus_f, float tau_c, const float* taus_c,
                            cudaStream_t st) {
  const int64_t N = (int64_t)cs.nb * cs.ny * cs.nx;
  restrict_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(ff, fs, fc, cs, m, tau_f, taus_f,
                                                               tau_c, taus_c);
  return cudaGetLastError();
}

cudaError_t launch_tgv_init_batch(float* f, const Shape& s, const double* prm, int pc,
                                  cudaStream_t st) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  tgv_init_batch_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(f, s, prm, pc);
  return cudaGetLastError();
}

}  // namespace lbmgnn
