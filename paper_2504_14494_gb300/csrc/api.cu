// C ABI entry points of liblbmgnn.so: argument validation, buffer
// ping-pong, and dispatch to the kernel launchers.  See include/lbmgnn.h for
// the meaning of every argument.
#include <cmath>

#include "common.cuh"
#include "launch.h"

using namespace lbmgnn;

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

// Checks a shape and converts it to the internal form.
int check_shape(const lbm_shape& s, Shape* out) {
  if (s.nx < 1 || s.ny < 1 || s.nb < 1) return LBM_ERR_SIZE;
  const int64_t n = (int64_t)s.nx * s.ny * s.nb;
  if (n > (int64_t(1) << 36)) return LBM_ERR_SIZE;
  const int64_t ps = s.plane_stride == 0 ? n : s.plane_stride;
  if (ps < n) return LBM_ERR_SIZE;
  *out = Shape{s.nx, s.ny, s.nb, ps};
  return LBM_OK;
}

int check_tau(float tau) {
  if (!std::isfinite(tau) || !(tau > 0.5f)) return LBM_ERR_TAU;
  return LBM_OK;
}

// Byte extent of one population buffer of shape s.
int64_t f_bytes(const Shape& s) {
  return (8 * s.ps + (int64_t)s.nb * s.ny * s.nx) * (int64_t)sizeof(float);
}

bool overlap(const void* a, const void* b, int64_t bytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bytes && pb < pa + bytes;
}

}  // namespace

extern "C" {

const char* lbm_status_string(int status) {
  switch (status) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_ARG: return "LBM_ERR_ARG: invalid argument";
    case LBM_ERR_ALIAS: return "LBM_ERR_ALIAS: output buffer aliases an input";
    case LBM_ERR_SIZE: return "LBM_ERR_SIZE: lattice shape out of range";
    case LBM_ERR_TAU: return "LBM_ERR_TAU: relaxation time must be > 1/2";
    case LBM_ERR_BLOB: return "LBM_ERR_BLOB: parameter blob of wrong size or version";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA: CUDA runtime error";
    case LBM_ERR_NONFINITE: return "LBM_ERR_NONFINITE: non-finite population produced";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT: device-side wait gave up";
    case LBM_ERR_BOUNDS: return "LBM_ERR_BOUNDS: device-side bounds check failed";
    case LBM_ERR_WORKSPACE: return "LBM_ERR_WORKSPACE: workspace missing or too small";
    default: return "unknown status";
  }
}

int lbm_get_status(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_ERR_CUDA;
  unsigned* w = status_word();
  if (!w) return LBM_ERR_CUDA;
  unsigned v = 0;
  if (cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return LBM_ERR_CUDA;
  if (v != 0 && cudaMemset(w, 0, sizeof(v)) != cudaSuccess) return LBM_ERR_CUDA;
  if (v & ST_TIMEOUT) return LBM_ERR_TIMEOUT;
  if (v & ST_BOUNDS) return LBM_ERR_BOUNDS;
  if (v & ST_NONFINITE) return LBM_ERR_NONFINITE;
  return LBM_OK;
}

int lbm_init_tgv(float* f, lbm_shape shape, double rho0, double u0, double kx, double ky,
                 int pressure_consistent, void* stream) {
  Shape s;
  if (!f) return LBM_ERR_ARG;
  if (int r = check_shape(shape, &s)) return r;
  if (!std::isfinite(rho0) || !std::isfinite(u0) || !std::isfinite(kx) || !std::isfinite(ky) ||
      !(rho0 > 0.0))
    return LBM_ERR_ARG;
  return cuda_status(launch_tgv_init(f, s, rho0, u0, kx, ky, pressure_consistent ? 1 : 0,
                                     static_cast<cudaStream_t>(stream)));
}

int lbm_step_bgk(const float* f_in, float* f_out, float* f_tmp, lbm_shape shape, float tau,
                 const float* taus, int nsteps, double* totals, void* stream) {
  Shape s;
  if (!f_in || !f_out || nsteps < 0) return LBM_ERR_ARG;
  if (int r = check_shape(shape, &s)) return r;
  if (!taus) {
    if (int r = check_tau(tau)) return r;
  }
  const int64_t bytes = f_bytes(s);
  if (overlap(f_in, f_out, bytes)) return LBM_ERR_ALIAS;
  if (nsteps > 1) {
    if (!f_tmp) return LBM_ERR_ARG;
    if (overlap(f_tmp, f_in, bytes) || overlap(f_tmp, f_out, bytes)) return LBM_ERR_ALIAS;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (totals && cudaMemsetAsync(totals, 0, 5 * sizeof(double), st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (nsteps == 0) {
    if (cudaMemcpyAsync(f_out, f_in, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return LBM_ERR_CUDA;
    return totals ? cuda_status(launch_moments(f_out, s, nullptr, nullptr, nullptr, totals, st))
                  : LBM_OK;
  }
  // Ping-pong so that the last step lands in f_out: f_in -> (out|tmp) -> ...
  const float* src = f_in;
  for (int k = 0; k < nsteps; ++k) {
    const int left = nsteps - k;  // steps still to do, this one included
    float* dst = (left % 2 == 1) ? f_out : f_tmp;
    const bool last = (left == 1);
    cudaError_t e = launch_bgk_step(src, dst, s, tau, taus, last ? totals : nullptr, st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    src = dst;
  }
  return LBM_OK;
}

int lbm_step_channel(const float* f_in, float* f_out, float* f_tmp, lbm_shape shape, float tau,
                     const float* taus, float force_x, int nsteps, double* totals, void* stream) {
  Shape s;
  if (!f_in || !f_out || nsteps < 0 || !std::isfinite(force_x)) return LBM_ERR_ARG;
  if (int r = check_shape(shape, &s)) return r;
  if (!taus) {
    if (int r = check_tau(tau)) return r;
  }
  const int64_t bytes = f_bytes(s);
  if (overlap(f_in, f_out, bytes)) return LBM_ERR_ALIAS;
  if (nsteps > 1) {
    if (!f_tmp) return LBM_ERR_ARG;
    if (overlap(f_tmp, f_in, bytes) || overlap(f_tmp, f_out, bytes)) return LBM_ERR_ALIAS;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (totals && cudaMemsetAsync(totals, 0, 5 * sizeof(double), st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (nsteps == 0) {
    if (cudaMemcpyAsync(f_out, f_in, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return LBM_ERR_CUDA;
    return totals ? cuda_status(launch_moments(f_out, s, nullptr, nullptr, nullptr, totals, st))
                  : LBM_OK;
  }
  const float* src = f_in;
  for (int k = 0; k < nsteps; ++k) {
    const int left = nsteps - k;
    float* dst = (left % 2 == 1) ? f_out : f_tmp;
    if (launch_channel_step(src, dst, s, tau, taus, force_x, left == 1 ? totals : nullptr, st) !=
        cudaSuccess)
      return LBM_ERR_CUDA;
    src = dst;
  }
  return LBM_OK;
}

int lbm_moments(const float* f, lbm_shape shape, float* rho, float* ux, float* uy,
                double* totals, void* stream) {
  Shape s;
  if (!f) return LBM_ERR_ARG;
  if (int r = check_shape(shape, &s)) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (totals && cudaMemsetAsync(totals, 0, 5 * sizeof(double), st) != cudaSuccess)
    return LBM_ERR_CUDA;
  return cuda_status(launch_moments(f, s, rho, ux, uy, totals, st));
}

}  // extern "C"
