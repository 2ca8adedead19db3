// C ABI entry points of liblbmgnn.so: argument validation, buffer
// ping-pong, and dispatch to the kernel launchers.  See include/lbmgnn.h for
// the meaning of every argument.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "launch.h"
#include "trace.h"

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

// Side stream and events of lbm_step_bgk_host, created once per device and
// kept for the life of the process.  Enqueueing is serialised by a mutex;
// an event may be re-recorded as soon as the waits on it are enqueued.
#ifndef LBM_HOST_CHUNKS
#define LBM_HOST_CHUNKS 16  // row blocks of the host copies (swept: 8, 16, 32, 64)
#endif
constexpr int HOST_CHUNKS = LBM_HOST_CHUNKS;
struct HostPipe {
  bool ready = false;
  cudaStream_t copy = nullptr;      // host-to-device row blocks
  cudaStream_t copy_out = nullptr;  // device-to-host row blocks of the final state
  cudaEvent_t entry = nullptr;
  cudaEvent_t out_done = nullptr;
  cudaEvent_t arrived[HOST_CHUNKS] = {};
  cudaEvent_t stepped[HOST_CHUNKS] = {};
};
std::mutex g_pipe_mu;
HostPipe g_pipe[64];

HostPipe* host_pipe() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  HostPipe& p = g_pipe[dev];
  if (!p.ready) {
    if (cudaStreamCreateWithFlags(&p.copy, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaStreamCreateWithFlags(&p.copy_out, cudaStreamNonBlocking) != cudaSuccess)
      return nullptr;
    if (cudaEventCreateWithFlags(&p.entry, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&p.out_done, cudaEventDisableTiming) != cudaSuccess)
      return nullptr;
    for (auto& e : p.arrived)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    for (auto& e : p.stepped)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    p.ready = true;
  }
  return &p;
}

// Workspace of lbm_step_bgk_host: two population buffers, the FP64 totals
// (256 bytes) and the per-lattice taus (nb floats), each 256-byte aligned.
int64_t host_ws_bytes(const Shape& s) {
  return 2 * ((f_bytes(s) + 255) / 256 * 256) + 256 + ((int64_t)s.nb * 4 + 255) / 256 * 256;
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

int lbm_version(int* abi, int* packed_layout) {
  if (abi) *abi = LBM_ABI_VERSION;
  if (packed_layout) *packed_layout = LBM_PACKED_LAYOUT_VERSION;
  return LBM_OK;
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
  if (v & ST_BLOB) return LBM_ERR_BLOB;
  if (v & ST_NONFINITE) return LBM_ERR_NONFINITE;
  return LBM_OK;
}

int lbm_init_tgv(float* f, lbm_shape shape, double rho0, double u0, double kx, double ky,
                 int pressure_consistent, void* stream) {
  LBM_TRACE("lbm_init_tgv");
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
  LBM_TRACE("lbm_step_bgk");
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
  LBM_TRACE("lbm_step_channel");
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
  LBM_TRACE("lbm_moments");
  Shape s;
  if (!f) return LBM_ERR_ARG;
  if (int r = check_shape(shape, &s)) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (totals && cudaMemsetAsync(totals, 0, 5 * sizeof(double), st) != cudaSuccess)
    return LBM_ERR_CUDA;
  return cuda_status(launch_moments(f, s, rho, ux, uy, totals, st));
}

size_t lbm_host_workspace_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape(shape, &s)) return 0;
  return (size_t)host_ws_bytes(s);
}

int lbm_step_bgk_host(const float* f_in_host, float* f_out_host, lbm_shape shape, float tau,
                      const float* taus_host, int nsteps, double* totals_host, void* workspace,
                      size_t ws_bytes, void* stream) {
  LBM_TRACE("lbm_step_bgk_host");
  Shape s;
  if (!f_in_host || nsteps < 1) return LBM_ERR_ARG;
  if (int r = check_shape(shape, &s)) return r;
  if (taus_host) {
    for (int b = 0; b < s.nb; ++b)
      if (int r = check_tau(taus_host[b])) return r;
  } else if (int r = check_tau(tau)) {
    return r;
  }
  if (!workspace || (int64_t)ws_bytes < host_ws_bytes(s) ||
      (uintptr_t)workspace % 256 != 0)
    return LBM_ERR_WORKSPACE;
  const int64_t fb = (f_bytes(s) + 255) / 256 * 256;
  auto* w = static_cast<char*>(workspace);
  float* da = reinterpret_cast<float*>(w);
  float* db = reinterpret_cast<float*>(w + fb);
  double* dtot = reinterpret_cast<double*>(w + 2 * fb);
  // per-lattice taus are copied from host memory into the workspace
  float* dtaus = taus_host ? reinterpret_cast<float*>(w + 2 * fb + 256) : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  std::lock_guard<std::mutex> lock(g_pipe_mu);
  HostPipe* p = host_pipe();
  if (!p) return LBM_ERR_CUDA;
  // Row blocks: rows [r0, r1) of the nb*ny lattice rows; block c can take
  // its first step once every row it pulls from (y -+ 1 with periodic wrap,
  // inside its own lattice) has arrived.
  const int64_t rows = (int64_t)s.nb * s.ny;
  const int nc = (int)std::min<int64_t>(HOST_CHUNKS, rows);
  const int64_t per = (rows + nc - 1) / nc;
  auto chunk_of = [&](int64_t r) { return (int)(r / per); };
  std::vector<int> need(nc, 0);
  for (int64_t r = 0; r < rows; ++r) {
    const int64_t b = r / s.ny, y = r - b * s.ny;
    const int64_t up = b * s.ny + (y + 1 == s.ny ? 0 : y + 1);
    const int64_t dn = b * s.ny + (y == 0 ? s.ny - 1 : y - 1);
    int& n = need[chunk_of(r)];
    n = std::max({n, chunk_of(r), chunk_of(up), chunk_of(dn)});
  }
  const int used = (int)((rows + per - 1) / per);

  if (cudaEventRecord(p->entry, st) != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaStreamWaitEvent(p->copy, p->entry, 0) != cudaSuccess) return LBM_ERR_CUDA;
  if (dtaus && cudaMemcpyAsync(dtaus, taus_host, s.nb * sizeof(float), cudaMemcpyHostToDevice,
                               st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (totals_host && cudaMemsetAsync(dtot, 0, 5 * sizeof(double), st) != cudaSuccess)
    return LBM_ERR_CUDA;
  // rows [r0, r1) of all 9 planes between host and device (one 2D copy)
  auto copy_rows = [&](float* dst, const float* src, int c, cudaMemcpyKind kind,
                       cudaStream_t cs) -> bool {
    const int64_t r0 = c * per, r1 = std::min(rows, r0 + per);
    const size_t width = (size_t)((r1 - r0) * s.nx) * sizeof(float);
    const size_t pitch = (size_t)s.ps * sizeof(float);
    const int64_t off = r0 * s.nx;
    if (pitch < (size_t(1) << 31))
      return cudaMemcpy2DAsync(dst + off, pitch, src + off, pitch, width, Q, kind, cs) ==
             cudaSuccess;
    for (int q = 0; q < Q; ++q)
      if (cudaMemcpyAsync(dst + q * s.ps + off, src + q * s.ps + off, width, kind, cs) !=
          cudaSuccess)
        return false;
    return true;
  };
  for (int c = 0; c < used; ++c) {
    if (!copy_rows(da, f_in_host, c, cudaMemcpyHostToDevice, p->copy)) return LBM_ERR_CUDA;
    if (cudaEventRecord(p->arrived[c], p->copy) != cudaSuccess) return LBM_ERR_CUDA;
  }
  // The final step is launched block by block; each block's rows of the final
  // state go back to the host on copy_out as soon as its kernel is done, so
  // the device-to-host copy overlaps the rest of the step (and, on the first
  // step, the host-to-device copy of the remaining blocks).
  auto block_done = [&](float* fin_dev, int c) -> bool {
    if (!f_out_host) return true;
    return cudaEventRecord(p->stepped[c], st) == cudaSuccess &&
           cudaStreamWaitEvent(p->copy_out, p->stepped[c], 0) == cudaSuccess &&
           copy_rows(f_out_host, fin_dev, c, cudaMemcpyDeviceToHost, p->copy_out);
  };
  // first step, block by block in order of readiness
  std::vector<int> order(used);
  for (int c = 0; c < used; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return need[a] < need[b]; });
  int waited = -1;
  double* tot1 = (nsteps == 1 && totals_host) ? dtot : nullptr;
  for (int c : order) {
    if (need[c] > waited) {
      if (cudaStreamWaitEvent(st, p->arrived[need[c]], 0) != cudaSuccess) return LBM_ERR_CUDA;
      waited = need[c];
    }
    const int64_t r0 = c * per, r1 = std::min(rows, r0 + per);
    if (launch_bgk_step_rows(da, db, s, tau, dtaus, tot1, r0, r1, st) != cudaSuccess)
      return LBM_ERR_CUDA;
    if (nsteps == 1 && !block_done(db, c)) return LBM_ERR_CUDA;
  }
  // (need[c] >= c, so st has waited for the last block: the copy stream has
  // no work left that st does not wait for.)  Remaining steps: db -> da -> ...
  float* src = db;
  float* dst = da;
  for (int k = 1; k < nsteps; ++k) {
    const bool last = (k == nsteps - 1);
    double* tk = (last && totals_host) ? dtot : nullptr;
    if (last && f_out_host) {
      for (int c = 0; c < used; ++c) {
        const int64_t r0 = c * per, r1 = std::min(rows, r0 + per);
        if (launch_bgk_step_rows(src, dst, s, tau, dtaus, tk, r0, r1, st) != cudaSuccess ||
            !block_done(dst, c))
          return LBM_ERR_CUDA;
      }
    } else if (launch_bgk_step(src, dst, s, tau, dtaus, tk, st) != cudaSuccess) {
      return LBM_ERR_CUDA;
    }
    std::swap(src, dst);
  }
  if (totals_host && cudaMemcpyAsync(totals_host, dtot, 5 * sizeof(double),
                                     cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (f_out_host) {  // the caller's stream completes only after the last block is back
    if (cudaEventRecord(p->out_done, p->copy_out) != cudaSuccess ||
        cudaStreamWaitEvent(st, p->out_done, 0) != cudaSuccess)
      return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

}  // extern "C"
