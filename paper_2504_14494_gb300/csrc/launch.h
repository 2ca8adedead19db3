// Internal launchers shared between the kernel files and the C ABI layer.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace lbmgnn {

cudaError_t launch_bgk_step(const float* fin, float* fout, const Shape& s, float tau,
                            const float* taus, double* totals, cudaStream_t st);
// The step restricted to lattice rows row0 .. row1-1 (of the nb*ny rows).
cudaError_t launch_bgk_step_rows(const float* fin, float* fout, const Shape& s, float tau,
                                 const float* taus, double* totals, int64_t row0, int64_t row1,
                                 cudaStream_t st);
cudaError_t launch_moments(const float* f, const Shape& s, float* rho, float* ux, float* uy,
                           double* totals, cudaStream_t st);
cudaError_t launch_tgv_init(float* f, const Shape& s, double rho0, double u0, double kx,
                            double ky, int pc, cudaStream_t st);

cudaError_t launch_channel_step(const float* fin, float* fout, const Shape& s, float tau,
                                const float* taus, float gx, double* totals, cudaStream_t st);
cudaError_t launch_stream(const float* fin, float* fout, const Shape& s, cudaStream_t st);
cudaError_t launch_restrict(const float* ff, const Shape& fs, float* fc, const Shape& cs, int m,
                            float tau_f, const float* taus_f, float tau_c, const float* taus_c,
                            cudaStream_t st);
cudaError_t launch_tgv_init_batch(float* f, const Shape& s, const double* prm, int pc,
                                  cudaStream_t st);

}  // namespace lbmgnn
