// Shared device-side definitions of the CUDA library (sm_103a).
//
// D2Q9 lattice (Sec. 2.1 of the paper names w_i and c_s without values; the
// textbook set is used): e_0=(0,0); e_1..4=(1,0),(0,1),(-1,0),(0,-1);
// e_5..8=(1,1),(-1,1),(-1,-1),(1,-1); w = 4/9, 1/9 x4, 1/36 x4; c_s^2 = 1/3.
//
// Population layout: plane q of node (x, y) of lattice b lives at
//   f[q * plane_stride + (b * ny + y) * nx + x]
// i.e. a stack of nb lattices of ny x nx nodes, q-major (SoA), x fastest.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/lbmgnn.h"

namespace lbmgnn {

constexpr int Q = 9;
__host__ __device__ constexpr int ex(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr float wq(int i) {
  return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}

// Device status word: bit flags raised by kernels, read (and cleared) by
// lbm_get_status().  One per device that loaded the library; kernels receive
// its address as an argument (status_word() returns it for the current
// device).
enum : unsigned {
  ST_NONFINITE = 1u << 0,
  ST_TIMEOUT = 1u << 1,
  ST_BOUNDS = 1u << 2,
};
unsigned* status_word();

__device__ __forceinline__ void raise_status(unsigned* w, unsigned bits) { atomicOr(w, bits); }

// Moments of one node: rho = sum f_i, (jx, jy) = sum f_i e_i.
struct Moments {
  float rho, ux, uy;
};

__device__ __forceinline__ Moments moments9(const float (&f)[Q]) {
  const float rho = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
  const float jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
  const float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const float inv = 1.0f / rho;
  return {rho, jx * inv, jy * inv};
}

// Eq. 2 for direction i, with c_s^2 = 1/3:
//   f_i^eq = rho w_i (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u)
__device__ __forceinline__ float feq_i(int i, const Moments& m, float usq15) {
  const float eu = float(ex(i)) * m.ux + float(ey(i)) * m.uy;
  return wq(i) * m.rho * (1.0f + 3.0f * eu + 4.5f * eu * eu - usq15);
}

// BGK collision of one node (Eq. 1 with Eq. 2), in place; omega = 1/tau.
__device__ __forceinline__ void bgk_collide(float (&f)[Q], float omega) {
  const Moments m = moments9(f);
  const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = f[i] - omega * (f[i] - feq_i(i, m, usq15));
}

struct Shape {
  int nx, ny, nb;
  int64_t ps;  // plane stride in elements
};

}  // namespace lbmgnn
