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
// the direction opposite to e_i
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}

// Device status word: bit flags raised by kernels, read (and cleared) by
// lbm_get_status().  One per device that loaded the library; kernels receive
// its address as an argument (status_word() returns it for the current
// device).
enum : unsigned {
  ST_NONFINITE = 1u << 0,
  ST_TIMEOUT = 1u << 1,
  ST_BOUNDS = 1u << 2,
  ST_BLOB = 1u << 3,  // a kernel was given a packed parameter image without its validity word
};
unsigned* status_word();

__device__ __forceinline__ void raise_status(unsigned* w, unsigned bits) { atomicOr(w, bits); }

// Bounds-checked builds (-DLBM_BOUNDS_CHECK, liblbmgnn_checked.so): a computed
// gather index outside [lo, hi) raises ST_BOUNDS and is replaced by lo, so
// the access stays inside the buffer and the run goes on; the regular build
// compiles the check away.  (The pool offers no memory checker; this build
// plus small cases and the oracle stand in for one.)
__device__ __forceinline__ int64_t checked(int64_t i, int64_t lo, int64_t hi, unsigned* stw) {
#ifdef LBM_BOUNDS_CHECK
  if (i < lo || i >= hi) {
    raise_status(stw, ST_BOUNDS);
    return lo;
  }
#endif
  return i;
}

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

// ---- totals (mass, momentum, kinetic energy) at FP64 accuracy -------------
// GB300 runs FP64 at a small fraction of its FP32 rate, so the per-node sums
// of the totals are carried as unevaluated pairs hi + lo of FP32 values
// ("double-float"): each addition is Knuth's error-free TwoSum (s + e equals
// a + b exactly), the rounding errors collect in lo, and the pair is
// renormalised by another TwoSum once per node.  About 2^-46 relative error
// per node; FP64 arithmetic is used once per warp.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_add(DF& a, float x) {  // a += x (lo not renormalised)
  float s, e;
  two_sum(a.hi, x, s, e);
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ void df_norm(DF& a) {
  float s, e;
  two_sum(a.hi, a.lo, s, e);
  a.hi = s;
  a.lo = e;
}
__device__ __forceinline__ void df_add(DF& a, const DF& b) {  // a += b, renormalised
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(b.lo, e));
  df_norm(a);
}
__device__ __forceinline__ DF df_shfl_xor(const DF& a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Per-thread totals of stored nodes: mass sum f_i, momentum sum f_i e_i,
// kinetic energy sum |j|^2 / (2 rho), and the count of nodes holding a
// non-finite population (excluded from the sums).
struct NodeTotals {
  DF m{0.f, 0.f}, px{0.f, 0.f}, py{0.f, 0.f}, e{0.f, 0.f};
  unsigned bad = 0;

  __device__ __forceinline__ void add(const float (&o)[Q]) {
    bool finite = true;
#pragma unroll
    for (int i = 0; i < Q; ++i) finite &= isfinite(o[i]);
    if (!finite) {
      ++bad;
      return;
    }
    DF r{o[0], 0.f}, jx{0.f, 0.f}, jy{0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      df_add(r, o[i]);
      if (ex(i)) df_add(jx, ex(i) > 0 ? o[i] : -o[i]);
      if (ey(i)) df_add(jy, ey(i) > 0 ? o[i] : -o[i]);
    }
    df_norm(r);
    df_norm(jx);
    df_norm(jy);
    const float en = 0.5f * (jx.hi * jx.hi + jy.hi * jy.hi) / r.hi;
    df_add(m, r);
    df_add(px, jx);
    df_add(py, jy);
    df_add(e, DF{en, 0.f});
  }

  // Sum over the block (NT threads) added to totals[0..4] in FP64.
  template <int NT>
  __device__ __forceinline__ void flush(double* __restrict__ totals) {
    __shared__ double red[NT / 32][5];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df_add(m, df_shfl_xor(m, o));
      df_add(px, df_shfl_xor(px, o));
      df_add(py, df_shfl_xor(py, o));
      df_add(e, df_shfl_xor(e, o));
    }
    const unsigned nbad = __reduce_add_sync(0xffffffffu, bad);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red[w][0] = (double)m.hi + (double)m.lo;
      red[w][1] = (double)px.hi + (double)px.lo;
      red[w][2] = (double)py.hi + (double)py.lo;
      red[w][3] = (double)e.hi + (double)e.lo;
      red[w][4] = (double)nbad;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < NT / 32; ++i) acc += red[i][threadIdx.x];
      if (acc != 0.0) atomicAdd(totals + threadIdx.x, acc);
    }
  }
};

struct Shape {
  int nx, ny, nb;
  int64_t ps;  // plane stride in elements
};

}  // namespace lbmgnn
