// The paper's Fig. 2 network (SimpleLBMGNN: features -> Linear + ReLU ->
// Linear + ReLU -> heads, no message passing; Sec. 2.3.1) as ONE fused
// GNN-LBM step kernel: pull-stream of the stored state, moments, features,
// the three dense layers on the tensor cores, the heads and the Eq. 3
// collision, and the store.  Per node it moves only the populations (9 FP32
// loads, 9 FP32 stores: 72 bytes), like the BGK step.
//
// Work unit: a tile of 128 consecutive nodes; a CTA of 128 threads (thread t
// = node t of the tile, warp w reads tensor-memory lanes 32w..32w+31) loops
// over tiles (persistent grid, several CTAs per SM).  The pulled populations
// of the next two tiles are fetched with 4-byte cp.async copies into a
// 3-stage shared-memory ring, so the loads are in flight while the current
// tile runs its three MMAs (M = 128 nodes, BF16 operands in 128-byte
// swizzled shared memory, FP32 accumulators in 64 tensor-memory columns):
//   D = [x_hi | x_lo] W1x^T   (K = 32: the FP32 features split into two BF16
//                              parts, ~16 bits kept)          -> ReLU(+b1)
//   D = g1 W2^T               (K = 64)                        -> ReLU(+b2)
//   D = h0 Wh^T               (K = 64, N = 16, 10 used)       -> y (+bh)
// and f* = f - (f - f^eq)/(tau tau_adj) + s_df y_1..9 (Eq. 3).  The one
// activation tile is reused by the three products (each epilogue writes it
// after the MMA that read it has completed).
#include "gnn.cuh"
#include "gnn_launch.h"

namespace lbmgnn {

namespace mlp {
constexpr int STAGES = 3;
constexpr int SLOTS = Q + 1;  // per node and stage: the 9 pulled populations and tau
constexpr uint32_t W1X = 0, W2 = 8192, ACT = 16384, WH = 32768, STG = 34816,
                   STG_BYTES = SLOTS * TILE * 4,                   // 5120 per stage
                   B2 = STG + STAGES * STG_BYTES,                  // 50176
                   BH = B2 + 256, NORM = BH + 64, SH = NORM + 128, BYTES = SH + 64;
}  // namespace mlp

#ifndef LBM_MLP_CTAS
#define LBM_MLP_CTAS 4  // resident CTAs per SM
#endif

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// ReLU(a), ReLU(b) rounded to BF16 and packed (a in the low half): one
// conversion instruction for both values (rounding commutes with ReLU).
__device__ __forceinline__ uint32_t relu_bf16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
__device__ __forceinline__ uint32_t bf16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// ReLU of 32 accumulator columns (plus a bias, if given) rounded to BF16 and
// stored into chunks c0 .. c0+3 of the swizzled activation row.
__device__ __forceinline__ void relu_row32(uint8_t* act, int row, int c0, const float (&z)[32],
                                           const float* b) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float2 v = make_float2(z[8 * c + 2 * j], z[8 * c + 2 * j + 1]);
      if (b) v = __fadd2_rn(v, *reinterpret_cast<const float2*>(b + 8 * c + 2 * j));
      w[j] = relu_bf16x2(v.x, v.y);
    }
    *reinterpret_cast<uint4*>(act + row * 128 + (((c0 + c) ^ (row & 7)) << 4)) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <class Geo>
__global__ void __launch_bounds__(128, LBM_MLP_CTAS) gnn_mlp_step_kernel(
    const float* __restrict__ f_in, float* __restrict__ f_out, Geo geo, float tau0,
    const float* __restrict__ taus, const uint8_t* __restrict__ packed, bool require_mlp,
    unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  const int variant = variant_of(reinterpret_cast<const float*>(packed + K::NORM));
  if (!(variant & VAR_MLP_ONLY)) {  // message-passing networks: the unfused kernels
    if (require_mlp && threadIdx.x == 0) raise_status(stw, ST_BLOB);
    return;
  }
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  TcShared* sh = reinterpret_cast<TcShared*>(sm + mlp::SH);
  float* stg = reinterpret_cast<float*>(sm + mlp::STG);
  const int t = threadIdx.x;
  const int64_t N = geo.count();
  const int64_t base = geo.base(), ps = geo.ps();
  const int64_t ntiles = (N + TILE - 1) / TILE;
  const int64_t first = blockIdx.x, stride = gridDim.x;

  // Node t of tile `tile` -> stage st (cp.async): its 9 populations pulled
  // from x - e_q (periodic wrap inside its lattice) and its relaxation time.
  auto fetch = [&](int64_t tile, int st) {
    if (tile < ntiles) {
      const int64_t m = tile * TILE + t;
      const GeoPos p = geo.pos(base + (m < N ? m : N - 1));
      const int xm = p.x == 0 ? p.nx - 1 : p.x - 1, xp = p.x == p.nx - 1 ? 0 : p.x + 1;
      const int64_t r0 = p.lat + (int64_t)p.y * p.nx;
      const int64_t rm = p.lat + (int64_t)(p.y == 0 ? p.ny - 1 : p.y - 1) * p.nx;
      const int64_t rp = p.lat + (int64_t)(p.y == p.ny - 1 ? 0 : p.y + 1) * p.nx;
      // source of q: (x, y) (x-1, y) (x, y-1) (x+1, y) (x, y+1) (x-1, y-1) (x+1, y-1)
      // (x+1, y+1) (x-1, y+1)
      const int64_t src[Q] = {r0 + p.x, r0 + xm, rm + p.x, r0 + xp, rp + p.x,
                              rm + xm,  rm + xp, rp + xp,  rp + xm};
      float* d = stg + st * (mlp::SLOTS * TILE) + t;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        cp_async4(d + q * TILE, f_in + q * ps + checked(src[q], base, base + N, stw));
      const float* tp = geo.tau_ptr(p, taus);
      if (tp) cp_async4(d + Q * TILE, tp); else d[Q * TILE] = tau0;
    }
    cp_async_commit();  // (an empty group past the last tile keeps the counting uniform)
  };
  fetch(first, 0);
  fetch(first + stride, 1);

  copy_g2s(sm + mlp::W1X, packed + K::W1X, 8192);
  copy_g2s(sm + mlp::W2, packed + K::W2, 8192);
  copy_g2s(sm + mlp::WH, packed + K::WH, 2048);
  copy_g2s(sm + mlp::B2, packed + K::B2, 256);
  copy_g2s(sm + mlp::BH, packed + K::BH, 64);
  copy_g2s(sm + mlp::NORM, packed + K::NORM, 128);
  __syncthreads();
  float* nrmw = reinterpret_cast<float*>(sm + mlp::NORM);
  if (t < NFEAT) nrmw[NFEAT + t] = 1.0f / nrmw[NFEAT + t];  // sigma -> 1/sigma
  if (t < HID) {
    // layer-1 bias folded into the MMA: K columns 12 and 13 of W1x hold b1 as
    // a BF16 pair hi + lo (~16 bits), multiplied by feature columns equal to 1
    const float b = __ldg(reinterpret_cast<const float*>(packed + K::B1) + t);
    const float hi = bf16_round(b);
    *reinterpret_cast<__nv_bfloat16*>(sm + mlp::W1X + sw128_off(t, 12)) = __float2bfloat16_rn(hi);
    *reinterpret_cast<__nv_bfloat16*>(sm + mlp::W1X + sw128_off(t, 13)) =
        __float2bfloat16_rn(b - hi);
  }
  TcCtx tc;
  tc_setup(sh, tc, 64);  // (its barrier also publishes the writes above)
  const float* b2 = reinterpret_cast<const float*>(sm + mlp::B2);
  const float* bh = reinterpret_cast<const float*>(sm + mlp::BH);
  const float* nrm = nrmw;
  uint8_t* act = sm + mlp::ACT;
  const uint32_t lb = lane_base(tc.tmem);
  const float sdf = nrm[24];
  const uint32_t ones = bf16x2(1.0f, 1.0f);

  int s = 0;
  for (int64_t tile = first; tile < ntiles; tile += stride) {
    fetch(tile + 2 * stride, s == 0 ? 2 : s - 1);  // the stage read two tiles ago
    cp_async_wait<2>();                             // this thread's copies of `tile`
    const int64_t n = tile * TILE + t;
    const bool on = n < N;
    float fv[Q];
    const float* sv = stg + s * (mlp::SLOTS * TILE) + t;
#pragma unroll
    for (int q = 0; q < Q; ++q) fv[q] = sv[q * TILE];
    const float tau = sv[Q * TILE];
    s = s == 2 ? 0 : s + 1;
    const Moments m = moments9(fv);
    {  // features normalised, as [x_hi (k 0..11), 1, 1, 0, 0 | x_lo (k 16..27), 0 x 4]
      float xh[NFEAT];
#pragma unroll
      for (int q = 0; q < Q; ++q) xh[q] = (fv[q] - nrm[q]) * nrm[NFEAT + q];
      xh[9] = (m.rho - nrm[9]) * nrm[NFEAT + 9];
      xh[10] = (m.ux - nrm[10]) * nrm[NFEAT + 10];
      xh[11] = (m.uy - nrm[11]) * nrm[NFEAT + 11];
      uint32_t hw[8], lw[8];
#pragma unroll
      for (int j = 0; j < NFEAT / 2; ++j) {
        hw[j] = bf16x2(xh[2 * j], xh[2 * j + 1]);
        const float2 lo = __fadd2_rn(make_float2(xh[2 * j], xh[2 * j + 1]),
                                     make_float2(-__uint_as_float(hw[j] << 16),
                                                 -__uint_as_float(hw[j] & 0xFFFF0000u)));
        lw[j] = bf16x2(lo.x, lo.y);
      }
      hw[6] = ones;
      hw[7] = lw[6] = lw[7] = 0u;
      uint8_t* row = act + t * 128;
      const int sw = t & 7;
      *reinterpret_cast<uint4*>(row + ((0 ^ sw) << 4)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(row + ((1 ^ sw) << 4)) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
      *reinterpret_cast<uint4*>(row + ((2 ^ sw) << 4)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      *reinterpret_cast<uint4*>(row + ((3 ^ sw) << 4)) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
    }
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(act), 0, smem_u32(sm + mlp::W1X), 0, 1, 64, false, 2);
        }))
      break;
    {  // g1 = ReLU(W1 x + b1) (the bias came with the MMA)
      float z[32];
      tmem_ld32(lb, z);
      relu_row32(act, t, 0, z, nullptr);
      tmem_ld32(lb + 32, z);
      relu_row32(act, t, 4, z, nullptr);
    }
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(act), 0, smem_u32(sm + mlp::W2), 0, 1, 64, false);
        }))
      break;
    {  // h0 = ReLU(W2 g1 + b2)
      float z[32];
      tmem_ld32(lb, z);
      relu_row32(act, t, 0, z, b2);
      tmem_ld32(lb + 32, z);
      relu_row32(act, t, 4, z, b2 + 32);
    }
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(act), 0, smem_u32(sm + mlp::WH), 0, 1, 16, false);
        }))
      break;
    {  // heads and Eq. 3
      float y[16];
      tmem_ld16(lb, y);
      const float inv = 1.0f / (tau * tau_adj_of(y[0] + bh[0], variant));
      float d[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) d[q] = sdf * (y[1 + q] + bh[1 + q]);
      if (variant & VAR_CONSERVATIVE) conserve9(d);
      const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
      if (on) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
          f_out[q * ps + base + n] = fv[q] - (fv[q] - feq_i(q, m, usq15)) * inv + d[q];
      }
    }
    tc_fence_before();
    __syncthreads();  // the head's accumulator is read before the next tile's MMA
  }
  cp_async_wait<0>();
  tc_teardown(sh, tc, 64);
}

template <class Geo>
static cudaError_t mlp_step(const float* f_in, float* f_out, const Geo& geo, int64_t N, float tau,
                            const float* taus, const uint8_t* packed, bool require_mlp,
                            cudaStream_t st, int per_sm) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  if (N <= 0) return cudaSuccess;
  const uint32_t bytes = mlp::BYTES + 1024;
  cudaError_t e;
  if ((e = set_smem(gnn_mlp_step_kernel<Geo>, bytes)) != cudaSuccess) return e;
  const unsigned grid = grid_for(N, per_sm);
  gnn_mlp_step_kernel<Geo><<<grid, 128, bytes, st>>>(f_in, f_out, geo, tau, taus, packed,
                                                      require_mlp, stw);
  return cudaGetLastError();
}

cudaError_t launch_gnn_mlp_step(const float* f_in, float* f_out, const Shape& s, float tau,
                                const float* taus, const uint8_t* packed, bool require_mlp,
                                cudaStream_t st) {
  return mlp_step(f_in, f_out, make_geo_stack(s), (int64_t)s.nb * s.ny * s.nx, tau, taus, packed,
                  require_mlp, st, LBM_MLP_CTAS);
}

cudaError_t launch_gnn_mlp_step_table(const float* f_in, float* f_out, const LatDesc* lat,
                                      int first, int n, const int* hint, int64_t base,
                                      int64_t count, int64_t ps, const uint8_t* packed,
                                      cudaStream_t st, int per_sm) {
  const GeoTable geo{lat, first, n, base, count, ps, hint};
  return mlp_step(f_in, f_out, geo, count, 0.0f, nullptr, packed, false, st,
                  per_sm >= 2 ? LBM_MLP_CTAS : per_sm);
}

}  // namespace lbmgnn
