// GNN-enhanced collision, reverse direction and training (paper Sec. 2.4,
// Eq. 3, Eq. 4): the Eq. 3 + MSE loss kernel, the head backward, the two
// kernels of each message-passing round's backward, the encoder backward,
// the deterministic gradient reduction and the AdamW update.
//
// Per-round recompute: the forward saves h, the aggregated messages a and
// the per-node edge terms A = W_a h, B = W_b h (FP16); the backward recomputes
// the node pre-activation W_n [h; a] + b_n with the same MMA and every edge
// pre-activation z_ik = A_i + B_j + c_k elementwise, so the 8 per-node edge
// activations are never stored.
//
// The edge terms need gradients scattered to neighbours (dB_j collects from
// every i with j = i + e_k).  They are gathered instead ("pull" form): node j
// reads da_i and A_i of its 8 neighbours i = j - e_k, so no atomics are used
// and the result is deterministic.  This needs da of every node first, hence
// two kernels per round.
//
// Weight gradients are contractions over nodes.  Each CTA accumulates them
// on the tensor cores over all tiles it owns (operands written transposed,
// nodes along K, into 128-byte swizzled shared memory; FP32 accumulators in
// tensor memory) and writes one partial row; a final kernel sums the rows in
// a fixed order.  Bias gradients (column sums) ride along as an extra MMA
// column of ones.
#include "gnn.cuh"
#include "gnn_launch.h"

namespace lbmgnn {

// ---- transposed operand writes ---------------------------------------------------
// Writes NV values v[c] to rows row0 + c, column `node` (0..127) of a K = 128
// operand made of two SW128 blocks of R rows each (nodes 0..63, 64..127).
template <int NV>
__device__ __forceinline__ void st_col(uint8_t* op, int R, int row0, int node, const float* v) {
  uint8_t* blk = op + (node >> 6) * (R * 128);
  const int k = node & 63;
#pragma unroll
  for (int c = 0; c < NV; ++c)
    *reinterpret_cast<__nv_bfloat16*>(blk + sw128_off(row0 + c, k)) = __float2bfloat16_rn(v[c]);
}

#ifndef LBM_BWD_PF
#define LBM_BWD_PF 1  // L2 prefetch of the next tile's per-node inputs
#endif

// L2 prefetch (a hint: no registers, no completion to wait for) of nodes
// [m0, m0 + 128) of plane `plane` of a per-node tensor: chunked planes of 16
// bytes per node (esz 16, plane stride N nodes) or FP32 planes (esz 4, plane
// stride `ps` nodes).  The range is shrunk to 16-byte boundaries inside the
// tensor's own bytes.
__device__ __forceinline__ void l2_prefetch_nodes(const void* base, int plane, int64_t ps,
                                                  int esz, int64_t m0, int64_t N) {
  if (m0 >= N) return;
  const int64_t cnt = N - m0 < 128 ? N - m0 : 128;
  const uintptr_t a = reinterpret_cast<uintptr_t>(base) + (uintptr_t)((plane * ps + m0) * esz);
  const uintptr_t lo = a & ~uintptr_t(15), hi = (a + (uintptr_t)(cnt * esz)) & ~uintptr_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo))
                 : "memory");
}

__device__ __forceinline__ void zero_smem(uint8_t* p, uint32_t bytes) {
  uint4* q = reinterpret_cast<uint4*>(p);
  for (uint32_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) q[i] = make_uint4(0, 0, 0, 0);
}

// Sets row `row` of a two-block K = 128 operand (R rows per block) to 1.
__device__ __forceinline__ void ones_row(uint8_t* op, int R, int row) {
  for (int n = threadIdx.x; n < 128; n += blockDim.x) {
    uint8_t* blk = op + (n >> 6) * (R * 128);
    *reinterpret_cast<__nv_bfloat16*>(blk + sw128_off(row, n & 63)) = __float2bfloat16_rn(1.0f);
  }
}

// Sum over the 32 lanes of v[0..31] (lane-private values): afterwards lane l
// holds the sum of v[l] over the warp (31 shuffles; halves the vector per step).
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = lane & w;  // keep the upper half of the current range
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float send = upper ? v[i] : v[i + w];
      const float keep = upper ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

__device__ __forceinline__ void ld_f32x32(const float* p, float* v) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 t = __ldg(q + i);
    v[4 * i] = t.x;
    v[4 * i + 1] = t.y;
    v[4 * i + 2] = t.z;
    v[4 * i + 3] = t.w;
  }
}
__device__ __forceinline__ void st_f32x32(float* p, const float* v) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int i = 0; i < 8; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// ---------------------------------------------------------------------------
// Eq. 3 followed by Eq. 4: per node f_pred = f - (f - f_eq)/(tau tau_adj) +
// s_df y_1..9, squared error against the target, and dL/dy.  The loss is the
// mean over nodes x 9 of the whole stack.  One thread per node.
// FORCED (the channel): a force (gx, 0) per unit volume (gxs[b] per lattice
// when set) enters by Guo's scheme, u = (sum f e + F/2)/rho and the source
// (1 - 1/(2t)) S with S_i = w_i [3 (e_ix - u_x) + 9 (e_i.u) e_ix] gx at the
// network's time t; d f_pred / d t = ((f - f_eq) + S/2) / t^2.
template <bool FORCED>
__global__ void __launch_bounds__(256) gnn_collide_loss_kernel(
    const float* __restrict__ f_pre, const float* __restrict__ y, const float* __restrict__ tgt,
    Shape s, float tau, const float* __restrict__ taus, float gx0,
    const float* __restrict__ gxs, const uint8_t* __restrict__ packed,
    double* __restrict__ lossp, float* __restrict__ dy, float* __restrict__ f_pred,
    const float* __restrict__ lw, unsigned* stw) {
  if (!blob_ok(packed, stw)) {  // no loss from an invalid image: NaN
    if (threadIdx.x == 0) lossp[blockIdx.x] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = n < N;
  const int64_t nn = on ? n : N - 1;
  const float sdf = reinterpret_cast<const float*>(packed + K::NORM)[24];
  const int variant = variant_of(reinterpret_cast<const float*>(packed + K::NORM));
  float fv[Q], yv[NOUT];
#pragma unroll
  for (int q = 0; q < Q; ++q) fv[q] = __ldg(f_pre + q * s.ps + nn);
#pragma unroll
  for (int o = 0; o < NOUT; ++o) yv[o] = __ldg(y + o * N + nn);
  const int64_t b = nn / ((int64_t)s.nx * s.ny);
  const float t = taus ? __ldg(taus + b) : tau;
  const float wb = lw ? __ldg(lw + b) : 1.0f;  // per-instance loss weight (1: Eq. 4)
  Moments m = moments9(fv);
  float gx = 0.0f;
  if constexpr (FORCED) {
    gx = gxs ? __ldg(gxs + b) : gx0;
    m.ux += 0.5f * gx / m.rho;
  }
  const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
  const bool fixed_tau = variant & VAR_FIXED_TAU;
  const float sg = sigmoid_acc(yv[0]);
  const float teff = t * tau_adj_of(yv[0], variant);
  const float inv = 1.0f / teff;
  const float scale = 2.0f * wb / (9.0f * (float)N);
  double lp = 0.0;
  float dta = 0.0f, dyv[NOUT], d[Q], g[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) d[q] = sdf * yv[1 + q];
  if (variant & VAR_CONSERVATIVE) conserve9(d);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float fe = feq_i(q, m, usq15);
    float fp = fv[q] - (fv[q] - fe) * inv + d[q];
    float dt = fv[q] - fe;  // t^2 d f_pred / d t
    if constexpr (FORCED) {
      const float eu = float(ex(q)) * m.ux + float(ey(q)) * m.uy;
      const float src = wq(q) * (3.0f * (float(ex(q)) - m.ux) + 9.0f * eu * float(ex(q))) * gx;
      fp += (1.0f - 0.5f * inv) * src;
      dt += 0.5f * src;
    }
    const float r = fp - __ldg(tgt + q * s.ps + nn);
    lp += (double)wb * (double)r * (double)r;
    g[q] = scale * r;  // dL/df*
    dta += g[q] * dt;
    if (on && f_pred) f_pred[q * s.ps + n] = fp;
  }
  // Delta f = s_df P y_1..9 with P the (symmetric) projection, or P = I
  if (variant & VAR_CONSERVATIVE) conserve9(g);
#pragma unroll
  for (int q = 0; q < Q; ++q) dyv[1 + q] = sdf * g[q];
  dyv[0] = fixed_tau ? 0.0f : dta * t * inv * inv * sg * (1.0f - sg);
  if (on && dy) {
#pragma unroll
    for (int o = 0; o < NOUT; ++o) dy[o * N + n] = dyv[o];
  }
  // block reduction of the squared error
  if (!on) lp = 0.0;
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lp += __shfl_xor_sync(0xffffffffu, lp, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < 8; ++i) acc += red[i];
    lossp[blockIdx.x] = acc;
  }
}

// Reverse mode of Eq. 3 for the K-step rollout loss, one thread per node:
// g = g_in + scale (f_post - target) is dL/df* of this step (g_in: the
// later steps' share, pulled back through streaming; NULL for the last
// step); writes dL/dy as the loss kernel does and the part of dL/df_pre that
// passes through the explicit f and f^eq(rho(f), u(f)):
//   dfd_j = g_j (1 - 1/t) + (1/t) [sum_i g_i f^eq_i / rho
//           + V . (e_j - u)],  V = sum_i g_i w_i (3 e_i + 9 (e_i.u) e_i - 3 u).
__global__ void __launch_bounds__(256) gnn_collide_adjoint_kernel(
    const float* __restrict__ f_pre, const float* __restrict__ y,
    const float* __restrict__ f_post, const float* __restrict__ tgt,
    const float* __restrict__ g_in, Shape s, float tau, const float* __restrict__ taus,
    const uint8_t* __restrict__ packed, float scale, float* __restrict__ dy,
    float* __restrict__ dfd, unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float* nrm = reinterpret_cast<const float*>(packed + K::NORM);
  const float sdf = nrm[24];
  const int variant = variant_of(nrm);
  float fv[Q], g[Q], gp[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    fv[q] = __ldg(f_pre + q * s.ps + n);
    const float r = __ldg(f_post + q * s.ps + n) - __ldg(tgt + q * s.ps + n);
    g[q] = (g_in ? __ldg(g_in + q * s.ps + n) : 0.0f) + scale * r;
    gp[q] = g[q];
  }
  const float y0 = __ldg(y + n);
  const int64_t b = n / ((int64_t)s.nx * s.ny);
  const float t0 = taus ? __ldg(taus + b) : tau;
  const float sg = sigmoid_acc(y0);
  const float t = t0 * tau_adj_of(y0, variant);
  const float inv = 1.0f / t;
  const Moments m = moments9(fv);
  const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
  float dta = 0.0f, a = 0.0f, vx = 0.0f, vy = 0.0f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float fe = feq_i(q, m, usq15);
    dta += g[q] * (fv[q] - fe);
    a += g[q] * fe;
    const float eu = float(ex(q)) * m.ux + float(ey(q)) * m.uy;
    const float gw = g[q] * wq(q);
    vx += gw * (3.0f * float(ex(q)) + 9.0f * eu * float(ex(q)) - 3.0f * m.ux);
    vy += gw * (3.0f * float(ey(q)) + 9.0f * eu * float(ey(q)) - 3.0f * m.uy);
  }
  a /= m.rho;
  if (variant & VAR_CONSERVATIVE) conserve9(gp);
#pragma unroll
  for (int q = 0; q < Q; ++q) dy[(int64_t)(1 + q) * N + n] = sdf * gp[q];
  dy[n] = (variant & VAR_FIXED_TAU) ? 0.0f : dta * t0 * inv * inv * sg * (1.0f - sg);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    dfd[q * s.ps + n] = g[q] * (1.0f - inv) +
                        inv * (a + vx * (float(ex(q)) - m.ux) + vy * (float(ey(q)) - m.uy));
}

// Adjoint of periodic pull streaming applied to a + b: out_q(x) =
// (a + b)_q(x + e_q) within each lattice (the transpose of
// f_q(x) = f*_q(x - e_q)).
__global__ void __launch_bounds__(256) stream_adjoint_sum_kernel(
    const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out, Shape s,
    unsigned* stw) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const NodeXY p = node_xy(n, s);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int64_t j = checked(node_at(p, ex(q), ey(q), s), 0, N, stw);
    out[q * s.ps + n] = __ldg(a + q * s.ps + j) + __ldg(b + q * s.ps + j);
  }
}

// Sum of the per-block squared errors, divided by 9 N (deterministic order).
__global__ void loss_finish_kernel(const double* __restrict__ lossp, int nblk, double count,
                                   double* __restrict__ loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += lossp[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / count;
}

// ---------------------------------------------------------------------------
// Head backward: dh2 = dy W_h (CUDA cores), dW_h and db_h accumulated on the
// tensor cores: D[o][i] += sum_n dy[n][o] [h2 | 1][n][i].
namespace hb {
constexpr uint32_t XT = 0, YT = 32768, WHF = 53248, DYS = 55808, SH = 60928, BYTES = 61056;
}

__global__ void __launch_bounds__(256, 2) gnn_head_bwd_kernel(
    const float* __restrict__ dy, const __nv_bfloat16* __restrict__ h2, float* __restrict__ dh,
    float* __restrict__ G, Shape s, const uint8_t* __restrict__ packed, unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_align1024(smem_raw);
  TcShared* sh = reinterpret_cast<TcShared*>(sm + hb::SH);
  zero_smem(sm, hb::WHF);
  copy_g2s(sm + hb::WHF, packed + K::WHF, 2560);
  __syncthreads();
  ones_row(sm + hb::YT, 80, 64);
  TcCtx tc;
  tc_setup(sh, tc);
  const float* whf = reinterpret_cast<const float*>(sm + hb::WHF);
  float* dys = reinterpret_cast<float*>(sm + hb::DYS);
  uint8_t* XT = sm + hb::XT;
  uint8_t* YT = sm + hb::YT;
  const int node = threadIdx.x & 127, half = threadIdx.x >> 7, f0 = half * 32;
  const uint32_t lb = lane_base(tc.tmem);
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t ntiles = (N + TILE - 1) / TILE;
  bool first = true, ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t n = tile * TILE + node;
    const bool on = n < N;
    const int64_t nn = on ? n : N - 1;
    if (LBM_BWD_PF && threadIdx.x < NOUT + 8) {  // next tile: dy (10 FP32 planes), h2 (8 planes)
      const int64_t m0 = (tile + gridDim.x) * TILE;
      if (threadIdx.x < NOUT) l2_prefetch_nodes(dy, threadIdx.x, N, 4, m0, N);
      else l2_prefetch_nodes(h2, threadIdx.x - NOUT, N, 16, m0, N);
    }
    if (half == 0) {
      float d[NOUT];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) {
        d[o] = on ? __ldg(dy + o * N + nn) : 0.0f;
        dys[node * NOUT + o] = d[o];
      }
      st_col<NOUT>(XT, 128, 0, node, d);
    }
    float hv[32];
    ld_pb32(h2, N, nn, f0, hv);
    st_col<32>(YT, 80, f0, node, hv);
    __syncthreads();
    float dv[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) dv[c] = 0.0f;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
      const float g = dys[node * NOUT + o];
#pragma unroll
      for (int c = 0; c < 32; ++c) dv[c] = fmaf(g, whf[o * HID + f0 + c], dv[c]);
    }
    if (on) st_pf32(dh, N, n, f0, dv);
    const bool acc = !first;
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(XT), 16384, smem_u32(YT), 10240, 2, 80, acc);
        })) {
      ok = false;
      break;
    }
    first = false;
  }
  if (ok && (threadIdx.x >> 5) == 0) {
    float v[32], w[32], u[16];
    tmem_ld32(lb, v);
    tmem_ld32(lb + 32, w);
    tmem_ld16(lb + 64, u);
    const int o = threadIdx.x & 31;
    if (o < NOUT) {
      float* g = G + (int64_t)blockIdx.x * P::TRAINABLE;
      for (int i = 0; i < 32; ++i) {
        g[P::HEAD_W + o * HID + i] = v[i];
        g[P::HEAD_W + o * HID + 32 + i] = w[i];
      }
      g[P::HEAD_B + o] = u[0];
    }
  }
  tc_teardown(sh, tc);
}

// ---------------------------------------------------------------------------
// Round backward, part 1 (per node): recompute z_n = W_n [h; a] + b_n,
// dz_n = dh_out * GELU'(z_n), d[h; a] = dz_n W_n; accumulate dW_n (tensor
// cores, [h; a]^T dz_n) and db_n (sum of dz_n, in registers by a butterfly
// reduction over each warp's nodes).  Outputs dh_part = dh_out + d[h; a]_h
// and da = d[h; a]_a (FP32).
namespace rb1 {
// U holds [h; a] node-major (A of the z_n recompute) until that MMA is done,
// then dz node-major (16 KB) and dz transposed (16 KB, 64 rows per K block).
constexpr uint32_t U = 0, HAT = 32768, WN = 65536, WNT = 81920, BN = 98304, DBR = 98560,
                   SH = 99584, BYTES = 99712;
}
#ifndef LBM_RB1_CTAS
#define LBM_RB1_CTAS 2  // resident CTAs per SM
#endif

__global__ void __launch_bounds__(256, LBM_RB1_CTAS) gnn_round_bwd1_kernel(
    const __nv_bfloat16* __restrict__ h_in, const __nv_bfloat16* __restrict__ a_in,
    const float* __restrict__ dh_out, float* __restrict__ dh_part, float* __restrict__ da,
    int round, float* __restrict__ G, Shape s, const uint8_t* __restrict__ packed, unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_align1024(smem_raw);
  TcShared* sh = reinterpret_cast<TcShared*>(sm + rb1::SH);
  const uint8_t* kr = packed + K::round_base(round);
  const bool mlp_only = variant_of(reinterpret_cast<const float*>(packed + K::NORM)) & VAR_MLP_ONLY;
  copy_g2s(sm + rb1::WN, kr + K::WN, 16384);
  copy_g2s(sm + rb1::WNT, kr + K::WNT, 16384);
  copy_g2s(sm + rb1::BN, kr + K::BN, 256);
  __syncthreads();
  TcCtx tc;
  tc_setup(sh, tc);
  const float* bn = reinterpret_cast<const float*>(sm + rb1::BN);
  uint8_t* HA = sm + rb1::U;
  uint8_t* DZ = sm + rb1::U;            // after the z_n MMA
  uint8_t* DZT = sm + rb1::U + 16384;   // after the z_n MMA
  uint8_t* HAT = sm + rb1::HAT;
  const int node = threadIdx.x & 127, half = threadIdx.x >> 7, f0 = half * 32;
  const uint32_t lb = lane_base(tc.tmem);
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t ntiles = (N + TILE - 1) / TILE;
  float dbacc = 0.0f;  // lane l: running sum of dz[f0 + l] over this warp's nodes
  bool first = true, ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t n = tile * TILE + node;
    const bool on = n < N;
    const int64_t nn = on ? n : N - 1;
    if (LBM_BWD_PF && threadIdx.x < 32) {  // next tile: h, a (8 planes each), dh_out (16)
      const int64_t m0 = (tile + gridDim.x) * TILE;
      const int t = threadIdx.x;
      if (t < 8) l2_prefetch_nodes(h_in, t, N, 16, m0, N);
      else if (t < 16) l2_prefetch_nodes(a_in, t - 8, N, 16, m0, N);
      else l2_prefetch_nodes(dh_out, t - 16, N, 16, m0, N);
    }
    {
      float v[32];
      ld_pb32(h_in, N, nn, f0, v);
      st_row32(HA, node, f0, v);
      st_col<32>(HAT, 128, f0, node, v);
      ld_pb32(a_in, N, nn, f0, v);
      st_row32(HA + 16384, node, f0, v);
      st_col<32>(HAT, 128, HID + f0, node, v);
    }
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(HA), 16384, smem_u32(sm + rb1::WN), 8192, 2, 64, false);
        })) {
      ok = false;
      break;
    }
    {
      float dz[32], dho[32];
      tmem_ld32(lb + f0, dz);
      ld_pf32(dh_out, N, nn, f0, dho);
      act_and_grad(dz, bn + f0, 32, false, nullptr, dz);  // GELU'(z_n), packed pairs
#pragma unroll
      for (int c = 0; c < 32; ++c) dz[c] = (on && !mlp_only) ? dho[c] * dz[c] : 0.0f;
      // the z_n MMA has read [h; a]: its space now takes dz
      st_row32(DZ, node, f0, dz);
      st_col<32>(DZT, 64, f0, node, dz);
      dbacc += warp_transpose_sum(dz);
    }
    const bool acc = !first;
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(DZ), 0, smem_u32(sm + rb1::WNT), 0, 1, 128, false);
          umma_128xN(tc.tmem + 128, smem_u32(HAT), 16384, smem_u32(DZT), 8192, 2, 64, acc);
        })) {
      ok = false;
      break;
    }
    first = false;
    {
      float d[32], dho[32];
      tmem_ld32(lb + f0, d);           // warp-collective: every lane takes part
      ld_pf32(dh_out, N, nn, f0, dho);  // again (an L2 hit): fewer values live across the MMA
#pragma unroll
      for (int c = 0; c < 32; ++c) d[c] += dho[c];
      if (on) st_pf32(dh_part, N, n, f0, d);
      tmem_ld32(lb + HID + f0, d);
      if (on) st_pf32(da, N, n, f0, d);
    }
    tc_fence_before();
    __syncthreads();
  }
  if (ok) {
    // D_wn[i][o] at columns 128..191 (row i = input feature of [h; a])
    const int row = 32 * ((threadIdx.x >> 5) & 3) + (threadIdx.x & 31);
    float* g = G + (int64_t)blockIdx.x * P::TRAINABLE + P::ROUND0 + round * P::ROUND_SIZE;
    float v[32];
    tmem_ld32(lb + 128 + f0, v);
    for (int c = 0; c < 32; ++c) g[P::NODE_W + (f0 + c) * 128 + row] = v[c];
    // db_n: the 4 warps of a feature half hold disjoint node sets; fixed order
    float* dbr = reinterpret_cast<float*>(sm + rb1::DBR);  // [8 warps][32]
    dbr[(threadIdx.x >> 5) * 32 + (threadIdx.x & 31)] = dbacc;
    __syncthreads();
    if (threadIdx.x < HID) {
      const int hh = threadIdx.x >> 5, l = threadIdx.x & 31;
      float t = 0.0f;
      for (int q = 0; q < 4; ++q) t += dbr[(hh * 4 + q) * 32 + l];
      g[P::NODE_B + threadIdx.x] = t;
    }
  }
  tc_teardown(sh, tc);
}

// ---------------------------------------------------------------------------
// Round backward, part 2 (pull form): for node j
//   dA_j = sum_k da_j * GELU'(A_j + B_{j+e_k} + c_k)
//   dB_j = sum_k da_i * GELU'(A_i + B_j + c_k),  i = j - e_k
//   dc_x,j / dc_y,j = the e_kx / e_ky weighted sums of the dA_j terms.
// dh_in = dh_part + [dA | dB] [W_a; W_b]; accumulates [dW_a; dW_b], db_e
// (= sum dA) on the tensor cores and the W_c columns (sum dc_x, sum dc_y) in
// registers (butterfly reduction over the warp's nodes).
namespace rb2 {
constexpr uint32_t DAB = 0, DABT = 32768, HT = 65536, WABT = 86016, CK = 102400, CKH = 104448,
                   DCR = 105472, SH = 107520, BYTES = 107648;
}
#ifndef LBM_RB2_CTAS
#define LBM_RB2_CTAS 1  // resident CTAs per SM (2 fit; measured slower)
#endif
#ifndef LBM_RB2_GROUP
#define LBM_RB2_GROUP 4  // neighbours whose loads are in flight together
#endif

// WALLS (the channel's graph): an edge whose far node lies beyond a wall
// (row outside [0, ny)) was left out of the forward's sum and passes no
// gradient; its neighbour address wraps to a row inside, so loads stay in
// range.
template <bool WALLS>
__global__ void __launch_bounds__(256, LBM_RB2_CTAS) gnn_round_bwd2_kernel(
    const __half* __restrict__ ab, const float* __restrict__ da,
    const float* __restrict__ dh_part, const __nv_bfloat16* __restrict__ h_in,
    float* __restrict__ dh_in, int round, float* __restrict__ G, Shape s,
    const uint8_t* __restrict__ packed, unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_align1024(smem_raw);
  TcShared* sh = reinterpret_cast<TcShared*>(sm + rb2::SH);
  const uint8_t* kr = packed + K::round_base(round);
  zero_smem(sm + rb2::HT, rb2::WABT - rb2::HT);
  copy_g2s(sm + rb2::WABT, kr + K::WABT, 16384);
  copy_g2s(sm + rb2::CK, kr + K::CK, 2048);
  __syncthreads();
  ones_row(sm + rb2::HT, 80, 64);
  {  // c_k as FP16 pairs
    const float* ckf = reinterpret_cast<const float*>(sm + rb2::CK);
    __half2* ckw = reinterpret_cast<__half2*>(sm + rb2::CKH);
    for (int i = threadIdx.x; i < 8 * HID / 2; i += blockDim.x)
      ckw[i] = __floats2half2_rn(ckf[2 * i], ckf[2 * i + 1]);
  }
  TcCtx tc;
  tc_setup(sh, tc);
  const __half2* ckh = reinterpret_cast<const __half2*>(sm + rb2::CKH);
  uint8_t* DAB = sm + rb2::DAB;
  uint8_t* DABT = sm + rb2::DABT;
  uint8_t* HT = sm + rb2::HT;
  // per chunk: lane l's running sum of value l of [dc_x | dc_y] over this warp's nodes
  float dcacc0 = 0.0f, dcacc1 = 0.0f;
  const int node = threadIdx.x & 127, half = threadIdx.x >> 7, f0 = half * 32;
  const uint32_t lb = lane_base(tc.tmem);
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t ntiles = (N + TILE - 1) / TILE;
  bool first = true, ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t n = tile * TILE + node;
    const bool on = n < N;
    const int64_t nn = on ? n : N - 1;
    const NodeXY p = node_xy(nn, s);
#pragma unroll 1
    for (int sc = 0; sc < 2; ++sc) {  // two chunks of 16 features
      const int c0 = f0 + 16 * sc;
      const int ch = c0 >> 3;
      // 2 GELU'(z) is evaluated in packed FP16 pairs (z = A + B + c_k is O(1)).
      // dA_j = da_j * sum_k GELU'(z_jk) factors: the sums over k (and their
      // e_kx / e_ky weighted forms) are taken in FP16 and multiplied by da_j
      // once.  dB_j needs the neighbours' da, so its terms are accumulated in
      // FP32 (gradients would underflow FP16).  The two halves run one after
      // the other to keep few values live.
      {  // dA_j and dc_j over the neighbours j + e_k
        uint32_t aj[8];
        {
          const uint4 a0 = __ldg(chunk8(ab, N, nn, c0)), a1 = __ldg(chunk8(ab, N, nn, c0 + 8));
          aj[0] = a0.x; aj[1] = a0.y; aj[2] = a0.z; aj[3] = a0.w;
          aj[4] = a1.x; aj[5] = a1.y; aj[6] = a1.z; aj[7] = a1.w;
        }
        __half2 S[8], Sx[8], Sy[8];  // sums over k of 2 GELU'(z_jk), e_kx and e_ky weighted
#pragma unroll
        for (int c = 0; c < 8; ++c) S[c] = Sx[c] = Sy[c] = __float2half2_rn(0.0f);
#pragma unroll
        for (int g = 0; g < 8; g += LBM_RB2_GROUP) {  // directions k = g+1 .. g+LBM_RB2_GROUP
          uint4 bn[LBM_RB2_GROUP][2];
#pragma unroll
          for (int kk = 0; kk < LBM_RB2_GROUP; ++kk) {
            const int k = g + kk + 1;
            const int64_t j = checked(node_at(p, ex(k), ey(k), s), 0, N, stw);
            bn[kk][0] = __ldg(chunk8(ab, N, j, HID + c0));
            bn[kk][1] = __ldg(chunk8(ab, N, j, HID + c0 + 8));
          }
#pragma unroll
          for (int kk = 0; kk < LBM_RB2_GROUP; ++kk) {
            const int k = g + kk + 1;
            const __half2* c_k = ckh + (k - 1) * (HID / 2) + c0 / 2;
            const uint32_t* bw = reinterpret_cast<const uint32_t*>(bn[kk]);
            const bool keep = !WALLS || (unsigned)(p.y + ey(k)) < (unsigned)s.ny;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const __half2 z = __hadd2(__hadd2(u32_as_h2(aj[c]), c_k[c]), u32_as_h2(bw[c]));
              const __half2 gp = keep ? gelu_grad2_h2(z) : __float2half2_rn(0.0f);
              S[c] = __hadd2(S[c], gp);
              if (ex(k) > 0) Sx[c] = __hadd2(Sx[c], gp);
              if (ex(k) < 0) Sx[c] = __hsub2(Sx[c], gp);
              if (ey(k) > 0) Sy[c] = __hadd2(Sy[c], gp);
              if (ey(k) < 0) Sy[c] = __hsub2(Sy[c], gp);
            }
          }
        }
        float gA[16], v[32];  // v = [dc_x | dc_y] of this node
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 t = __ldg(chunk4(da, N, nn, c0 + 4 * i));
          const float dd[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {  // the factor 1/2 of 2 GELU' is applied here
            const int c = 4 * i + q;
            const float d = on ? 0.5f * dd[q] : 0.0f;
            const float2 sv = __half22float2(S[c >> 1]), sx = __half22float2(Sx[c >> 1]);
            const float2 sy = __half22float2(Sy[c >> 1]);
            gA[c] = d * ((c & 1) ? sv.y : sv.x);
            v[c] = d * ((c & 1) ? sx.y : sx.x);
            v[16 + c] = d * ((c & 1) ? sy.y : sy.x);
          }
        }
        // node-major dA (A operand of the dh MMA) and its transpose
        *reinterpret_cast<uint4*>(DAB + node * 128 + ((ch ^ (node & 7)) << 4)) = pack_bf16x8(gA);
        *reinterpret_cast<uint4*>(DAB + node * 128 + (((ch + 1) ^ (node & 7)) << 4)) =
            pack_bf16x8(gA + 8);
        st_col<16>(DABT, 128, c0, node, gA);
        // dc sums over this warp's 32 nodes: lane l gets value l of [dc_x | dc_y]
        const float t = warp_transpose_sum(v);
        if (sc == 0)
          dcacc0 += t;
        else
          dcacc1 += t;
      }
      {  // dB_j over the neighbours i = j - e_k
        uint32_t bj[8];
        {
          const uint4 b0 = __ldg(chunk8(ab, N, nn, HID + c0));
          const uint4 b1 = __ldg(chunk8(ab, N, nn, HID + c0 + 8));
          bj[0] = b0.x; bj[1] = b0.y; bj[2] = b0.z; bj[3] = b0.w;
          bj[4] = b1.x; bj[5] = b1.y; bj[6] = b1.z; bj[7] = b1.w;
        }
        float gB[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) gB[c] = 0.0f;
#pragma unroll
        for (int g = 0; g < 8; g += LBM_RB2_GROUP) {
          uint4 ai[LBM_RB2_GROUP][2];
          float4 di[LBM_RB2_GROUP][4];
#pragma unroll
          for (int kk = 0; kk < LBM_RB2_GROUP; ++kk) {
            const int k = g + kk + 1;
            const int64_t i = checked(node_at(p, -ex(k), -ey(k), s), 0, N, stw);
            ai[kk][0] = __ldg(chunk8(ab, N, i, c0));
            ai[kk][1] = __ldg(chunk8(ab, N, i, c0 + 8));
#pragma unroll
            for (int t4 = 0; t4 < 4; ++t4) di[kk][t4] = __ldg(chunk4(da, N, i, c0 + 4 * t4));
          }
#pragma unroll
          for (int kk = 0; kk < LBM_RB2_GROUP; ++kk) {
            const int k = g + kk + 1;
            const __half2* c_k = ckh + (k - 1) * (HID / 2) + c0 / 2;
            const uint32_t* aw = reinterpret_cast<const uint32_t*>(ai[kk]);
            const float* dv = reinterpret_cast<const float*>(di[kk]);
            // the edge (i, k) into this node exists if i lies inside
            const bool keep = !WALLS || (unsigned)(p.y - ey(k)) < (unsigned)s.ny;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const __half2 z = __hadd2(__hadd2(u32_as_h2(aw[c]), c_k[c]), u32_as_h2(bj[c]));
              const float2 gp = keep ? __half22float2(gelu_grad2_h2(z)) : make_float2(0.0f, 0.0f);
              gB[2 * c] = fmaf(dv[2 * c], gp.x, gB[2 * c]);
              gB[2 * c + 1] = fmaf(dv[2 * c + 1], gp.y, gB[2 * c + 1]);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) gB[c] = on ? 0.5f * gB[c] : 0.0f;
        uint8_t* b1 = DAB + 16384;
        *reinterpret_cast<uint4*>(b1 + node * 128 + ((ch ^ (node & 7)) << 4)) = pack_bf16x8(gB);
        *reinterpret_cast<uint4*>(b1 + node * 128 + (((ch + 1) ^ (node & 7)) << 4)) =
            pack_bf16x8(gB + 8);
        st_col<16>(DABT, 128, HID + c0, node, gB);
      }
    }
    {
      float h[32];
      ld_pb32(h_in, N, nn, f0, h);
      st_col<32>(HT, 80, f0, node, h);
    }
    const bool acc = !first;
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(DAB), 16384, smem_u32(sm + rb2::WABT), 8192, 2, 64, false);
          umma_128xN(tc.tmem + 64, smem_u32(DABT), 16384, smem_u32(HT), 10240, 2, 80, acc);
        })) {
      ok = false;
      break;
    }
    first = false;
    float d[32], dp[32];
    tmem_ld32(lb + f0, d);
    if (on) {
      ld_pf32(dh_part, N, n, f0, dp);
#pragma unroll
      for (int c = 0; c < 32; ++c) d[c] += dp[c];
      st_pf32(dh_in, N, n, f0, d);
    }
    tc_fence_before();
    __syncthreads();
  }
  if (ok) {
    const int row = 32 * ((threadIdx.x >> 5) & 3) + (threadIdx.x & 31);  // o' (a rows, then b rows)
    float* g = G + (int64_t)blockIdx.x * P::TRAINABLE + P::ROUND0 + round * P::ROUND_SIZE;
    const int o = row & 63;
    const int col_off = row < HID ? 0 : HID;
    float v[32];
    tmem_ld32(lb + 64 + f0, v);
    for (int c = 0; c < 32; ++c) g[P::EDGE_W + o * 130 + col_off + f0 + c] = v[c];
    if (half == 0) {
      float u[16];
      tmem_ld16(lb + 128, u);  // column sum of [dA | dB]
      if (row < HID) g[P::EDGE_B + o] = u[0];
    }
    // W_c columns: the 4 warps of a feature half hold disjoint node sets;
    // summed in fixed order.
    float* dcr = reinterpret_cast<float*>(sm + rb2::DCR);  // [8 warps][2 chunks][32]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    dcr[(w * 2 + 0) * 32 + lane] = dcacc0;
    dcr[(w * 2 + 1) * 32 + lane] = dcacc1;
    __syncthreads();
    if (threadIdx.x < 128) {
      const int hh = threadIdx.x >> 6, sc = (threadIdx.x >> 5) & 1, l = threadIdx.x & 31;
      float t = 0.0f;
      for (int q = 0; q < 4; ++q) t += dcr[((hh * 4 + q) * 2 + sc) * 32 + l];
      const int of = 32 * hh + 16 * sc + (l & 15);
      g[P::EDGE_W + of * 130 + 128 + (l >> 4)] = t;
    }
  }
  tc_teardown(sh, tc);
}

// ---------------------------------------------------------------------------
// Encoder backward: recompute x_hat, z1, g1, z2; dz2 = dh0 * GELU'(z2),
// dg1 = dz2 W2, dz1 = dg1 * GELU'(z1); accumulate
// D[o'][i'] = sum_n [dz2 | dz1][n][o'] [g1 | x_hat | 1][n][i'], which holds
// dW2, db2 (rows 0..63) and dW1, db1 (rows 64..127).  Optionally the input
// gradient dL/df_pre through x_hat (f_i, rho and u = j / rho).
namespace eb {
// U holds, one after the other within a tile, g1 node-major (A of the z2
// MMA), dz2 node-major (A of the dg1 MMA) and the df partial sums.
constexpr uint32_t U = 0, XT = 16384, YT = 49152, W2 = 69632, W2T = 77824, W1F = 86016,
                   B1 = 89088, B2 = 89344, NORM = 89600, SH = 89728, BYTES = 89856;
}
#ifndef LBM_EB_CTAS
#define LBM_EB_CTAS 2  // resident CTAs per SM
#endif

// The channel's velocity feature is (sum f e + F/2)/rho with F = (fx, 0)
// (fxs[b] per lattice when set; fx = 0 and fxs NULL elsewhere); its
// derivative w.r.t. f_i is (e_i - u)/rho with that u.
__global__ void __launch_bounds__(256, LBM_EB_CTAS) gnn_encode_bwd_kernel(
    const float* __restrict__ f_pre, const float* __restrict__ dh0, float* __restrict__ df,
    float* __restrict__ G, Shape s, float fx, const float* __restrict__ fxs,
    const uint8_t* __restrict__ packed, unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_align1024(smem_raw);
  TcShared* sh = reinterpret_cast<TcShared*>(sm + eb::SH);
  zero_smem(sm + eb::YT, eb::W2 - eb::YT);
  copy_g2s(sm + eb::W2, packed + K::W2, 8192);
  copy_g2s(sm + eb::W2T, packed + K::W2T, 8192);
  copy_g2s(sm + eb::W1F, packed + K::W1F, 3712);
  __syncthreads();
  ones_row(sm + eb::YT, 80, 76);
  // 1 / sigma (the forward encoder normalises by this product too), beside
  // the tensor-core context
  float* isg = reinterpret_cast<float*>(sm + eb::SH + 64);
  if (threadIdx.x < NFEAT)
    isg[threadIdx.x] = 1.0f / reinterpret_cast<const float*>(sm + eb::NORM)[NFEAT + threadIdx.x];
  TcCtx tc;
  tc_setup(sh, tc);
  const float* w1 = reinterpret_cast<const float*>(sm + eb::W1F);
  const float* b1 = reinterpret_cast<const float*>(sm + eb::B1);
  const float* b2 = reinterpret_cast<const float*>(sm + eb::B2);
  const float* nrm = reinterpret_cast<const float*>(sm + eb::NORM);
  float* dxh = reinterpret_cast<float*>(sm + eb::U);  // after the dg1 MMA
  uint8_t* G1 = sm + eb::U;
  uint8_t* DZ2 = sm + eb::U;                           // after the z2 MMA
  uint8_t* XT = sm + eb::XT;
  uint8_t* YT = sm + eb::YT;
  const int node = threadIdx.x & 127, half = threadIdx.x >> 7, f0 = half * 32;
  const bool relu = variant_of(nrm) & VAR_MLP_ONLY;
  const uint32_t lb = lane_base(tc.tmem);
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const int64_t ntiles = (N + TILE - 1) / TILE;
  bool first = true, ok = true;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t n = tile * TILE + node;
    const bool on = n < N;
    const int64_t nn = on ? n : N - 1;
    if (LBM_BWD_PF && threadIdx.x < Q + 16) {  // next tile: f_pre (9 FP32 planes), dh0 (16)
      const int64_t m0 = (tile + gridDim.x) * TILE;
      if (threadIdx.x < Q) l2_prefetch_nodes(f_pre, threadIdx.x, s.ps, 4, m0, N);
      else l2_prefetch_nodes(dh0, threadIdx.x - Q, N, 16, m0, N);
    }
    float fv[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) fv[q] = __ldg(f_pre + q * s.ps + nn);
    Moments m = moments9(fv);
    if (fxs || fx != 0.0f)
      m.ux += 0.5f * (fxs ? __ldg(fxs + nn / ((int64_t)s.nx * s.ny)) : fx) / m.rho;
    float xh[NFEAT];
#pragma unroll
    for (int q = 0; q < Q; ++q) xh[q] = (fv[q] - nrm[q]) * isg[q];
    xh[9] = (m.rho - nrm[9]) * isg[9];
    xh[10] = (m.ux - nrm[10]) * isg[10];
    xh[11] = (m.uy - nrm[11]) * isg[11];
    // GELU'(z1), the only later use of z1, kept as FP16 pairs (values in
    // [-0.2, 1.2]; dz1 is rounded to BF16 for the weight-gradient MMA anyway)
    __half2 gp1[16];
    {
      float z1[32], g[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float z = b1[f0 + c];
#pragma unroll
        for (int j = 0; j < NFEAT; ++j) z = fmaf(w1[(f0 + c) * NFEAT + j], xh[j], z);
        z1[c] = z;
      }
      act_and_grad(z1, nullptr, 32, relu, g, z1);
#pragma unroll
      for (int c = 0; c < 16; ++c) gp1[c] = __floats2half2_rn(z1[2 * c], z1[2 * c + 1]);
      st_row32(G1, node, f0, g);
      st_col<32>(YT, 80, f0, node, g);
    }
    if (half == 0) st_col<NFEAT>(YT, 80, HID, node, xh);
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(G1), 0, smem_u32(sm + eb::W2), 0, 1, 64, false);
        })) {
      ok = false;
      break;
    }
    float d[32];
    {
      float z2[32], g0[32];
      tmem_ld32(lb + f0, z2);
      ld_pf32(dh0, N, nn, f0, g0);
      act_and_grad(z2, b2 + f0, 32, relu, nullptr, d);
#pragma unroll
      for (int c = 0; c < 32; ++c) d[c] = on ? g0[c] * d[c] : 0.0f;
    }
    st_row32(DZ2, node, f0, d);
    st_col<32>(XT, 128, f0, node, d);
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem, smem_u32(DZ2), 0, smem_u32(sm + eb::W2T), 0, 1, 64, false);
        })) {
      ok = false;
      break;
    }
    tmem_ld32(lb + f0, d);
#pragma unroll
    for (int c = 0; c < 16; ++c) {  // dz1 = dg1 GELU'(z1) (0 for idle nodes)
      const float2 gp = __half22float2(gp1[c]);
      d[2 * c] *= gp.x;
      d[2 * c + 1] *= gp.y;
    }
    st_col<32>(XT, 128, HID + f0, node, d);
    if (df) {
      float px[NFEAT];
#pragma unroll
      for (int j = 0; j < NFEAT; ++j) px[j] = 0.0f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
#pragma unroll
        for (int j = 0; j < NFEAT; ++j) px[j] = fmaf(d[c], w1[(f0 + c) * NFEAT + j], px[j]);
      }
#pragma unroll
      for (int j = 0; j < NFEAT; ++j) dxh[(half * 128 + node) * NFEAT + j] = px[j];
    }
    const bool acc = !first;
    if (!tc_run(sh, tc, stw, [&] {
          umma_128xN(tc.tmem + 64, smem_u32(XT), 16384, smem_u32(YT), 10240, 2, 80, acc);
        })) {
      ok = false;
      break;
    }
    first = false;
    if (df && half == 0 && on) {
      float dx[NFEAT];
#pragma unroll
      for (int j = 0; j < NFEAT; ++j)
        dx[j] = (dxh[node * NFEAT + j] + dxh[(128 + node) * NFEAT + j]) * isg[j];
      const float ir = 1.0f / m.rho;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        df[q * s.ps + n] =
            dx[q] + dx[9] + (dx[10] * (float(ex(q)) - m.ux) + dx[11] * (float(ey(q)) - m.uy)) * ir;
    }
    tc_fence_before();
    __syncthreads();
  }
  if (ok) {
    const int row = 32 * ((threadIdx.x >> 5) & 3) + (threadIdx.x & 31);
    float* g = G + (int64_t)blockIdx.x * P::TRAINABLE;
    float v[32];
    tmem_ld32(lb + 64 + f0, v);
    if (row < HID) {
      for (int c = 0; c < 32; ++c) g[P::ENC2_W + row * HID + f0 + c] = v[c];
    }
    if (half == 0) {
      float u[16];
      tmem_ld16(lb + 128, u);  // columns 64..79: x_hat (12), ones (1)
      if (row < HID) {
        g[P::ENC2_B + row] = u[12];
      } else {
        for (int j = 0; j < NFEAT; ++j) g[P::ENC1_W + (row - HID) * NFEAT + j] = u[j];
        g[P::ENC1_B + row - HID] = u[12];
      }
    }
  }
  tc_teardown(sh, tc);
}

// ---------------------------------------------------------------------------
// Sum of the per-CTA gradient rows in a fixed order.
// accumulate: add to the gradient already in grad (the steps of a rollout).
__global__ void grad_reduce_kernel(const float* __restrict__ G, int rows,
                                   float* __restrict__ grad, bool accumulate) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P::TRAINABLE) return;
  float acc = 0.0f;
  for (int r = 0; r < rows; ++r) acc += G[(int64_t)r * P::TRAINABLE + p];
  grad[p] = accumulate ? grad[p] + acc : acc;
}

// AdamW (decoupled weight decay) on the trainable prefix.
__global__ void adamw_kernel(float* __restrict__ theta, const float* __restrict__ g,
                             float* __restrict__ m, float* __restrict__ v, float lr, float wd,
                             float b1, float b2, float eps, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P::TRAINABLE) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float mh = mp * bc1, vh = vp * bc2;
  theta[p] = theta[p] * (1.0f - lr * wd) - lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// Launchers
cudaError_t launch_collide_loss(const float* f_pre, const float* y, const float* tgt,
                                const Shape& s, float tau, const float* taus,
                                const uint8_t* packed, double* lossp, int* nblk, float* dy,
                                float* f_pred, cudaStream_t st, const float* lw) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const unsigned blocks = (unsigned)((N + 255) / 256);
  *nblk = (int)blocks;
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  gnn_collide_loss_kernel<false><<<blocks, 256, 0, st>>>(f_pre, y, tgt, s, tau, taus, 0.0f,
                                                          nullptr, packed, lossp, dy, f_pred, lw,
                                                          stw);
  return cudaGetLastError();
}

cudaError_t launch_collide_loss_channel(const float* f_pre, const float* y, const float* tgt,
                                        const Shape& s, float tau, const float* taus, float gx,
                                        const float* gxs, const uint8_t* packed, double* lossp,
                                        int* nblk, float* dy, float* f_pred, cudaStream_t st,
                                        const float* lw) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const unsigned blocks = (unsigned)((N + 255) / 256);
  *nblk = (int)blocks;
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  gnn_collide_loss_kernel<true><<<blocks, 256, 0, st>>>(f_pre, y, tgt, s, tau, taus, gx, gxs,
                                                         packed, lossp, dy, f_pred, lw, stw);
  return cudaGetLastError();
}

cudaError_t launch_collide_adjoint(const float* f_pre, const float* y, const float* f_post,
                                   const float* tgt, const float* g_in, const Shape& s, float tau,
                                   const float* taus, const uint8_t* packed, float scale,
                                   float* dy, float* dfd, cudaStream_t st) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  gnn_collide_adjoint_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(
      f_pre, y, f_post, tgt, g_in, s, tau, taus, packed, scale, dy, dfd, stw);
  return cudaGetLastError();
}

cudaError_t launch_stream_adjoint_sum(const float* a, const float* b, float* out, const Shape& s,
                                      cudaStream_t st) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  stream_adjoint_sum_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(a, b, out, s, stw);
  return cudaGetLastError();
}

cudaError_t launch_loss_finish(const double* lossp, int nblk, double count, double* loss,
                               cudaStream_t st) {
  loss_finish_kernel<<<1, 256, 0, st>>>(lossp, nblk, count, loss);
  return cudaGetLastError();
}

static unsigned grad_grid(int64_t N, int per_sm) {
  unsigned g = grid_for(N, per_sm);
  return g > (unsigned)GRAD_ROWS ? (unsigned)GRAD_ROWS : g;
}

cudaError_t launch_gnn_backward(const BackwardLaunch& bl, const Shape& s, const uint8_t* packed,
                                cudaStream_t st) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  cudaError_t e;
  if ((e = cudaMemsetAsync(bl.G, 0, (size_t)GRAD_ROWS * P::TRAINABLE * sizeof(float), st)) !=
      cudaSuccess)
    return e;
  // head: dh2 -> dh[0]
  {
    const uint32_t bytes = hb::BYTES + 1024;
    if ((e = set_smem(gnn_head_bwd_kernel, bytes)) != cudaSuccess) return e;
    gnn_head_bwd_kernel<<<grad_grid(N, 2), 256, bytes, st>>>(bl.dy, bl.h2, bl.dh[0], bl.G, s,
                                                             packed, stw);
  }
  // rounds 2 and 1 (index 1, 0): dh[0] -> dh[1] (part) -> dh[0] (in)
  const __nv_bfloat16* hs[2] = {bl.h0, bl.h1};
  const __nv_bfloat16* as[2] = {bl.a0, bl.a1};
  const __half* abs_[2] = {bl.ab0, bl.ab1};
  for (int r = 1; r >= 0; --r) {
    {
      const uint32_t bytes = rb1::BYTES + 1024;
      if ((e = set_smem(gnn_round_bwd1_kernel, bytes)) != cudaSuccess) return e;
      gnn_round_bwd1_kernel<<<grad_grid(N, LBM_RB1_CTAS), 256, bytes, st>>>(hs[r], as[r], bl.dh[0], bl.dh[1],
                                                                 bl.da, r, bl.G, s, packed, stw);
    }
    {
      const uint32_t bytes = rb2::BYTES + 1024;
      auto* kern = bl.walls ? gnn_round_bwd2_kernel<true> : gnn_round_bwd2_kernel<false>;
      if ((e = set_smem(kern, bytes)) != cudaSuccess) return e;
      kern<<<grad_grid(N, LBM_RB2_CTAS), 256, bytes, st>>>(abs_[r], bl.da, bl.dh[1], hs[r],
                                                           bl.dh[0], r, bl.G, s, packed, stw);
    }
  }
  {
    const uint32_t bytes = eb::BYTES + 1024;
    if ((e = set_smem(gnn_encode_bwd_kernel, bytes)) != cudaSuccess) return e;
    gnn_encode_bwd_kernel<<<grad_grid(N, LBM_EB_CTAS), 256, bytes, st>>>(
        bl.f_pre, bl.dh[0], bl.df, bl.G, s, bl.fx, bl.fxs, packed, stw);
  }
  grad_reduce_kernel<<<(P::TRAINABLE + 255) / 256, 256, 0, st>>>(bl.G, GRAD_ROWS, bl.grad,
                                                                   bl.accumulate);
  return cudaGetLastError();
}

cudaError_t launch_adamw(float* theta, const float* g, float* m, float* v, float lr, float wd,
                         float b1, float b2, float eps, float bc1, float bc2, cudaStream_t st) {
  adamw_kernel<<<(P::TRAINABLE + 255) / 256, 256, 0, st>>>(theta, g, m, v, lr, wd, b1, b2, eps,
                                                           bc1, bc2);
  return cudaGetLastError();
}

}  // namespace lbmgnn
