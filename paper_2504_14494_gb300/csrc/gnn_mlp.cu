// The paper's Fig. 2 network (SimpleLBMGNN: features -> Linear + ReLU ->
// Linear + ReLU -> heads, no message passing; Sec. 2.3.1) as ONE fused
// GNN-LBM step kernel: pull-stream of the stored state, moments, features,
// the three dense layers on the tensor cores, the heads and the Eq. 3
// collision, and the store.  Per node it moves only the populations (9 FP32
// loads, 9 FP32 stores: 72 bytes), like the BGK step.
//
// Work unit: a tile of 128 consecutive nodes.  One CTA per SM runs 4
// independent groups of 128 threads (thread t = node t of the group's tile,
// warp w of the group owns tensor-memory lanes 32 (w % 4)..), each looping
// over its own tiles with its own staging ring, mbarrier, named barrier and
// tensor-memory slice; the weights are shared.  The pulled populations of a
// group's next two tiles are fetched with cp.async into a 3-stage
// shared-memory ring (where lattice rows are whole tiles: per population the
// tile's source run in 16-byte chunks shared out over the group; otherwise
// 4-byte copies per node) while the current tile runs its three MMAs
// (M = 128 nodes, FP32 accumulators in tensor memory):
//   D = [x_hi | x_lo] W1x^T   (K = 32: the FP32 features split into two BF16
//                              parts, ~16 bits kept; b1 rides along as two
//                              extra K columns against feature columns of 1)
//   D = g1 W2^T + 1 b2^T      (K = 64, plus one K step for the bias)
//   D = h0 Wh'^T + 1 bh'^T    (K = 64 + bias, N = 32: the tau head and the
//                              BF16 pair hi + lo of s_df P W_h, P the
//                              conserving projection or the identity)
// and f* = f - (f - f^eq)/(tau tau_adj) + Delta f (Eq. 3, in packed FP32
// pairs of directions).  The
// activations never touch shared memory: each epilogue reads the node's
// accumulator row from tensor memory, applies ReLU, rounds to BF16
// and stores the row back into tensor memory, where the next MMA reads its
// A operand (weights B from shared memory).  Shared memory then carries
// only the weights and the staged populations, and the tensor core reads
// 14 KB of it per tile instead of 54 KB.
//
// The same kernel in its encoder mode (ENC) is the inference encoder of the
// message-passing network: the same pull and features, the two layers with
// GELU instead of ReLU, then B = W_b h0 (round 0's edge term of the
// neighbours) in place of the head; h0 and B go to HBM for the round kernels.
#include "gnn.cuh"
#include "gnn_launch.h"

namespace lbmgnn {

#ifndef LBM_MLP_GROUPS
#define LBM_MLP_GROUPS 4  // independent 128-thread tile groups per CTA (one CTA per SM)
#endif

namespace mlp {
// Shared memory holds only the weights and the staged populations: the
// activations live in tensor memory (columns 0..63: accumulator, 64..95:
// the BF16 input of the next product).
constexpr int STAGES = 3;
// Per stage and population q a run of RUN floats: position 4 + t - e_qx
// holds the value node t of the tile pulls (so a tile whose 128 nodes lie in
// one lattice row can fetch each population's source run [x0 - 4, x0 + 132)
// as 34 aligned 16-byte chunks); then 128 slots of tau.
constexpr int RUN = TILE + 8;
constexpr int CHUNKS = RUN / 4;  // 16-byte chunks per population run
constexpr int STAGE_FLOATS = Q * RUN + TILE;
// B2X / BHX: SW128 blocks whose K columns 0 and 1 hold the layer-2 and head
// biases as BF16 pairs hi + lo (~16 bits): one extra K step against a
// constant A of ones adds the bias inside the MMA.  WH is the head as this
// kernel uses it (32 output rows, see the prologue).
constexpr int NG = LBM_MLP_GROUPS;
// Encoder mode (the inference encoder of a message-passing network): the
// round-0 edge weights W_b (SW128, 64 x 64) at WB_E and the layer-2 bias
// block at B2X_E instead of the head blocks.
constexpr uint32_t WB_E = 16384, B2X_E = 24576;
constexpr uint32_t W1X = 0, W2 = 8192, WH = 16384, B2X = 20480, BHX = 28672, STG = 32768,
                   STG_BYTES = STAGE_FLOATS * 4,                   // 5408 per stage and group
                   NORM = STG + NG * STAGES * STG_BYTES,
                   SH = NORM + 128, BYTES = SH + NG * 16;
// tensor memory: group g's accumulator D at 64 g (64 columns), its A
// operand at 64 NG + 32 g (32 columns of BF16 pairs); one constant block of
// ones after them
constexpr uint32_t TM_COLS = 512, TM_ONES = 96 * NG;
__host__ __device__ constexpr uint32_t tm_d(int g) { return 64u * g; }
__host__ __device__ constexpr uint32_t tm_a(int g) { return 64u * NG + 32u * g; }
static_assert(TM_ONES + 16 <= TM_COLS, "tensor-memory columns");
static_assert(TM_COLS == 512, "one allocation of the whole tensor memory (power of two)");
}  // namespace mlp

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
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
// Moments with a fast reciprocal of rho (the MUFU approximation, ~1 ulp).
__device__ __forceinline__ Moments moments9_fast(const float (&f)[Q]) {
  const float rho = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
  const float jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
  const float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const float inv = __fdividef(1.0f, rho);
  return {rho, jx * inv, jy * inv};
}

// One layer's epilogue: ReLU(D) of the node's 64 accumulator columns (the
// bias is already in D), rounded to BF16, written back to tensor memory as
// the next product's A (32 columns of BF16 pairs).  Both halves of D are
// loaded before the one wait.
__device__ __forceinline__ void relu_to_tmem(uint32_t lane_d, uint32_t lane_a) {
  uint32_t z0[32], z1[32], w[32];
  tmem_ld32_async(lane_d, z0);
  tmem_ld32_async(lane_d + 32u, z1);
  tmem_ld_wait();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    w[j] = relu_bf16x2(__uint_as_float(z0[2 * j]), __uint_as_float(z0[2 * j + 1]));
    w[16 + j] = relu_bf16x2(__uint_as_float(z1[2 * j]), __uint_as_float(z1[2 * j + 1]));
  }
  tmem_st32(lane_a, w);
}

// The encoder's epilogue: GELU(D) (bias already in D) of the node's 64
// accumulator columns in packed FP32 pairs, rounded to BF16 pairs (w, in
// feature order), written back to tensor memory as the next product's A.
__device__ __forceinline__ void gelu_to_tmem(uint32_t lane_d, uint32_t lane_a,
                                             uint32_t (&w)[32]) {
  uint32_t z0[32], z1[32];
  tmem_ld32_async(lane_d, z0);
  tmem_ld32_async(lane_d + 32u, z1);
  tmem_ld_wait();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float2 a = gelu2(make_float2(__uint_as_float(z0[2 * j]), __uint_as_float(z0[2 * j + 1])));
    const float2 b = gelu2(make_float2(__uint_as_float(z1[2 * j]), __uint_as_float(z1[2 * j + 1])));
    w[j] = bf16x2(a.x, a.y);
    w[16 + j] = bf16x2(b.x, b.y);
  }
  tmem_st32(lane_a, w);
}

// One fused GNN-LBM step of the MLP-only network over the nodes of `geo`
// (ENC = false), or (ENC = true) the inference encoder of a message-passing
// network: the same pull, features and first two layers with GELU, then the
// round-0 edge term B = W_b h0; h0 (BF16) and B (FP16) go to HBM in the
// chunked plane layout of the round kernels.
template <class Geo, bool ENC>
__global__ void __launch_bounds__(128 * LBM_MLP_GROUPS, 1) gnn_mlp_step_kernel(
    const float* __restrict__ f_in, float* __restrict__ f_out, Geo geo, float tau0,
    const float* __restrict__ taus, const uint8_t* __restrict__ packed, bool require_mlp,
    bool rows, __nv_bfloat16* __restrict__ h0_out, __half* __restrict__ b_out, unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  const int variant = variant_of(reinterpret_cast<const float*>(packed + K::NORM));
  if (ENC ? (variant & VAR_MLP_ONLY) != 0 : !(variant & VAR_MLP_ONLY)) {
    // the MLP-only network is stepped by the MLP mode alone; message-passing
    // networks by the encoder mode and the round kernels
    if (!ENC && require_mlp && threadIdx.x == 0) raise_status(stw, ST_BLOB);
    return;
  }
  extern __shared__ uint8_t smem_raw[];
  // aligned through an integer: the staged populations are then read with
  // generic loads, measured faster here than shared-memory loads (the other
  // tensor-core kernels use smem_align1024)
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  TcShared* sh = reinterpret_cast<TcShared*>(sm + mlp::SH);
  // group grp of 128 threads: t = node of its tile, warp (t / 32) owns
  // tensor-memory lanes 32 (t / 32)..; its own tile sequence, staging ring,
  // mbarrier, tensor-memory slice and named barrier
  const int grp = threadIdx.x >> 7, t = threadIdx.x & 127;
  float* stg = reinterpret_cast<float*>(sm + mlp::STG) + grp * (mlp::STAGES * mlp::STAGE_FLOATS);
  const int64_t N = geo.count();
  const int64_t base = geo.base(), ps = geo.ps();
  const int64_t ntiles = (N + TILE - 1) / TILE;
  const int64_t first = (int64_t)blockIdx.x * mlp::NG + grp,
                stride = (int64_t)gridDim.x * mlp::NG;

  // The pulled populations of tile `tile` -> stage st (cp.async), and each
  // node's relaxation time.  rows (a stack whose rows are whole tiles,
  // 16-byte aligned planes): per population q the run [x0 - 4, x0 + 132) of
  // row y - e_qy in 16-byte chunks, wrapped at the row's ends, the chunks
  // shared out over the group's threads; otherwise each node pulls its 9
  // values from x - e_q (periodic wrap inside its lattice) with 4-byte copies.
  auto fetch = [&](int64_t tile, int st) {
    if (tile < ntiles) {
      float* sg = stg + st * mlp::STAGE_FLOATS;
      if (rows) {
        const GeoPos p = geo.pos(base + tile * TILE);  // node t = (x0 + t, y)
        if (t < 3 * mlp::CHUNKS) {  // thread t: chunk c of the 3 populations of row set rs
          const int rs = t / mlp::CHUNKS, c = t - rs * mlp::CHUNKS;
          const int dy = rs == 0 ? 0 : (rs == 1 ? -1 : 1);  // source row y + dy
          const int ys = p.y + dy < 0 ? p.ny - 1 : (p.y + dy >= p.ny ? 0 : p.y + dy);
          int xs = p.x - 4 + 4 * c;
          xs += xs < 0 ? p.nx : 0;
          xs -= xs >= p.nx ? p.nx : 0;
          const int64_t src = checked(p.lat + (int64_t)ys * p.nx + xs, base, base + N, stw);
          // row y: q = 0, 1, 3; row y - 1: q = 2, 5, 6; row y + 1: q = 4, 7, 8
          const int q0 = rs == 0 ? 0 : (rs == 1 ? 2 : 4);
          const int q1 = rs == 0 ? 1 : (rs == 1 ? 5 : 7);
          const int q2 = rs == 0 ? 3 : (rs == 1 ? 6 : 8);
          cp_async16(sg + q0 * mlp::RUN + 4 * c, f_in + q0 * ps + src);
          cp_async16(sg + q1 * mlp::RUN + 4 * c, f_in + q1 * ps + src);
          cp_async16(sg + q2 * mlp::RUN + 4 * c, f_in + q2 * ps + src);
        }
        const float* tp = geo.tau_ptr(p, taus);
        if (tp) cp_async4(sg + Q * mlp::RUN + t, tp); else sg[Q * mlp::RUN + t] = tau0;
      } else {
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
#pragma unroll
        for (int q = 0; q < Q; ++q)
          cp_async4(sg + q * mlp::RUN + 4 + t - ex(q),
                    f_in + q * ps + checked(src[q], base, base + N, stw));
        const float* tp = geo.tau_ptr(p, taus);
        if (tp) cp_async4(sg + Q * mlp::RUN + t, tp); else sg[Q * mlp::RUN + t] = tau0;
      }
    }
    cp_async_commit();  // (an empty group past the last tile keeps the counting uniform)
  };
  fetch(first, 0);
  fetch(first + stride, 1);

  copy_g2s(sm + mlp::W1X, packed + K::W1X, 8192);
  copy_g2s(sm + mlp::W2, packed + K::W2, 8192);
  copy_g2s(sm + mlp::NORM, packed + K::NORM, 128);
  if constexpr (ENC) {  // W_b: rows 64..127 of round 0's [W_a; W_b] block; the bias block 0
    copy_g2s(sm + mlp::WB_E, packed + K::round_base(0) + K::WAB + 8192, 8192);
    for (uint32_t i = threadIdx.x; i < (mlp::STG - mlp::B2X_E) / 16; i += blockDim.x)
      reinterpret_cast<uint4*>(sm + mlp::B2X_E)[i] = make_uint4(0u, 0u, 0u, 0u);
  } else {
    for (uint32_t i = threadIdx.x; i < (mlp::STG - mlp::WH) / 16; i += blockDim.x)  // head, biases: 0
      reinterpret_cast<uint4*>(sm + mlp::WH)[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();
  float* nrmw = reinterpret_cast<float*>(sm + mlp::NORM);
  if (threadIdx.x < NFEAT) {  // (mu, sigma) -> (-mu / sigma, 1 / sigma): x_hat = x rs + c
    const float rs = 1.0f / nrmw[NFEAT + threadIdx.x];
    nrmw[NFEAT + threadIdx.x] = rs;
    nrmw[threadIdx.x] = -nrmw[threadIdx.x] * rs;
  }
  // The biases ride along in the MMAs as BF16 pairs hi + lo (~16 bits):
  // b1 in K columns 12 and 13 of W1x (multiplied by feature columns equal to
  // 1), b2 and the head bias in K columns 0 and 1 of their own blocks
  // (multiplied by a constant A of ones in tensor memory).
  auto put_pair = [&](uint32_t blk, int row, int k, float b) {
    const float hi = bf16_round(b);
    *reinterpret_cast<__nv_bfloat16*>(sm + blk + sw128_off(row, k)) = __float2bfloat16_rn(hi);
    *reinterpret_cast<__nv_bfloat16*>(sm + blk + sw128_off(row, k + 1)) =
        __float2bfloat16_rn(b - hi);
  };
  if (threadIdx.x < HID) {
    const int o = threadIdx.x;
    put_pair(mlp::W1X, o, 12, __ldg(reinterpret_cast<const float*>(packed + K::B1) + o));
    put_pair(ENC ? mlp::B2X_E : mlp::B2X, o, 0,
             __ldg(reinterpret_cast<const float*>(packed + K::B2) + o));
  }
  // (MLP mode) The head as this kernel uses it (N = 32): row 0 is the tau head W_h[0]
  // (BF16 already); rows 1..9 and 17..25 hold the BF16 pair hi + lo of
  // s_df P W_h[1..9], with P the projection of the conserving variant (else
  // the identity), so that Delta f = y_q + y_{16+q} comes out of the MMA
  // (bias likewise: s_df P b_h[1..9] and b_h[0] in BHX).
  if constexpr (!ENC) {
    const float* whf = reinterpret_cast<const float*>(packed + K::WHF);  // FP32 [10][64]
    const float* bhg = reinterpret_cast<const float*>(packed + K::BH);
    const float sdf0 = __ldg(reinterpret_cast<const float*>(packed + K::NORM) + 24);
    const bool cons = variant & VAR_CONSERVATIVE;
    auto proj = [&](int q, int k) {  // s_df (P w)_q of column k (k = HID: the bias)
      auto w = [&](int r) { return k < HID ? __ldg(whf + (1 + r) * HID + k) : __ldg(bhg + 1 + r); };
      if (!cons) return sdf0 * w(q);
      float s0 = 0.f, sx = 0.f, sy = 0.f;
      for (int r = 0; r < Q; ++r) {
        const float v = w(r);
        s0 += v;
        sx += float(ex(r)) * v;
        sy += float(ey(r)) * v;
      }
      return sdf0 * (w(q) - s0 * (1.0f / 9.0f) - float(ex(q)) * sx * (1.0f / 6.0f) -
                     float(ey(q)) * sy * (1.0f / 6.0f));
    };
    for (int i = threadIdx.x; i < (Q + 1) * (HID + 1); i += blockDim.x) {
      const int q = i / (HID + 1) - 1, k = i % (HID + 1);  // q = -1: the tau row
      if (k < HID) {
        if (q < 0) {
          *reinterpret_cast<__nv_bfloat16*>(sm + mlp::WH + sw128_off(0, k)) =
              __float2bfloat16_rn(__ldg(whf + k));
        } else {
          const float v = proj(q, k), hi = bf16_round(v);
          *reinterpret_cast<__nv_bfloat16*>(sm + mlp::WH + sw128_off(1 + q, k)) =
              __float2bfloat16_rn(hi);
          *reinterpret_cast<__nv_bfloat16*>(sm + mlp::WH + sw128_off(17 + q, k)) =
              __float2bfloat16_rn(v - hi);
        }
      } else {
        put_pair(mlp::BHX, 1 + q, 0, q < 0 ? __ldg(bhg) : proj(q, HID));
      }
    }
  }
  // one mbarrier per group; warp 0 allocates all 512 tensor-memory columns
  // (a power of two, as tcgen05.alloc requires; one CTA per SM)
  if (threadIdx.x == 0)
    for (int g = 0; g < mlp::NG; ++g) {
      mbar_init(&sh[g].bar, 1);
      sh[g].abort = 0;
    }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&sh[0].tmem, mlp::TM_COLS);
  tc_fence_before();
  __syncthreads();  // (also publishes the shared-memory writes above)
  tc_fence_after();
  TcCtx tc;
  tc.bar = &sh[grp].bar;  // the group's own mbarrier; its slice of the columns:
  tc.phase = 0;
  tc.tmem = sh[0].tmem;
  const uint32_t tbase = sh[0].tmem;
  const float* nrm = nrmw;
  const uint32_t lb = lane_base(tbase);
  const uint32_t ld = lb + mlp::tm_d(grp), la = lb + mlp::tm_a(grp);
  const uint32_t td = tbase + mlp::tm_d(grp), ta = tbase + mlp::tm_a(grp),
                 tones = tbase + mlp::TM_ONES;
  const uint32_t w1x = smem_u32(sm + mlp::W1X), w2 = smem_u32(sm + mlp::W2),
                 wh = smem_u32(sm + mlp::WH), b2x = smem_u32(sm + (ENC ? mlp::B2X_E : mlp::B2X)),
                 bhx = smem_u32(sm + mlp::BHX), wb = smem_u32(sm + mlp::WB_E);
  if (grp == 0) {  // the constant A of ones for the bias K steps: K 0, 1 = 1, the rest 0
    uint32_t w[16] = {0x3F803F80u};
    tmem_st16(lane_base(tbase) + mlp::TM_ONES, w);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();  // the ones are in place for every group's MMAs
  tc_fence_after();
  // D = A W^T over nks K steps, then D += ones bias^T (one more K step)
  auto mma_bias = [&](uint32_t w, uint32_t bias, int n_out) {
    const uint32_t id = idesc_bf16(128, n_out);
    for (int ks = 0; ks < 4; ++ks)
      umma_bf16_ts(td, ta + 8u * ks, sw128_desc(w + ks * 32), id, ks > 0 ? 1u : 0u);
    umma_bf16_ts(td, tones, sw128_desc(bias), id, 1u);
  };

  // The A operand was stored to tensor memory by every thread -> barrier ->
  // one thread issues the MMA chain and commits it; all threads wait.  A
  // wait that gives up marks the group's abort word; the group leaves the
  // tile loop together at the next end-of-tile barrier (every wait after a
  // lost one is bounded too, and every thread passes the same barriers).
  volatile int* abort_flag = &sh[grp].abort;
  auto run = [&](auto issue) {
    tmem_st_wait();
    tc_fence_before();
    group_sync(grp, 128);
    if (t == 0) {
      tc_fence_after();
      issue();
      umma_commit(tc.bar);
    }
    if (!mbar_wait(tc.bar, tc.phase)) *abort_flag = 1;
    tc.phase ^= 1u;
    tc_fence_after();
  };

  int s = 0;
  for (int64_t tile = first; tile < ntiles; tile += stride) {
    fetch(tile + 2 * stride, s == 0 ? 2 : s - 1);  // the stage read two tiles ago
    cp_async_wait<2>();                             // this thread's copies of `tile`
    if (rows) group_sync(grp, 128);                 // and the other threads' chunks
    const int64_t n = tile * TILE + t;
    const float* sv = stg + s * mlp::STAGE_FLOATS + 4 + t;  // read again by the collision
    s = s == 2 ? 0 : s + 1;
    Moments m;  // of the pulled populations, kept for the collision
    {  // features normalised: A = [x_hi (k 0..11), 1, 1, 0, 0 | x_lo (k 16..27), 0 x 4]
      float fv[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) fv[q] = sv[q * mlp::RUN - ex(q)];
      m = moments9_fast(fv);
      float xh[NFEAT];
#pragma unroll
      for (int q = 0; q < Q; ++q) xh[q] = fmaf(fv[q], nrm[NFEAT + q], nrm[q]);
      xh[9] = fmaf(m.rho, nrm[NFEAT + 9], nrm[9]);
      xh[10] = fmaf(m.ux, nrm[NFEAT + 10], nrm[10]);
      xh[11] = fmaf(m.uy, nrm[NFEAT + 11], nrm[11]);
      uint32_t w[16];
#pragma unroll
      for (int j = 0; j < NFEAT / 2; ++j) {
        const uint32_t hw = bf16x2(xh[2 * j], xh[2 * j + 1]);
        const float2 lo = __fadd2_rn(make_float2(xh[2 * j], xh[2 * j + 1]),
                                     make_float2(-__uint_as_float(hw << 16),
                                                 -__uint_as_float(hw & 0xFFFF0000u)));
        w[j] = hw;
        w[8 + j] = bf16x2(lo.x, lo.y);
      }
      w[6] = 0x3F803F80u;  // BF16 pair (1, 1): the bias columns
      w[7] = w[14] = w[15] = 0u;
      tmem_st16(la, w);
    }
    run([&] { umma_128xN_ts(td, ta, w1x, 64, 2); });
    if constexpr (ENC) {
      uint32_t w[32];
      gelu_to_tmem(ld, la, w);  // g1 = GELU(W1 x + b1) (bias in D)
      run([&] { mma_bias(w2, b2x, 64); });
      gelu_to_tmem(ld, la, w);  // h0 = GELU(W2 g1 + b2), and to HBM
      if (n < N) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
          *chunk8w(h0_out, N, n, 8 * c) =
              make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
      }
      run([&] { umma_128xN_ts(td, ta, wb, 64, 4); });  // B = W_b h0 (no bias)
      uint32_t z0[32], z1[32];
      tmem_ld32_async(ld, z0);
      tmem_ld32_async(ld + 32u, z1);
      tmem_ld_wait();
      if (n < N) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t* z = c < 4 ? z0 + 8 * c : z1 + 8 * (c - 4);
          uint32_t hv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __half2 hh = __floats2half2_rn(__uint_as_float(z[2 * j]),
                                                 __uint_as_float(z[2 * j + 1]));
            hv[j] = *reinterpret_cast<const uint32_t*>(&hh);
          }
          *chunk8w(b_out, N, n, 8 * c) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        }
      }
    } else {  // MLP mode: the head and Eq. 3
      relu_to_tmem(ld, la);  // g1 = ReLU(W1 x + b1) (bias in D)
      run([&] { mma_bias(w2, b2x, 64); });
      relu_to_tmem(ld, la);  // h0 = ReLU(W2 g1 + b2) (bias in D)
      run([&] { mma_bias(wh, bhx, 32); });
      {  // heads and Eq. 3
        float y[32];
        tmem_ld32(ld, y);
        float fv[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) fv[q] = sv[q * mlp::RUN - ex(q)];
        const float tau = sv[Q * mlp::RUN - 4];
        // tau_adj = 1/2 + sigmoid(y_0) = 1 + tanh(y_0 / 2) / 2 (or 1)
        const float tadj = (variant & VAR_FIXED_TAU)
                               ? 1.0f
                               : fmaf(0.5f, tanh_fast(0.5f * y[0]), 1.0f);
        const float inv = __fdividef(1.0f, tau * tadj);
        // Delta f = s_df P y_1..9 (hi + lo rows of the head)
        auto dpair = [&](int q) {
          return __fadd2_rn(make_float2(y[1 + q], y[2 + q]), make_float2(y[17 + q], y[18 + q]));
        };
        // Eq. 3, f* = f (1 - 1/t) + f^eq / t + Delta f, in packed FP32 pairs
        // of directions with equal weights: f^eq_q = w rho (c1 + e.u (3 + 4.5 e.u)),
        // c1 = 1 - 1.5 u^2; directions 3, 4 and 7, 8 are 1, 2 and 5, 6 with
        // e.u negated (the sign moves onto the 3).
        const float c1 = 1.0f - 1.5f * (m.ux * m.ux + m.uy * m.uy);
        const float omi = 1.0f - inv;
        const float2 C1 = make_float2(c1, c1), INV = make_float2(inv, inv),
                     OMI = make_float2(omi, omi), H45 = make_float2(4.5f, 4.5f);
        const float2 E1 = make_float2(m.ux, m.uy);                  // e.u of q = 1, 2
        const float2 E2 = make_float2(m.ux + m.uy, m.uy - m.ux);    // e.u of q = 5, 6
        const float r9 = m.rho * (1.0f / 9.0f), r36 = m.rho * (1.0f / 36.0f);
        auto pair = [&](int q, float2 e, float sg, float w) {
          const float2 tt = __ffma2_rn(e, __ffma2_rn(e, H45, make_float2(3.0f * sg, 3.0f * sg)), C1);
          const float2 feq = __fmul2_rn(tt, make_float2(w, w));
          const float2 fq = make_float2(fv[q], fv[q + 1]);
          return __fadd2_rn(__ffma2_rn(feq, INV, __fmul2_rn(fq, OMI)), dpair(q));
        };
        const float2 o12 = pair(1, E1, 1.0f, r9), o34 = pair(3, E1, -1.0f, r9);
        const float2 o56 = pair(5, E2, 1.0f, r36), o78 = pair(7, E2, -1.0f, r36);
        const float o0 = fmaf(m.rho * (4.0f / 9.0f) * c1, inv, fv[0] * omi) + (y[1] + y[17]);
        if (n < N) {
          float* o = f_out + base + n;
          o[0] = o0;
          o[ps] = o12.x, o[2 * ps] = o12.y, o[3 * ps] = o34.x, o[4 * ps] = o34.y;
          o[5 * ps] = o56.x, o[6 * ps] = o56.y, o[7 * ps] = o78.x, o[8 * ps] = o78.y;
        }
      }
    }
    tc_fence_before();
    group_sync(grp, 128);  // the head's accumulator is read before the next tile's MMA
    if (*abort_flag) {     // a wait gave up: the whole group stops here
      if (t == 0) raise_status(stw, ST_TIMEOUT);
      break;
    }
  }
  cp_async_wait<0>();
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tbase, mlp::TM_COLS);
}

template <class Geo, bool ENC = false>
static cudaError_t mlp_step(const float* f_in, float* f_out, const Geo& geo, int64_t N, float tau,
                            const float* taus, const uint8_t* packed, bool require_mlp, bool rows,
                            cudaStream_t st, __nv_bfloat16* h0 = nullptr, __half* b = nullptr) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  if (N <= 0) return cudaSuccess;
  const uint32_t bytes = mlp::BYTES + 1024;
  cudaError_t e;
  if ((e = set_smem(gnn_mlp_step_kernel<Geo, ENC>, bytes)) != cudaSuccess) return e;
  // one CTA (NG tile groups) per SM, fewer for small lattices
  const int64_t ntiles = (N + TILE - 1) / TILE;
  const int64_t want = (ntiles + mlp::NG - 1) / mlp::NG;
  const unsigned grid = (unsigned)(want < num_sms() ? want : num_sms());
  gnn_mlp_step_kernel<Geo, ENC><<<grid, 128 * mlp::NG, bytes, st>>>(
      f_in, f_out, geo, tau, taus, packed, require_mlp, rows, h0, b, stw);
  return cudaGetLastError();
}

cudaError_t launch_gnn_mlp_step(const float* f_in, float* f_out, const Shape& s, float tau,
                                const float* taus, const uint8_t* packed, bool require_mlp,
                                cudaStream_t st) {
  // row runs: every tile inside one lattice row, 16-byte aligned population planes
  const bool rows = s.nx % TILE == 0 && s.ps % 4 == 0 &&
                    (reinterpret_cast<uintptr_t>(f_in) & 15) == 0;
  return mlp_step(f_in, f_out, make_geo_stack(s), (int64_t)s.nb * s.ny * s.nx, tau, taus, packed,
                  require_mlp, rows, st);
}

cudaError_t launch_gnn_encode_fused(const float* f_in, const Shape& s, const uint8_t* packed,
                                    __nv_bfloat16* h0, __half* b, cudaStream_t st) {
  const bool rows = s.nx % TILE == 0 && s.ps % 4 == 0 &&
                    (reinterpret_cast<uintptr_t>(f_in) & 15) == 0;
  return mlp_step<GeoStack, true>(f_in, nullptr, make_geo_stack(s), (int64_t)s.nb * s.ny * s.nx,
                                  1.0f, nullptr, packed, false, rows, st, h0, b);
}

cudaError_t launch_gnn_encode_fused_table(const float* f_in, const LatDesc* lat, int first, int n,
                                          const int* hint, int64_t base, int64_t count, int64_t ps,
                                          const uint8_t* packed, __nv_bfloat16* h0, __half* b,
                                          cudaStream_t st) {
  const GeoTable geo{lat, first, n, base, count, ps, hint};
  return mlp_step<GeoTable, true>(f_in, nullptr, geo, count, 0.0f, nullptr, packed, false, false,
                                  st, h0, b);
}

cudaError_t launch_gnn_mlp_step_table(const float* f_in, float* f_out, const LatDesc* lat,
                                      int first, int n, const int* hint, int64_t base,
                                      int64_t count, int64_t ps, const uint8_t* packed,
                                      cudaStream_t st, int per_sm) {
  const GeoTable geo{lat, first, n, base, count, ps, hint};
  (void)per_sm;  // one CTA of LBM_MLP_GROUPS tile groups per SM, whatever the batch plan chose
  return mlp_step(f_in, f_out, geo, count, 0.0f, nullptr, packed, false, false, st);
}

}  // namespace lbmgnn
