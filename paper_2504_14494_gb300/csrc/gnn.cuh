// GNN-enhanced collision: shared definitions (paper Sec. 2.2-2.3, Fig. 2,
// Eq. 3).
//
// Network (widths and message form are this library's reading; the paper
// gives the components, not the formulas):
//   x_hat = ([f_0..f_8, rho, u_x, u_y] - mu) / sigma                  (12)
//   h0 = GELU(W2 GELU(W1 x_hat + b1) + b2)                            (64)
//   round r = 0, 1 over the 8 lattice neighbours j = i + e_k (periodic):
//     m_ik = GELU(W_e [h_i; h_j; e_k] + b_e)
//          = GELU(A_i + B_j + c_k), A = W_a h, B = W_b h, c_k = W_c e_k + b_e
//     a_i = sum_k m_ik;   h_i <- h_i + GELU(W_n [h_i; a_i] + b_n)
//   y = W_h h2 + b_h                                                  (10)
//   tau_adj = 1/2 + sigmoid(y_0),  Delta f_i = s_df y_{1+i}
//   f*_i = f_i - (f_i - f_i^eq) / (tau tau_adj) + Delta f_i            (Eq. 3)
// GELU is the tanh form.  Weight matrices are used as BF16 (round to nearest
// even of the FP32 parameters); biases, mu, sigma, s_df as FP32.  Dense
// contractions over 128-node tiles run on tcgen05 (BF16 in, FP32 accumulate).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "umma.cuh"

namespace lbmgnn {

constexpr int HID = 64;
constexpr int NFEAT = 12;
constexpr int NOUT = 10;
constexpr int TILE = 128;  // nodes per MMA tile (M)

// ---- flat FP32 parameter vector (interface, see include/lbmgnn.h) -----------
namespace P {
constexpr int ENC1_W = 0, ENC1_B = 768, ENC2_W = 832, ENC2_B = 4928;
constexpr int ROUND0 = 4992, ROUND_SIZE = 16640;
constexpr int EDGE_W = 0, EDGE_B = 8320, NODE_W = 8384, NODE_B = 16576;  // within a round
constexpr int HEAD_W = 38272, HEAD_B = 38912;
constexpr int TRAINABLE = 38922;
constexpr int MU = 38922, SIGMA = 38934, S_DF = 38946, VARIANT = 38947;
constexpr int TOTAL = 38948;
}  // namespace P

// ---- packed device image of the parameters (byte offsets) -------------------
// SW128 blocks are the exact shared-memory images the MMAs read.
namespace K {
constexpr uint32_t W1F = 0;       // fp32 [64][12] (BF16-rounded values)
constexpr uint32_t B1 = 3072;     // fp32 [64]
constexpr uint32_t B2 = 3328;     // fp32 [64]
constexpr uint32_t NORM = 3584;   // fp32 mu[12], sigma[12], s_df, variant, pad, validity word
constexpr uint32_t BH = 3712;     // fp32 [16] (10 used)
constexpr uint32_t WHF = 3776;    // fp32 [10][64] (BF16-rounded values)
constexpr uint32_t W2 = 7168;     // SW128 [64 out x 64 in]
constexpr uint32_t W2T = 15360;   // SW128 [64 in x 64 out]
constexpr uint32_t WH = 23552;    // SW128 [16 out (10 used) x 64 in]
constexpr uint32_t ROUND0 = 25600;
constexpr uint32_t ROUND_SIZE = 68608;
// within a round
constexpr uint32_t WAB = 0;        // SW128 [128 out (a rows, then b rows) x 64 in]
constexpr uint32_t WABT = 16384;   // 2 SW128 blocks [64 in x 64 out], block kb = W_a / W_b
constexpr uint32_t WN = 32768;     // 2 SW128 blocks [64 out x 64 in], block 0: h part, 1: a part
constexpr uint32_t WNT = 49152;    // SW128 [128 in x 64 out]
constexpr uint32_t CK = 65536;     // fp32 [8][64]: c_k = W_c e_k + b_e, k = 1..8
constexpr uint32_t BE = 67584;     // fp32 [64]
constexpr uint32_t BN = 67840;     // fp32 [64]
// SW128 [64 out x 64]: k 0..11 = W1 (BF16), k 16..27 = W1 again, rest 0; the
// encoder's first layer multiplies it with [x_hi | x_lo] (x = x_hi + x_lo,
// both BF16), which keeps ~16 bits of the FP32 features.
constexpr uint32_t W1X = ROUND0 + 2 * ROUND_SIZE;  // 162816
constexpr uint32_t TOTAL = W1X + 8192;              // 171008
__host__ __device__ constexpr uint32_t round_base(int r) { return ROUND0 + r * ROUND_SIZE; }
// Validity word of the image (slot 31 of NORM), written by the pack kernel
// when the fixed values of the parameter vector are usable: "LBG" followed
// by the layout version (LBM_PACKED_LAYOUT_VERSION, as an ASCII digit).
constexpr uint32_t MAGIC_SLOT = NORM + 31 * 4;
constexpr uint32_t MAGIC = 0x4C424730u + LBM_PACKED_LAYOUT_VERSION;
static_assert(LBM_PACKED_LAYOUT_VERSION >= 1 && LBM_PACKED_LAYOUT_VERSION <= 9,
              "layout version is one ASCII digit of the validity word");
}  // namespace K

// Every kernel that reads a packed image checks its validity word first; on
// a mismatch (an image never packed, or packed from invalid fixed values)
// thread 0 of each CTA raises ST_BLOB and the whole CTA returns before any
// other access, so nothing is computed from it.
__device__ __forceinline__ bool blob_ok(const uint8_t* packed, unsigned* stw) {
  if (__ldg(reinterpret_cast<const unsigned*>(packed + K::MAGIC_SLOT)) == K::MAGIC) return true;
  if (threadIdx.x == 0 && stw) atomicOr(stw, (unsigned)ST_BLOB);
  return false;
}

// ---- activations ----------------------------------------------------------------
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// GELU, tanh form: 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
__device__ __forceinline__ float gelu(float z) {
  const float u = z * (0.7978845608028654f + 0.0356774081363001f * z * z);
  const float hz = 0.5f * z;
  return fmaf(hz, tanh_fast(u), hz);
}
// Two GELUs with Blackwell's packed FP32 pair arithmetic (FMUL2/FFMA2: one
// instruction for both lanes); same formula as gelu().
__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 c0 = make_float2(0.7978845608028654f, 0.7978845608028654f);
  const float2 c1 = make_float2(0.0356774081363001f, 0.0356774081363001f);
  const float2 h = make_float2(0.5f, 0.5f);
  const float2 u = __fmul2_rn(z, __ffma2_rn(c1, __fmul2_rn(z, z), c0));
  const float2 hz = __fmul2_rn(h, z);
  return __ffma2_rn(hz, make_float2(tanh_fast(u.x), tanh_fast(u.y)), hz);
}
// v[c] <- act(v[c] + b[c]) for c < n (n even), GELU in packed pairs.
__device__ __forceinline__ void bias_act(float* v, const float* b, int n, bool relu) {
  if (relu) {
#pragma unroll
    for (int c = 0; c < n; ++c) v[c] = fmaxf(v[c] + b[c], 0.0f);
    return;
  }
#pragma unroll
  for (int c = 0; c < n; c += 2) {
    const float2 z = __fadd2_rn(make_float2(v[c], v[c + 1]), make_float2(b[c], b[c + 1]));
    const float2 g = gelu2(z);
    v[c] = g.x;
    v[c + 1] = g.y;
  }
}
// GELU and its derivative.
__device__ __forceinline__ float gelu_grad(float z) {
  const float z2 = z * z;
  const float u = z * (0.7978845608028654f + 0.0356774081363001f * z2);
  const float t = tanh_fast(u);
  const float du = 0.7978845608028654f + 0.1070322244089003f * z2;
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * du;
}
__device__ __forceinline__ float sigmoid_acc(float y) { return 0.5f * (1.0f + tanhf(0.5f * y)); }

// Network variants (flags in the last fixed parameter): MLP-only network of
// the paper's Fig. 2 (ReLU encoder, no message passing), the correction
// Delta f projected to carry no mass and no momentum, and a network whose
// relaxation-time head is not used (tau_adj = 1: Eq. 3 keeps the BGK
// relaxation time and the network acts through Delta f alone).
enum : int { VAR_MLP_ONLY = 1, VAR_CONSERVATIVE = 2, VAR_FIXED_TAU = 4, VAR_ALL = 7 };
__device__ __forceinline__ int variant_of(const float* nrm) { return __float2int_rn(nrm[25]); }
// tau_adj of Eq. 3: 1/2 + sigmoid(y_0), or 1 for the fixed-tau variant.
__device__ __forceinline__ float tau_adj_of(float y0, int variant) {
  return (variant & VAR_FIXED_TAU) ? 1.0f : 0.5f + sigmoid_acc(y0);
}
__device__ __forceinline__ float act(float z, bool relu) { return relu ? fmaxf(z, 0.0f) : gelu(z); }
// gelu_grad() of two values with packed FP32 pair arithmetic.
__device__ __forceinline__ float2 gelu_grad2(float2 z) {
  const float2 c0 = make_float2(0.7978845608028654f, 0.7978845608028654f);
  const float2 c1 = make_float2(0.0356774081363001f, 0.0356774081363001f);
  const float2 c3 = make_float2(0.1070322244089003f, 0.1070322244089003f);
  const float2 h = make_float2(0.5f, 0.5f), one = make_float2(1.0f, 1.0f);
  const float2 z2 = __fmul2_rn(z, z);
  const float2 u = __fmul2_rn(z, __ffma2_rn(c1, z2, c0));
  const float2 t = make_float2(tanh_fast(u.x), tanh_fast(u.y));
  const float2 omt = __ffma2_rn(make_float2(-t.x, -t.y), t, one);  // 1 - t^2
  const float2 q = __fmul2_rn(__fmul2_rn(__fmul2_rn(h, z), omt), __ffma2_rn(c3, z2, c0));
  return __fadd2_rn(__ffma2_rn(h, t, h), q);
}
// v[c] <- act(v[c] + b[c]) for c < n (n even): g receives the activations,
// d the derivatives at the same points (either may be NULL).
__device__ __forceinline__ void act_and_grad(const float* z, const float* b, int n, bool relu,
                                             float* g, float* d) {
#pragma unroll
  for (int c = 0; c < n; c += 2) {
    const float2 x = b ? __fadd2_rn(make_float2(z[c], z[c + 1]), make_float2(b[c], b[c + 1]))
                       : make_float2(z[c], z[c + 1]);
    if (relu) {
      if (g) g[c] = fmaxf(x.x, 0.0f), g[c + 1] = fmaxf(x.y, 0.0f);
      if (d) d[c] = x.x > 0.0f ? 1.0f : 0.0f, d[c + 1] = x.y > 0.0f ? 1.0f : 0.0f;
    } else {
      if (g) {
        const float2 r = gelu2(x);
        g[c] = r.x, g[c + 1] = r.y;
      }
      if (d) {
        const float2 r = gelu_grad2(x);
        d[c] = r.x, d[c + 1] = r.y;
      }
    }
  }
}
__device__ __forceinline__ float act_grad(float z, bool relu) {
  return relu ? (z > 0.0f ? 1.0f : 0.0f) : gelu_grad(z);
}
// d <- d - sum(d)/9 - e_x sum(e_x d)/6 - e_y sum(e_y d)/6 (D2Q9: 1, e_x, e_y
// are orthogonal with squared norms 9, 6, 6).
__device__ __forceinline__ void conserve9(float (&d)[9]) {
  float s = 0.0f, sx = 0.0f, sy = 0.0f;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    s += d[q];
    sx += float(ex(q)) * d[q];
    sy += float(ey(q)) * d[q];
  }
#pragma unroll
  for (int q = 0; q < 9; ++q)
    d[q] -= s * (1.0f / 9.0f) + float(ex(q)) * sx * (1.0f / 6.0f) + float(ey(q)) * sy * (1.0f / 6.0f);
}

// ---- BF16 vectors ------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ void unpack_bf16x8(const uint4& u, float* out) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    out[2 * i] = __uint_as_float(w[i] << 16);
    out[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}
__device__ __forceinline__ uint4 pack_bf16x8(const float* v) {
  return make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                    pack_bf16x2(v[6], v[7]));
}
// FP16 vectors (the edge terms A | B are stored as FP16: 11-bit significand).
__device__ __forceinline__ void unpack_h8(const uint4& u, float* out) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
    out[2 * i] = f.x;
    out[2 * i + 1] = f.y;
  }
}
__device__ __forceinline__ uint4 pack_h8(const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void st_h32(__half* p, const float* v) {
  uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c] = pack_h8(v + 8 * c);
}
__device__ __forceinline__ __half2 u32_as_h2(uint32_t u) {
  return *reinterpret_cast<const __half2*>(&u);
}
__device__ __forceinline__ uint32_t h2_as_u32(__half2 h) {
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ __half2 tanh_h2(__half2 x) {
  uint32_t y;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<const uint32_t*>(&x)));
  return u32_as_h2(y);
}
// GELU (tanh form) on two FP16 values: 0.5 z (1 + tanh(z (c0 + c1 z^2))).
// Saturated arguments give exact results: z^2 may overflow to inf, which
// only makes u = +-inf and tanh(u) = +-1, and hz + hz tanh(u) is one fused
// operation, so a strongly negative z gives exactly 0.
__device__ __forceinline__ __half2 gelu_h2(__half2 z) {
  const __half2 c0 = __float2half2_rn(0.7978845608028654f);
  const __half2 c1 = __float2half2_rn(0.0356774081363001f);
  const __half2 hh = __float2half2_rn(0.5f);
  const __half2 u = __hmul2(z, __hfma2(c1, __hmul2(z, z), c0));
  const __half2 hz = __hmul2(hh, z);
  return __hfma2(hz, tanh_h2(u), hz);
}

// z^2 for the GELU derivative in FP16, capped at 64.  z^2 itself overflows
// FP16 for |z| >= 256, and inf times the exact zero 1 - t^2 of the saturated
// tanh would give NaN.  Beyond |z| = 8 the cap changes nothing: u = z (c0 +
// 64 c1) is then past 24, where tanh(u) is +-1 in FP16, so the derivative is
// already its saturated value (1 for z > 0, 0 for z < 0).
__device__ __forceinline__ __half2 zsq_capped_h2(__half2 z) {
  return __hmin2(__hmul2(z, z), __float2half2_rn(64.0f));
}

// Derivative of the tanh-form GELU on two FP16 values:
// 1/2 (1 + t) + 1/2 z (1 - t^2) u'(z), t = tanh(u), u = z (c0 + c1 z^2).
__device__ __forceinline__ __half2 gelu_grad_h2(__half2 z) {
  const __half2 c0 = __float2half2_rn(0.7978845608028654f);
  const __half2 c1 = __float2half2_rn(0.0356774081363001f);
  const __half2 c3 = __float2half2_rn(0.1070322244089003f);
  const __half2 hh = __float2half2_rn(0.5f);
  const __half2 one = __float2half2_rn(1.0f);
  const __half2 z2 = zsq_capped_h2(z);
  const __half2 t = tanh_h2(__hmul2(z, __hfma2(c1, z2, c0)));
  const __half2 q = __hmul2(__hmul2(z, __hfma2(__hneg2(t), t, one)), __hfma2(c3, z2, c0));
  return __hfma2(hh, __hadd2(t, q), hh);
}

// Twice the derivative, 2 GELU'(z) = 1 + t + z (1 - t^2) (c0 + 3 c1 z^2), in
// packed FP16 (sums of these stay well conditioned: each term is in
// [-0.26, 2.26]).
__device__ __forceinline__ __half2 gelu_grad2_h2(__half2 z) {
  const __half2 c0 = __float2half2_rn(0.7978845608028654f);
  const __half2 c1 = __float2half2_rn(0.0356774081363001f);
  const __half2 c3 = __float2half2_rn(0.1070322244089003f);
  const __half2 one = __float2half2_rn(1.0f);
  const __half2 z2 = zsq_capped_h2(z);
  const __half2 t = tanh_h2(__hmul2(z, __hfma2(c1, z2, c0)));
  const __half2 zr = __hmul2(z, __hfma2(__hneg2(t), t, one));
  return __hfma2(zr, __hfma2(c3, z2, c0), __hadd2(t, one));
}

__device__ __forceinline__ float bf16_round(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// Writes 32 values (features f0..f0+31, f0 a multiple of 8) of row `row` of an
// SW128 block at `blk` as BF16.
__device__ __forceinline__ void st_row32(uint8_t* blk, int row, int f0, const float* v) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int chunk = (f0 >> 3) + c;
    *reinterpret_cast<uint4*>(blk + row * 128 + ((chunk ^ (row & 7)) << 4)) = pack_bf16x8(v + 8 * c);
  }
}
// Reads 32 BF16 values (features f0..f0+31) of row `row` of an SW128 block.
__device__ __forceinline__ void ld_row32(const uint8_t* blk, int row, int f0, float* v) {
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int chunk = (f0 >> 3) + c;
    unpack_bf16x8(*reinterpret_cast<const uint4*>(blk + row * 128 + ((chunk ^ (row & 7)) << 4)),
                  v + 8 * c);
  }
}
// 32 consecutive BF16 values from global memory (64 bytes, 16-byte aligned).
__device__ __forceinline__ void ld_g32(const __nv_bfloat16* p, float* v) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int c = 0; c < 4; ++c) unpack_bf16x8(__ldg(q + c), v + 8 * c);
}
__device__ __forceinline__ void st_g32(__nv_bfloat16* p, const float* v) {
  uint4* q = reinterpret_cast<uint4*>(p);
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c] = pack_bf16x8(v + 8 * c);
}

// ---- chunked ("plane") layout of per-node activations ---------------------------
// A per-node tensor [N][F] is stored as F/8 planes (2-byte types) or F/4
// planes (FP32) of N nodes x 16 bytes: value (n, f) of a 2-byte tensor sits at
// ((f / 8) * N + n) * 8 + f % 8, of an FP32 tensor at ((f / 4) * N + n) * 4 +
// f % 4.  A warp reading one 16-byte chunk of 32 consecutive nodes then reads
// 512 contiguous bytes.
template <typename T>
__device__ __forceinline__ const uint4* chunk8(const T* base, int64_t N, int64_t n, int f) {
  return reinterpret_cast<const uint4*>(base + ((int64_t)(f >> 3) * N + n) * 8);
}
template <typename T>
__device__ __forceinline__ uint4* chunk8w(T* base, int64_t N, int64_t n, int f) {
  return reinterpret_cast<uint4*>(base + ((int64_t)(f >> 3) * N + n) * 8);
}
__device__ __forceinline__ const float4* chunk4(const float* base, int64_t N, int64_t n, int f) {
  return reinterpret_cast<const float4*>(base + ((int64_t)(f >> 2) * N + n) * 4);
}
__device__ __forceinline__ float4* chunk4w(float* base, int64_t N, int64_t n, int f) {
  return reinterpret_cast<float4*>(base + ((int64_t)(f >> 2) * N + n) * 4);
}
// 32 BF16 values (features f0..f0+31) of node n / their store.
__device__ __forceinline__ void ld_pb32(const __nv_bfloat16* base, int64_t N, int64_t n, int f0,
                                        float* v) {
#pragma unroll
  for (int c = 0; c < 4; ++c) unpack_bf16x8(__ldg(chunk8(base, N, n, f0 + 8 * c)), v + 8 * c);
}
__device__ __forceinline__ void st_pb32(__nv_bfloat16* base, int64_t N, int64_t n, int f0,
                                        const float* v) {
#pragma unroll
  for (int c = 0; c < 4; ++c) *chunk8w(base, N, n, f0 + 8 * c) = pack_bf16x8(v + 8 * c);
}
__device__ __forceinline__ void st_ph32(__half* base, int64_t N, int64_t n, int f0, const float* v) {
#pragma unroll
  for (int c = 0; c < 4; ++c) *chunk8w(base, N, n, f0 + 8 * c) = pack_h8(v + 8 * c);
}
// 32 FP32 values (features f0..f0+31) of node n / their store.
__device__ __forceinline__ void ld_pf32(const float* base, int64_t N, int64_t n, int f0, float* v) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float4 t = __ldg(chunk4(base, N, n, f0 + 4 * c));
    v[4 * c] = t.x;
    v[4 * c + 1] = t.y;
    v[4 * c + 2] = t.z;
    v[4 * c + 3] = t.w;
  }
}
__device__ __forceinline__ void st_pf32(float* base, int64_t N, int64_t n, int f0, const float* v) {
#pragma unroll
  for (int c = 0; c < 8; ++c)
    *chunk4w(base, N, n, f0 + 4 * c) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}

// NF (16 or 32) values versions of the helpers above.
template <int NF>
__device__ __forceinline__ void ld_pb(const __nv_bfloat16* base, int64_t N, int64_t n, int f0,
                                      float* v) {
#pragma unroll
  for (int c = 0; c < NF / 8; ++c) unpack_bf16x8(__ldg(chunk8(base, N, n, f0 + 8 * c)), v + 8 * c);
}
template <int NF>
__device__ __forceinline__ void st_pb(__nv_bfloat16* base, int64_t N, int64_t n, int f0,
                                      const float* v) {
#pragma unroll
  for (int c = 0; c < NF / 8; ++c) *chunk8w(base, N, n, f0 + 8 * c) = pack_bf16x8(v + 8 * c);
}
template <int NF>
__device__ __forceinline__ void st_ph(__half* base, int64_t N, int64_t n, int f0, const float* v) {
#pragma unroll
  for (int c = 0; c < NF / 8; ++c) *chunk8w(base, N, n, f0 + 8 * c) = pack_h8(v + 8 * c);
}
template <int NF>
__device__ __forceinline__ void st_row(uint8_t* blk, int row, int f0, const float* v) {
#pragma unroll
  for (int c = 0; c < NF / 8; ++c) {
    const int chunk = (f0 >> 3) + c;
    *reinterpret_cast<uint4*>(blk + row * 128 + ((chunk ^ (row & 7)) << 4)) = pack_bf16x8(v + 8 * c);
  }
}
template <int NF>
__device__ __forceinline__ void ld_row(const uint8_t* blk, int row, int f0, float* v) {
#pragma unroll
  for (int c = 0; c < NF / 8; ++c) {
    const int chunk = (f0 >> 3) + c;
    unpack_bf16x8(*reinterpret_cast<const uint4*>(blk + row * 128 + ((chunk ^ (row & 7)) << 4)),
                  v + 8 * c);
  }
}
template <int NF>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[NF]) {
  if constexpr (NF == 32) {
    tmem_ld32(taddr, v);
  } else {
    tmem_ld16(taddr, v);
  }
}

// Division of a 32-bit unsigned n < 2^31 by a fixed divisor d >= 1 with one
// multiply-high (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1 (the low 32 bits of the 33-bit multiplier
// floor(2^(32+l) / d) + 1), n / d = (umulhi(m, n) + n) >> l.
struct FastDiv {
  uint32_t d, m, l;
};
inline FastDiv fast_div(uint32_t d) {
  uint32_t l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
  return {d, (uint32_t)m, l};
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (__umulhi(f.m, n) + n) >> f.l;
}

// Node coordinates within the stacked lattices.
struct NodeXY {
  int x, y;
  int64_t lat;  // index of the lattice's first node
};
__device__ __forceinline__ NodeXY node_xy(int64_t n, const Shape& s) {
  const int64_t row = n / s.nx;
  const int x = (int)(n - row * s.nx);
  const int64_t b = row / s.ny;
  const int y = (int)(row - b * s.ny);
  return {x, y, b * s.ny * s.nx};
}
__device__ __forceinline__ int64_t node_at(const NodeXY& p, int dx, int dy, const Shape& s) {
  int x = p.x + dx, y = p.y + dy;
  x = x < 0 ? x + s.nx : (x >= s.nx ? x - s.nx : x);
  y = y < 0 ? y + s.ny : (y >= s.ny ? y - s.ny : y);
  return p.lat + (int64_t)y * s.nx + x;
}

// ---- node geometry -------------------------------------------------------------
// The forward kernels see a contiguous range of `count()` nodes starting at
// global node `base()` of the population buffers (plane stride `ps()`), and
// map a global node to its lattice through one of two geometries: a stack
// of equal lattices, or a table of lattices of any size (batched runs).
struct GeoPos {
  int x, y, nx, ny;
  int64_t lat;  // global index of the lattice's first node
  int b;        // lattice index (relaxation-time lookup)
};
__device__ __forceinline__ int64_t geo_nbr(const GeoPos& p, int dx, int dy) {
  int x = p.x + dx, y = p.y + dy;
  x = x < 0 ? x + p.nx : (x >= p.nx ? x - p.nx : x);
  y = y < 0 ? y + p.ny : (y >= p.ny ? y - p.ny : y);
  return p.lat + (int64_t)y * p.nx + x;
}

struct GeoStack {
  static constexpr bool kWalls = false;  // periodic in x and y
  Shape s;
  FastDiv dnx, dny;  // for stacks of fewer than 2^31 nodes (`small`)
  bool small;
  __device__ __forceinline__ int64_t count() const { return (int64_t)s.nb * s.ny * s.nx; }
  __device__ __forceinline__ int64_t base() const { return 0; }
  __device__ __forceinline__ int64_t ps() const { return s.ps; }
  __device__ __forceinline__ GeoPos pos(int64_t g) const {
    if (small) {
      const uint32_t gu = (uint32_t)g, row = fdiv(gu, dnx), b = fdiv(row, dny);
      return {(int)(gu - row * (uint32_t)s.nx), (int)(row - b * (uint32_t)s.ny), s.nx, s.ny,
              (int64_t)b * s.ny * s.nx, (int)b};
    }
    const int64_t row = g / s.nx;
    const int x = (int)(g - row * s.nx);
    const int64_t b = row / s.ny;
    const int y = (int)(row - b * s.ny);
    return {x, y, s.nx, s.ny, b * s.ny * s.nx, (int)b};
  }
  __device__ __forceinline__ float tau(const GeoPos& p, float tau0, const float* taus) const {
    return taus ? __ldg(taus + p.b) : tau0;
  }
  // address of the node's relaxation time, or NULL for the scalar tau0
  __device__ __forceinline__ const float* tau_ptr(const GeoPos& p, const float* taus) const {
    return taus ? taus + p.b : nullptr;
  }
  __device__ __forceinline__ bool inside(const GeoPos&, int) const { return true; }
  __device__ __forceinline__ float force_x(const GeoPos&) const { return 0.0f; }
};

// A stack of channels (Sec. 3.1): periodic in x, walls halfway beyond the
// first and last rows of every lattice, a body force (fx, 0), or (fxs[b], 0)
// per lattice b when fxs is set.  The network's graph stops at the walls: a
// neighbour x + e_k exists only if its row lies inside the channel.
struct GeoChannel : GeoStack {
  static constexpr bool kWalls = true;
  float fx;
  const float* fxs;
  __device__ __forceinline__ bool inside(const GeoPos& p, int dy) const {
    return (unsigned)(p.y + dy) < (unsigned)p.ny;
  }
  __device__ __forceinline__ float force_x(const GeoPos& p) const {
    return fxs ? __ldg(fxs + p.b) : fx;
  }
};

// One lattice of a batched run: first node in the packed buffers, size and
// relaxation time.
inline GeoStack make_geo_stack(const Shape& s) {
  GeoStack g;
  g.s = s;
  g.dnx = fast_div((uint32_t)s.nx);
  g.dny = fast_div((uint32_t)s.ny);
  g.small = (int64_t)s.nb * s.ny * s.nx < (int64_t(1) << 31);
  return g;
}

struct LatDesc {
  int64_t offset;
  int32_t nx, ny;
  float tau;
  int32_t pad;
};

struct GeoTable {
  static constexpr bool kWalls = false;
  const LatDesc* lat;  // device table, sorted by offset
  int first, n;        // lattices first .. first+n-1 form this range
  int64_t base_, cnt, ps_;
  // optional: hint[g >> 7] = the lattice holding global node (g >> 7) << 7
  const int* hint;
  __device__ __forceinline__ int64_t count() const { return cnt; }
  __device__ __forceinline__ int64_t base() const { return base_; }
  __device__ __forceinline__ int64_t ps() const { return ps_; }
  __device__ __forceinline__ GeoPos pos(int64_t g) const {
    int lo;  // last lattice whose offset <= g
    if (hint) {  // from the lattice of g's 128-node block, forward over the lattices it spans
      lo = max(__ldg(hint + (g >> 7)), first);
      while (lo + 1 < first + n && __ldg(&lat[lo + 1].offset) <= g) ++lo;
    } else {
      lo = first;
      int hi = first + n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&lat[mid].offset) <= g) lo = mid; else hi = mid - 1;
      }
    }
    const int64_t off = __ldg(&lat[lo].offset);
    const int nx = __ldg(&lat[lo].nx), ny = __ldg(&lat[lo].ny);
    const uint32_t r = (uint32_t)(g - off);  // a lattice holds fewer than 2^31 nodes
    const uint32_t y = r / (uint32_t)nx;
    return {(int)(r - y * (uint32_t)nx), (int)y, nx, ny, off, lo};
  }
  __device__ __forceinline__ float tau(const GeoPos& p, float, const float*) const {
    return __ldg(&lat[p.b].tau);
  }
  __device__ __forceinline__ const float* tau_ptr(const GeoPos& p, const float*) const {
    return &lat[p.b].tau;
  }
  __device__ __forceinline__ bool inside(const GeoPos&, int) const { return true; }
  __device__ __forceinline__ float force_x(const GeoPos&) const { return 0.0f; }
};

// The dynamic shared-memory block aligned up to 1024 bytes (the SW128
// operand layouts need it), by pointer arithmetic on the __shared__ array:
// the compiler then still knows the address space and emits shared-memory
// loads and stores rather than generic ones.
__device__ __forceinline__ uint8_t* smem_align1024(uint8_t* raw) {
  return raw + ((1024u - (static_cast<uint32_t>(__cvta_generic_to_shared(raw)) & 1023u)) & 1023u);
}

// Copies `bytes` (multiple of 16) from global to shared memory with all threads.
__device__ __forceinline__ void copy_g2s(void* dst, const void* src, uint32_t bytes) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (uint32_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

// Per-CTA tensor-core context: TMEM base, MMA-completion barrier and phase.
struct TcCtx {
  uint32_t tmem;
  uint64_t* bar;
  uint32_t phase;
};

// ---------------------------------------------------------------------------
// Shared prologue/epilogue of the tensor-core kernels.
struct TcShared {
  uint64_t bar;
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ void tc_setup(TcShared* sh, TcCtx& tc, uint32_t ncols = 256) {
  if (threadIdx.x == 0) {
    mbar_init(&sh->bar, 1);
    sh->abort = 0;
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&sh->tmem, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc.tmem = sh->tmem;
  tc.bar = &sh->bar;
  tc.phase = 0;
}

__device__ __forceinline__ void tc_teardown(TcShared* sh, const TcCtx& tc,
                                            uint32_t ncols = 256) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tc.tmem, ncols);
}

// Issues the MMA chain (thread 0) after all threads wrote their operands,
// then waits for it.  Returns false if the wait gave up (status raised).
template <typename Issue>
__device__ __forceinline__ bool tc_run(TcShared* sh, TcCtx& tc, unsigned* stw, Issue issue) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_fence_after();
    issue();
    umma_commit(tc.bar);
  }
  const bool ok = mbar_wait(tc.bar, tc.phase);
  tc.phase ^= 1u;
  tc_fence_after();
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) raise_status(stw, ST_TIMEOUT);
    return false;
  }
  return true;
}

// ---- thread groups sharing a CTA --------------------------------------------
// A CTA may run NG independent groups of GT threads, each with its own tile,
// shared-memory operands, mbarrier and tensor-memory columns, synchronised by
// named barrier 1 + g (barrier 0 stays __syncthreads).
__device__ __forceinline__ void group_sync(int g, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(nthreads) : "memory");
}
// OR of `v` over the group (also a group barrier).
__device__ __forceinline__ bool group_any(int g, int nthreads, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + g), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Prologue of a CTA of `ng` groups: one mbarrier per group, cols_per_group
// tensor-memory columns per group (allocated together by warp 0).
__device__ __forceinline__ void tc_setup_groups(TcShared* sh, TcCtx& tc, int ng, int g,
                                                uint32_t cols_per_group) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < ng; ++i) {
      mbar_init(&sh[i].bar, 1);
      sh[i].abort = 0;
    }
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&sh[0].tmem, cols_per_group * ng);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc.tmem = sh[0].tmem + (uint32_t)g * cols_per_group;
  tc.bar = &sh[g].bar;
  tc.phase = 0;
}
__device__ __forceinline__ void tc_teardown_groups(TcShared* sh, int ng,
                                                   uint32_t cols_per_group) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(sh[0].tmem, cols_per_group * ng);
}
// tc_run for group g of nthreads threads (its first thread issues).
template <typename Issue>
__device__ __forceinline__ bool tc_run_group(TcCtx& tc, unsigned* stw, int g, int nthreads,
                                             Issue issue) {
  fence_async_smem();
  tc_fence_before();
  group_sync(g, nthreads);
  const bool issuer = (int)threadIdx.x == g * nthreads;
  if (issuer) {
    tc_fence_after();
    issue();
    umma_commit(tc.bar);
  }
  const bool ok = mbar_wait(tc.bar, tc.phase);
  tc.phase ^= 1u;
  tc_fence_after();
  if (group_any(g, nthreads, !ok)) {
    if (issuer) raise_status(stw, ST_TIMEOUT);
    return false;
  }
  return true;
}

// tc_run_group without the OR-barrier after the wait: a wait that gives up
// sets the group's abort word, which the caller tests after its next group
// barrier (every later wait is bounded as well, and all threads keep passing
// the same barriers until then).
template <typename Issue>
__device__ __forceinline__ void tc_run_group_flag(TcCtx& tc, volatile int* abort_word, int g,
                                                  int nthreads, Issue issue) {
  fence_async_smem();
  tc_fence_before();
  group_sync(g, nthreads);
  if ((int)threadIdx.x == g * nthreads) {
    tc_fence_after();
    issue();
    umma_commit(tc.bar);
  }
  if (!mbar_wait(tc.bar, tc.phase)) *abort_word = 1;
  tc.phase ^= 1u;
  tc_fence_after();
}

__device__ __forceinline__ uint32_t lane_base(uint32_t tmem) {
  return tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16);
}

// ---- launch helpers ----------------------------------------------------------
inline int num_sms() {
  static int g_num_sms = 0;
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

inline unsigned grid_for(int64_t N, int per_sm) {
  const int64_t ntiles = (N + TILE - 1) / TILE;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  return (unsigned)(ntiles < cap ? ntiles : cap);
}

template <typename KernelT>
inline cudaError_t set_smem(KernelT k, uint32_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace lbmgnn
