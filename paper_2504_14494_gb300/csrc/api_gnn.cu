// C ABI entry points of the GNN path (forward).  See include/lbmgnn.h.
#include <cmath>

#include "common.cuh"
#include "gnn.cuh"
#include "gnn_launch.h"
#include "launch.h"
#include "trace.h"

using namespace lbmgnn;

namespace {

int check_shape_g(const lbm_shape& s, Shape* out) {
  if (s.nx < 1 || s.ny < 1 || s.nb < 1) return LBM_ERR_SIZE;
  const int64_t n = (int64_t)s.nx * s.ny * s.nb;
  if (n > (int64_t(1) << 34)) return LBM_ERR_SIZE;
  const int64_t ps = s.plane_stride == 0 ? n : s.plane_stride;
  if (ps < n) return LBM_ERR_SIZE;
  *out = Shape{s.nx, s.ny, s.nb, ps};
  return LBM_OK;
}

int64_t nodes(const Shape& s) { return (int64_t)s.nb * s.ny * s.nx; }

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool overlap(const void* a, int64_t na, const void* b, int64_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

int64_t f_bytes(const Shape& s) { return (8 * s.ps + nodes(s)) * (int64_t)sizeof(float); }

// lbm_step_gnn scratch per node: BF16 h0, h1 and FP16 B0, B1 ([N][64] each).
constexpr int64_t STEP_WS_PER_NODE = 512;

// lbm_step_gnn_channel scratch: f_pre (rounded up to 256 bytes), then per
// node BF16 h0 [64], FP16 AB0 [128], BF16 h1 [64], FP16 AB1 [128], FP32 y [10].
int64_t channel_ws_bytes(const Shape& s) {
  return ((f_bytes(s) + 255) / 256) * 256 + nodes(s) * (128 + 256 + 128 + 256 + 40);
}

}  // namespace

extern "C" {

size_t gnn_param_count(void) { return P::TOTAL; }

int gnn_params_init_xavier(float* params, uint64_t seed, float s_df, int variant) {
  if (!params || !std::isfinite(s_df) || !(s_df > 0.0f) || variant < 0 || variant > VAR_ALL)
    return LBM_ERR_ARG;
  uint64_t state = seed;
  auto uniform = [&state]() {  // SplitMix64 (Steele, Lea and Flood 2014), top 24 bits
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 40) * (1.0 / 16777216.0);  // [0, 1)
  };
  auto matrix = [&](int off, int rows, int cols) {
    const double b = std::sqrt(6.0 / (double)(rows + cols));
    for (int i = 0; i < rows * cols; ++i) params[off + i] = (float)((2.0 * uniform() - 1.0) * b);
  };
  auto zeros = [&](int off, int n) {
    for (int i = 0; i < n; ++i) params[off + i] = 0.0f;
  };
  matrix(P::ENC1_W, HID, NFEAT);
  zeros(P::ENC1_B, HID);
  matrix(P::ENC2_W, HID, HID);
  zeros(P::ENC2_B, HID);
  for (int r = 0; r < 2; ++r) {
    const int base = P::ROUND0 + r * P::ROUND_SIZE;
    matrix(base + P::EDGE_W, HID, 2 * HID + 2);
    zeros(base + P::EDGE_B, HID);
    matrix(base + P::NODE_W, HID, 2 * HID);
    zeros(base + P::NODE_B, HID);
  }
  matrix(P::HEAD_W, NOUT, HID);
  zeros(P::HEAD_B, NOUT);
  const float rest[Q] = {4.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9,
                         1.0f / 36, 1.0f / 36, 1.0f / 36, 1.0f / 36};
  for (int q = 0; q < Q; ++q) {
    params[P::MU + q] = rest[q];
    params[P::SIGMA + q] = 0.1f * rest[q];
  }
  params[P::MU + 9] = 1.0f;
  params[P::MU + 10] = params[P::MU + 11] = 0.0f;
  params[P::SIGMA + 9] = params[P::SIGMA + 10] = params[P::SIGMA + 11] = 0.01f;
  params[P::S_DF] = s_df;
  params[P::VARIANT] = (float)variant;
  return LBM_OK;
}
size_t gnn_trainable_count(void) { return P::TRAINABLE; }
size_t gnn_packed_bytes(void) { return K::TOTAL; }

int gnn_pack(const float* params, void* packed, void* stream) {
  LBM_TRACE("gnn_pack");
  if (!params || !packed) return LBM_ERR_ARG;
  if (!aligned(packed, 16)) return LBM_ERR_ARG;
  if (cudaMemsetAsync(packed, 0, K::TOTAL, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return LBM_ERR_CUDA;
  return launch_gnn_pack(params, static_cast<uint8_t*>(packed),
                         static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

size_t gnn_step_workspace_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape_g(shape, &s)) return 0;
  return (size_t)nodes(s) * STEP_WS_PER_NODE;
}

int lbm_step_gnn(const float* f_in, float* f_out, lbm_shape shape, float tau, const float* taus,
                 const void* packed, double* totals, void* workspace, size_t ws_bytes,
                 void* stream) {
  LBM_TRACE("lbm_step_gnn");
  Shape s;
  if (!f_in || !f_out || !packed) return LBM_ERR_ARG;
  if (int r = check_shape_g(shape, &s)) return r;
  if (!taus && (!std::isfinite(tau) || !(tau > 0.5f))) return LBM_ERR_TAU;
  if (!aligned(packed, 16)) return LBM_ERR_ARG;
  const int64_t N = nodes(s);
  const int64_t wsb = N * STEP_WS_PER_NODE;
  if (!workspace || (int64_t)ws_bytes < wsb) return LBM_ERR_WORKSPACE;
  if (!aligned(workspace, 16)) return LBM_ERR_WORKSPACE;
  if (overlap(f_in, f_bytes(s), f_out, f_bytes(s))) return LBM_ERR_ALIAS;
  if (overlap(workspace, wsb, f_in, f_bytes(s)) || overlap(workspace, wsb, f_out, f_bytes(s)))
    return LBM_ERR_ALIAS;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint8_t* pk = static_cast<const uint8_t*>(packed);
  auto* ws = static_cast<__nv_bfloat16*>(workspace);
  // Between the kernels only h and B = W_b h travel through HBM; each round
  // recomputes its A = W_a h from h.
  __nv_bfloat16* h0 = ws;
  __half* b0 = reinterpret_cast<__half*>(h0 + N * 64);
  __nv_bfloat16* h1 = reinterpret_cast<__nv_bfloat16*>(b0 + N * 64);
  __half* b1 = reinterpret_cast<__half*>(h1 + N * 64);
  // The paper's Fig. 2 network (MLP-only variant, read from the image on the
  // device) is stepped by one fused kernel; for it the three kernels below
  // return at once, for every other network the fused kernel does.
  if (launch_gnn_mlp_step(f_in, f_out, s, tau, taus, pk, false, st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (launch_gnn_encode_fused(f_in, s, pk, h0, b0, st) != cudaSuccess) return LBM_ERR_CUDA;
  RoundLaunch r0;
  r0.h_in = h0;
  r0.ab_in = b0;
  r0.a_from_h = true;
  r0.h_skip = h0;
  r0.h_out = h1;
  r0.ab_out = b1;
  r0.round = 0;
  if (launch_gnn_round(0, r0, s, pk, st) != cudaSuccess) return LBM_ERR_CUDA;
  RoundLaunch r1;
  r1.h_in = h1;
  r1.ab_in = b1;
  r1.a_from_h = true;
  r1.h_skip = h0;
  r1.f_post = f_in;
  r1.f_out = f_out;
  r1.tau = tau;
  r1.taus = taus;
  r1.round = 1;
  if (launch_gnn_round(1, r1, s, pk, st) != cudaSuccess) return LBM_ERR_CUDA;
  if (totals) {
    if (cudaMemsetAsync(totals, 0, 5 * sizeof(double), st) != cudaSuccess) return LBM_ERR_CUDA;
    if (launch_moments(f_out, s, nullptr, nullptr, nullptr, totals, st) != cudaSuccess)
      return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

int lbm_step_gnn_mlp(const float* f_in, float* f_out, lbm_shape shape, float tau,
                     const float* taus, const void* packed, double* totals, void* stream) {
  LBM_TRACE("lbm_step_gnn_mlp");
  Shape s;
  if (!f_in || !f_out || !packed) return LBM_ERR_ARG;
  if (int r = check_shape_g(shape, &s)) return r;
  if (!taus && (!std::isfinite(tau) || !(tau > 0.5f))) return LBM_ERR_TAU;
  if (!aligned(packed, 16)) return LBM_ERR_ARG;
  if (overlap(f_in, f_bytes(s), f_out, f_bytes(s))) return LBM_ERR_ALIAS;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (launch_gnn_mlp_step(f_in, f_out, s, tau, taus, static_cast<const uint8_t*>(packed), true,
                          st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (totals) {
    if (cudaMemsetAsync(totals, 0, 5 * sizeof(double), st) != cudaSuccess) return LBM_ERR_CUDA;
    if (launch_moments(f_out, s, nullptr, nullptr, nullptr, totals, st) != cudaSuccess)
      return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

size_t gnn_channel_workspace_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape_g(shape, &s)) return 0;
  return (size_t)channel_ws_bytes(s);
}

int lbm_step_gnn_channel(const float* f_in, float* f_out, lbm_shape shape, float tau,
                         const float* taus, float force_x, const void* packed, double* totals,
                         void* workspace, size_t ws_bytes, void* stream) {
  LBM_TRACE("lbm_step_gnn_channel");
  Shape s;
  if (!f_in || !f_out || !packed || !std::isfinite(force_x)) return LBM_ERR_ARG;
  if (int r = check_shape_g(shape, &s)) return r;
  if (!taus && (!std::isfinite(tau) || !(tau > 0.5f))) return LBM_ERR_TAU;
  if (!aligned(packed, 16)) return LBM_ERR_ARG;
  const int64_t N = nodes(s), wsb = channel_ws_bytes(s);
  if (!workspace || (int64_t)ws_bytes < wsb || !aligned(workspace, 256)) return LBM_ERR_WORKSPACE;
  if (overlap(f_in, f_bytes(s), f_out, f_bytes(s))) return LBM_ERR_ALIAS;
  if (overlap(workspace, wsb, f_in, f_bytes(s)) || overlap(workspace, wsb, f_out, f_bytes(s)))
    return LBM_ERR_ALIAS;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint8_t* pk = static_cast<const uint8_t*>(packed);
  char* w = static_cast<char*>(workspace);
  float* f_pre = reinterpret_cast<float*>(w);
  w += ((f_bytes(s) + 255) / 256) * 256;
  auto* h0 = reinterpret_cast<__nv_bfloat16*>(w);
  auto* ab0 = reinterpret_cast<__half*>(w + N * 128);
  auto* h1 = reinterpret_cast<__nv_bfloat16*>(w + N * 384);
  auto* ab1 = reinterpret_cast<__half*>(w + N * 512);
  auto* y = reinterpret_cast<float*>(w + N * 768);
  if (totals && cudaMemsetAsync(totals, 0, 5 * sizeof(double), st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (launch_channel_pull(f_in, f_pre, s, st) != cudaSuccess) return LBM_ERR_CUDA;
  ChannelSaved sv;
  sv.h0 = h0;
  sv.ab0 = ab0;
  sv.h1 = h1;
  sv.ab1 = ab1;
  if (launch_gnn_forward_channel(f_pre, s, force_x, nullptr, pk, sv, y, st) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (launch_channel_gnn_collide(f_pre, y, f_out, s, tau, taus, force_x, pk, totals, st) !=
      cudaSuccess)
    return LBM_ERR_CUDA;
  return LBM_OK;
}

size_t gnn_saved_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape_g(shape, &s)) return 0;
  return (size_t)nodes(s) * 1152;
}

int gnn_forward(const float* f_pre, lbm_shape shape, const void* packed, void* saved, float* y,
                void* stream) {
  LBM_TRACE("gnn_forward");
  Shape s;
  if (!f_pre || !packed || !saved || !y) return LBM_ERR_ARG;
  if (int r = check_shape_g(shape, &s)) return r;
  if (!aligned(packed, 16) || !aligned(saved, 16)) return LBM_ERR_ARG;
  const int64_t N = nodes(s);
  if (overlap(saved, N * 1152, f_pre, f_bytes(s)) || overlap(y, N * 40, f_pre, f_bytes(s)) ||
      overlap(saved, N * 1152, y, N * 40))
    return LBM_ERR_ALIAS;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint8_t* pk = static_cast<const uint8_t*>(packed);
  auto* sv = static_cast<__nv_bfloat16*>(saved);
  __nv_bfloat16* h0 = sv;
  __nv_bfloat16* h1 = h0 + N * 64;
  __nv_bfloat16* h2 = h1 + N * 64;
  __nv_bfloat16* a0 = h2 + N * 64;
  __nv_bfloat16* a1 = a0 + N * 64;
  __half* ab0 = reinterpret_cast<__half*>(a1 + N * 64);
  __half* ab1 = ab0 + N * 128;
  if (launch_gnn_encode(f_pre, false, false, s, pk, h0, ab0, st) != cudaSuccess)
    return LBM_ERR_CUDA;
  RoundLaunch r0;
  r0.h_in = h0;
  r0.ab_in = ab0;
  r0.h_out = h1;
  r0.a_out = a0;
  r0.ab_out = ab1;
  r0.round = 0;
  if (launch_gnn_round(0, r0, s, pk, st) != cudaSuccess) return LBM_ERR_CUDA;
  RoundLaunch r1;
  r1.h_in = h1;
  r1.ab_in = ab1;
  r1.h_out = h2;
  r1.a_out = a1;
  r1.y_out = y;
  r1.round = 1;
  if (launch_gnn_round(2, r1, s, pk, st) != cudaSuccess) return LBM_ERR_CUDA;
  return LBM_OK;
}

}  // extern "C"
