// C ABI entry points of the training side and the auxiliary lattice
// operations (streaming only, restriction, per-lattice TGV initial states).
// See include/lbmgnn.h.
#include <cmath>

#include "common.cuh"
#include "gnn.cuh"
#include "gnn_launch.h"
#include "launch.h"
#include "trace.h"

using namespace lbmgnn;

namespace {

int check_shape_t(const lbm_shape& s, Shape* out) {
  if (s.nx < 1 || s.ny < 1 || s.nb < 1) return LBM_ERR_SIZE;
  const int64_t n = (int64_t)s.nx * s.ny * s.nb;
  if (n > (int64_t(1) << 34)) return LBM_ERR_SIZE;
  const int64_t ps = s.plane_stride == 0 ? n : s.plane_stride;
  if (ps < n) return LBM_ERR_SIZE;
  *out = Shape{s.nx, s.ny, s.nb, ps};
  return LBM_OK;
}

int64_t nodes(const Shape& s) { return (int64_t)s.nb * s.ny * s.nx; }
int64_t up16(int64_t b) { return (b + 15) & ~int64_t(15); }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
int64_t f_bytes(const Shape& s) { return (8 * s.ps + nodes(s)) * (int64_t)sizeof(float); }
bool overlap(const void* a, int64_t na, const void* b, int64_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

constexpr int64_t G_BYTES = (int64_t)GRAD_ROWS * P::TRAINABLE * sizeof(float);
int64_t loss_blocks(int64_t N) { return (N + 255) / 256; }
int64_t bwd_ws(int64_t N) { return G_BYTES + 3 * N * HID * (int64_t)sizeof(float); }
int64_t loss_ws(int64_t N) { return up16(loss_blocks(N) * (int64_t)sizeof(double)); }
// f_pre | saved | y | dy | loss partials | backward workspace | gradients
int64_t train_ws(const Shape& s) {
  const int64_t N = nodes(s);
  return up16(9 * s.ps * (int64_t)sizeof(float)) + N * 1152 + up16(N * 40) * 2 + loss_ws(N) +
         bwd_ws(N) + up16(P::TRAINABLE * (int64_t)sizeof(float));
}

// K-step rollout: per step f_pre, f_post (9 planes of ps), saved
// activations, y; then dy, g, dfd, dfn, the loss partials of all K steps,
// the backward workspace and the gradient.
int64_t rollout_ws(const Shape& s, int K) {
  const int64_t N = nodes(s), fp = up16(9 * s.ps * (int64_t)sizeof(float));
  return K * (2 * fp + N * 1152 + up16(N * 40)) + up16(N * 40) + 3 * fp +
         up16(K * loss_blocks(N) * (int64_t)sizeof(double)) + bwd_ws(N) +
         up16(P::TRAINABLE * (int64_t)sizeof(float));
}

// Carves the backward workspace.
void carve_bwd(uint8_t* ws, int64_t N, BackwardLaunch& bl) {
  bl.G = reinterpret_cast<float*>(ws);
  float* p = reinterpret_cast<float*>(ws + G_BYTES);
  bl.dh[0] = p;
  bl.dh[1] = p + N * HID;
  bl.da = p + 2 * N * HID;
}

void set_saved(const void* saved, int64_t N, BackwardLaunch& bl) {
  auto* sv = static_cast<const __nv_bfloat16*>(saved);
  bl.h0 = sv;
  bl.h1 = sv + N * 64;
  bl.h2 = sv + 2 * N * 64;
  bl.a0 = sv + 3 * N * 64;
  bl.a1 = sv + 4 * N * 64;
  bl.ab0 = reinterpret_cast<const __half*>(sv + 5 * N * 64);
  bl.ab1 = reinterpret_cast<const __half*>(sv + 5 * N * 64 + N * 128);
}

}  // namespace

extern "C" {

int lbm_stream(const float* f_in, float* f_out, lbm_shape shape, void* stream) {
  LBM_TRACE("lbm_stream");
  Shape s;
  if (!f_in || !f_out) return LBM_ERR_ARG;
  if (int r = check_shape_t(shape, &s)) return r;
  if (overlap(f_in, f_bytes(s), f_out, f_bytes(s))) return LBM_ERR_ALIAS;
  return launch_stream(f_in, f_out, s, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

int lbm_init_tgv_batch(float* f, lbm_shape shape, const double* params, int pressure_consistent,
                       void* stream) {
  LBM_TRACE("lbm_init_tgv_batch");
  Shape s;
  if (!f || !params) return LBM_ERR_ARG;
  if (int r = check_shape_t(shape, &s)) return r;
  return launch_tgv_init_batch(f, s, params, pressure_consistent ? 1 : 0,
                               static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

int lbm_restrict(const float* f_fine, lbm_shape fine, float* f_coarse, lbm_shape coarse,
                 int factor, float tau_f, const float* taus_f, float tau_c, const float* taus_c,
                 void* stream) {
  LBM_TRACE("lbm_restrict");
  Shape fs, cs;
  if (!f_fine || !f_coarse || factor < 1) return LBM_ERR_ARG;
  if (int r = check_shape_t(fine, &fs)) return r;
  if (int r = check_shape_t(coarse, &cs)) return r;
  if (fs.nb != cs.nb || (int64_t)fs.nx != (int64_t)factor * cs.nx ||
      (int64_t)fs.ny != (int64_t)factor * cs.ny)
    return LBM_ERR_SIZE;
  if (!taus_f && (!std::isfinite(tau_f) || !(tau_f > 0.5f))) return LBM_ERR_TAU;
  if (!taus_c && (!std::isfinite(tau_c) || !(tau_c > 0.5f))) return LBM_ERR_TAU;
  if (overlap(f_fine, f_bytes(fs), f_coarse, f_bytes(cs))) return LBM_ERR_ALIAS;
  return launch_restrict(f_fine, fs, f_coarse, cs, factor, tau_f, taus_f, tau_c, taus_c,
                         static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

size_t gnn_loss_workspace_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape_t(shape, &s)) return 0;
  return (size_t)loss_ws(nodes(s));
}

int gnn_collide_loss(const float* f_pre, const float* y, const float* f_target, lbm_shape shape,
                     float tau, const float* taus, const void* packed, double* loss, float* dy,
                     float* f_pred, void* workspace, size_t ws_bytes, void* stream) {
  LBM_TRACE("gnn_collide_loss");
  Shape s;
  if (!f_pre || !y || !f_target || !packed || !loss) return LBM_ERR_ARG;
  if (int r = check_shape_t(shape, &s)) return r;
  if (!taus && (!std::isfinite(tau) || !(tau > 0.5f))) return LBM_ERR_TAU;
  const int64_t N = nodes(s);
  if (!workspace || (int64_t)ws_bytes < loss_ws(N) || !aligned16(workspace))
    return LBM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int nblk = 0;
  auto* lossp = static_cast<double*>(workspace);
  if (launch_collide_loss(f_pre, y, f_target, s, tau, taus, static_cast<const uint8_t*>(packed),
                          lossp, &nblk, dy, f_pred, st) != cudaSuccess)
    return LBM_ERR_CUDA;
  return launch_loss_finish(lossp, nblk, 9.0 * (double)N, loss, st) == cudaSuccess ? LBM_OK
                                                                                   : LBM_ERR_CUDA;
}

size_t gnn_backward_workspace_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape_t(shape, &s)) return 0;
  return (size_t)bwd_ws(nodes(s));
}

int gnn_backward(const float* f_pre, lbm_shape shape, const void* packed, const void* saved,
                 const float* dy, float* dparams, float* df_pre, void* workspace, size_t ws_bytes,
                 void* stream) {
  LBM_TRACE("gnn_backward");
  Shape s;
  if (!f_pre || !packed || !saved || !dy || !dparams) return LBM_ERR_ARG;
  if (int r = check_shape_t(shape, &s)) return r;
  if (!aligned16(packed) || !aligned16(saved) || !aligned16(dy)) return LBM_ERR_ARG;
  const int64_t N = nodes(s);
  if (!workspace || (int64_t)ws_bytes < bwd_ws(N) || !aligned16(workspace))
    return LBM_ERR_WORKSPACE;
  if (df_pre && overlap(df_pre, f_bytes(s), f_pre, f_bytes(s))) return LBM_ERR_ALIAS;
  BackwardLaunch bl;
  bl.f_pre = f_pre;
  bl.dy = dy;
  set_saved(saved, N, bl);
  carve_bwd(static_cast<uint8_t*>(workspace), N, bl);
  bl.grad = dparams;
  bl.df = df_pre;
  return launch_gnn_backward(bl, s, static_cast<const uint8_t*>(packed),
                             static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

int gnn_adamw(float* params, const float* grads, float* m, float* v, int64_t step, float lr,
              float wd, float beta1, float beta2, float eps, void* stream) {
  LBM_TRACE("gnn_adamw");
  if (!params || !grads || !m || !v || step < 1) return LBM_ERR_ARG;
  if (!(lr >= 0.0f) || !(wd >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return LBM_ERR_ARG;
  const double bc1 = 1.0 / (1.0 - std::pow((double)beta1, (double)step));
  const double bc2 = 1.0 / (1.0 - std::pow((double)beta2, (double)step));
  return launch_adamw(params, grads, m, v, lr, wd, beta1, beta2, eps, (float)bc1, (float)bc2,
                      static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

size_t gnn_train_workspace_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape_t(shape, &s)) return 0;
  return (size_t)train_ws(s);
}

}  // extern "C"

namespace {
// The channel's force of a training step: (fx, 0), or (fxs[b], 0) per lattice.
struct ChannelForce {
  float fx;
  const float* fxs;
};

// The fused training step; lw: per-lattice loss weights or NULL (Eq. 4); ch:
// the channel (walled graph, Guo forcing) or NULL (periodic lattices).
int train_step(const float* f_in, const float* f_target, lbm_shape shape, float tau,
               const float* taus, const float* lw, float* params, void* packed, float* adam_m,
               float* adam_v, int64_t step, float lr, float wd, double* loss, float* grads,
               void* workspace, size_t ws_bytes, void* stream, const ChannelForce* ch = nullptr) {
  Shape s;
  if (!f_in || !f_target || !params || !packed || !adam_m || !adam_v || !loss || step < 1)
    return LBM_ERR_ARG;
  if (int r = check_shape_t(shape, &s)) return r;
  if (!taus && (!std::isfinite(tau) || !(tau > 0.5f))) return LBM_ERR_TAU;
  if (ch && !ch->fxs && !std::isfinite(ch->fx)) return LBM_ERR_ARG;
  if (!aligned16(packed)) return LBM_ERR_ARG;
  const int64_t N = nodes(s);
  if (!workspace || (int64_t)ws_bytes < train_ws(s) || !aligned16(workspace))
    return LBM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* pk = static_cast<uint8_t*>(packed);
  uint8_t* w = static_cast<uint8_t*>(workspace);
  float* f_pre = reinterpret_cast<float*>(w);
  w += up16(9 * s.ps * (int64_t)sizeof(float));
  void* saved = w;
  w += N * 1152;
  float* y = reinterpret_cast<float*>(w);
  w += up16(N * 40);
  float* dy = reinterpret_cast<float*>(w);
  w += up16(N * 40);
  double* lossp = reinterpret_cast<double*>(w);
  w += loss_ws(N);
  uint8_t* bws = w;
  w += bwd_ws(N);
  float* g = grads ? grads : reinterpret_cast<float*>(w);

  int nblk = 0;
  if (!ch) {
    if (launch_stream(f_in, f_pre, s, st) != cudaSuccess) return LBM_ERR_CUDA;
    if (int r = gnn_forward(f_pre, shape, packed, saved, y, stream)) return r;
    if (launch_collide_loss(f_pre, y, f_target, s, tau, taus, pk, lossp, &nblk, dy, nullptr, st,
                            lw) != cudaSuccess)
      return LBM_ERR_CUDA;
  } else {
    // the saved activations in gnn_forward's layout (set_saved)
    auto* sb = static_cast<__nv_bfloat16*>(saved);
    ChannelSaved sv;
    sv.h0 = sb;
    sv.h1 = sb + N * 64;
    sv.h2 = sb + 2 * N * 64;
    sv.a0 = sb + 3 * N * 64;
    sv.a1 = sb + 4 * N * 64;
    sv.ab0 = reinterpret_cast<__half*>(sb + 5 * N * 64);
    sv.ab1 = sv.ab0 + N * 128;
    if (launch_channel_pull(f_in, f_pre, s, st) != cudaSuccess) return LBM_ERR_CUDA;
    if (launch_gnn_forward_channel(f_pre, s, ch->fx, ch->fxs, pk, sv, y, st) != cudaSuccess)
      return LBM_ERR_CUDA;
    if (launch_collide_loss_channel(f_pre, y, f_target, s, tau, taus, ch->fx, ch->fxs, pk, lossp,
                                    &nblk, dy, nullptr, st, lw) != cudaSuccess)
      return LBM_ERR_CUDA;
  }
  if (launch_loss_finish(lossp, nblk, 9.0 * (double)N, loss, st) != cudaSuccess)
    return LBM_ERR_CUDA;
  BackwardLaunch bl;
  bl.f_pre = f_pre;
  bl.dy = dy;
  set_saved(saved, N, bl);
  carve_bwd(bws, N, bl);
  bl.grad = g;
  if (ch) {
    bl.walls = true;
    bl.fx = ch->fx;
    bl.fxs = ch->fxs;
  }
  if (launch_gnn_backward(bl, s, pk, st) != cudaSuccess) return LBM_ERR_CUDA;
  if (int r = gnn_adamw(params, g, adam_m, adam_v, step, lr, wd, 0.9f, 0.999f, 1e-8f, stream))
    return r;
  return gnn_pack(params, packed, stream);
}
}  // namespace

extern "C" {

int gnn_train_step(const float* f_in, const float* f_target, lbm_shape shape, float tau,
                   const float* taus, float* params, void* packed, float* adam_m, float* adam_v,
                   int64_t step, float lr, float wd, double* loss, float* grads, void* workspace,
                   size_t ws_bytes, void* stream) {
  LBM_TRACE("gnn_train_step");
  return train_step(f_in, f_target, shape, tau, taus, nullptr, params, packed, adam_m, adam_v,
                    step, lr, wd, loss, grads, workspace, ws_bytes, stream);
}

int gnn_train_step_weighted(const float* f_in, const float* f_target, lbm_shape shape, float tau,
                            const float* taus, const float* lat_weights, float* params,
                            void* packed, float* adam_m, float* adam_v, int64_t step, float lr,
                            float wd, double* loss, float* grads, void* workspace,
                            size_t ws_bytes, void* stream) {
  LBM_TRACE("gnn_train_step_weighted");
  if (!lat_weights) return LBM_ERR_ARG;
  return train_step(f_in, f_target, shape, tau, taus, lat_weights, params, packed, adam_m,
                    adam_v, step, lr, wd, loss, grads, workspace, ws_bytes, stream);
}

int gnn_train_step_channel(const float* f_in, const float* f_target, lbm_shape shape, float tau,
                           const float* taus, float force_x, const float* forces_x,
                           const float* lat_weights, float* params, void* packed, float* adam_m,
                           float* adam_v, int64_t step, float lr, float wd, double* loss,
                           float* grads, void* workspace, size_t ws_bytes, void* stream) {
  LBM_TRACE("gnn_train_step_channel");
  const ChannelForce ch{force_x, forces_x};
  return train_step(f_in, f_target, shape, tau, taus, lat_weights, params, packed, adam_m, adam_v,
                    step, lr, wd, loss, grads, workspace, ws_bytes, stream, &ch);
}

int lbm_restrict_channel(const float* f_fine, lbm_shape fine, float* f_coarse, lbm_shape coarse,
                         int factor, float tau_f, const float* taus_f, float tau_c,
                         const float* taus_c, float force_x_f, const float* forces_x_f,
                         void* stream) {
  LBM_TRACE("lbm_restrict_channel");
  Shape fs, cs;
  if (!f_fine || !f_coarse || factor < 1 || factor % 2 == 0) return LBM_ERR_ARG;
  if (!forces_x_f && !std::isfinite(force_x_f)) return LBM_ERR_ARG;
  if (int r = check_shape_t(fine, &fs)) return r;
  if (int r = check_shape_t(coarse, &cs)) return r;
  if (fs.nb != cs.nb || (int64_t)fs.nx != (int64_t)factor * cs.nx ||
      (int64_t)fs.ny != (int64_t)factor * cs.ny)
    return LBM_ERR_SIZE;
  if (!taus_f && (!std::isfinite(tau_f) || !(tau_f > 0.5f))) return LBM_ERR_TAU;
  if (!taus_c && (!std::isfinite(tau_c) || !(tau_c > 0.5f))) return LBM_ERR_TAU;
  if (overlap(f_fine, f_bytes(fs), f_coarse, f_bytes(cs))) return LBM_ERR_ALIAS;
  return launch_channel_restrict(f_fine, fs, f_coarse, cs, factor, tau_f, taus_f, tau_c, taus_c,
                                 force_x_f, forces_x_f, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

size_t gnn_rollout_workspace_bytes(lbm_shape shape, int K) {
  Shape s;
  if (K < 1 || K > 64 || check_shape_t(shape, &s)) return 0;
  return (size_t)rollout_ws(s, K);
}

int gnn_train_step_rollout(const float* f_in, const float* f_targets, int K, lbm_shape shape,
                           float tau, const float* taus, float* params, void* packed,
                           float* adam_m, float* adam_v, int64_t step, float lr, float wd,
                           double* loss, float* grads, void* workspace, size_t ws_bytes,
                           void* stream) {
  LBM_TRACE("gnn_train_step_rollout");
  Shape s;
  if (!f_in || !f_targets || !params || !packed || !adam_m || !adam_v || !loss || step < 1 ||
      K < 1 || K > 64)
    return LBM_ERR_ARG;
  if (int r = check_shape_t(shape, &s)) return r;
  if (!taus && (!std::isfinite(tau) || !(tau > 0.5f))) return LBM_ERR_TAU;
  if (!aligned16(packed)) return LBM_ERR_ARG;
  const int64_t N = nodes(s);
  if (!workspace || (int64_t)ws_bytes < rollout_ws(s, K) || !aligned16(workspace))
    return LBM_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* pk = static_cast<uint8_t*>(packed);
  const int64_t fp = up16(9 * s.ps * (int64_t)sizeof(float));
  uint8_t* w = static_cast<uint8_t*>(workspace);
  auto take = [&w](int64_t bytes) {
    uint8_t* p = w;
    w += bytes;
    return p;
  };
  float* fpre[64];
  float* fpost[64];
  void* saved[64];
  float* y[64];
  for (int k = 0; k < K; ++k) {
    fpre[k] = reinterpret_cast<float*>(take(fp));
    fpost[k] = reinterpret_cast<float*>(take(fp));
    saved[k] = take(N * 1152);
    y[k] = reinterpret_cast<float*>(take(up16(N * 40)));
  }
  float* dy = reinterpret_cast<float*>(take(up16(N * 40)));
  float* g = reinterpret_cast<float*>(take(fp));
  float* dfd = reinterpret_cast<float*>(take(fp));
  float* dfn = reinterpret_cast<float*>(take(fp));
  const int nblk = (int)loss_blocks(N);
  auto* lossp = reinterpret_cast<double*>(take(up16(K * nblk * (int64_t)sizeof(double))));
  uint8_t* bws = take(bwd_ws(N));
  float* gr = grads ? grads : reinterpret_cast<float*>(take(up16(P::TRAINABLE * sizeof(float))));
  const float* tgt[64];
  for (int k = 0; k < K; ++k) tgt[k] = f_targets + (int64_t)k * 9 * s.ps;

  // forward: K GNN-LBM steps, each with its Eq. 4 partial sums
  const float* src = f_in;
  for (int k = 0; k < K; ++k) {
    if (launch_stream(src, fpre[k], s, st) != cudaSuccess) return LBM_ERR_CUDA;
    if (int r = gnn_forward(fpre[k], shape, packed, saved[k], y[k], stream)) return r;
    int nb = 0;
    if (launch_collide_loss(fpre[k], y[k], tgt[k], s, tau, taus, pk, lossp + k * nblk, &nb,
                            nullptr, fpost[k], st) != cudaSuccess)
      return LBM_ERR_CUDA;
    src = fpost[k];
  }
  if (launch_loss_finish(lossp, K * nblk, 9.0 * (double)N * K, loss, st) != cudaSuccess)
    return LBM_ERR_CUDA;
  // reverse: step K first; g carries dL/df* of the step being reversed
  const float scale = (float)(2.0 / (9.0 * (double)N * K));
  for (int k = K - 1; k >= 0; --k) {
    if (launch_collide_adjoint(fpre[k], y[k], fpost[k], tgt[k], k == K - 1 ? nullptr : g, s, tau,
                               taus, pk, scale, dy, dfd, st) != cudaSuccess)
      return LBM_ERR_CUDA;
    BackwardLaunch bl;
    bl.f_pre = fpre[k];
    bl.dy = dy;
    set_saved(saved[k], N, bl);
    carve_bwd(bws, N, bl);
    bl.grad = gr;
    bl.df = k > 0 ? dfn : nullptr;
    bl.accumulate = k != K - 1;
    if (launch_gnn_backward(bl, s, pk, st) != cudaSuccess) return LBM_ERR_CUDA;
    if (k > 0 && launch_stream_adjoint_sum(dfd, dfn, g, s, st) != cudaSuccess)
      return LBM_ERR_CUDA;
  }
  if (int r = gnn_adamw(params, gr, adam_m, adam_v, step, lr, wd, 0.9f, 0.999f, 1e-8f, stream))
    return r;
  return gnn_pack(params, packed, stream);
}

size_t lbm_pair_weights_workspace_bytes(lbm_shape shape) {
  Shape s;
  if (check_shape_t(shape, &s)) return 0;
  return (size_t)pair_weights_ws(s);
}

int lbm_pair_weights(const float* f_in, const float* f_target, lbm_shape shape, float tau,
                     const float* taus, float* weights, void* workspace, size_t ws_bytes,
                     void* stream) {
  LBM_TRACE("lbm_pair_weights");
  Shape s;
  if (!f_in || !f_target || !weights) return LBM_ERR_ARG;
  if (int r = check_shape_t(shape, &s)) return r;
  if (s.nb > 65535) return LBM_ERR_SIZE;
  if (!taus && (!std::isfinite(tau) || !(tau > 0.5f))) return LBM_ERR_TAU;
  if (!workspace || (int64_t)ws_bytes < pair_weights_ws(s) || !aligned16(workspace))
    return LBM_ERR_WORKSPACE;
  return launch_pair_weights(f_in, f_target, s, tau, taus, weights, workspace,
                             static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBM_OK
             : LBM_ERR_CUDA;
}

}  // extern "C"
