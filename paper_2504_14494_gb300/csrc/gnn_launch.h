// Internal launchers of the GNN kernels (forward, backward, training).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lbmgnn {

struct RoundLaunch {
  const __nv_bfloat16* h_in = nullptr;
  const __half* ab_in = nullptr;     // A | B ([N][128]) or B alone ([N][64]), FP16
  bool a_from_h = false;             // ab_in/ab_out hold B alone; A = W_a h recomputed
  __nv_bfloat16* h_out = nullptr;
  __nv_bfloat16* a_out = nullptr;
  __half* ab_out = nullptr;
  float* y_out = nullptr;
  const float* f_post = nullptr;
  float* f_out = nullptr;
  float tau = 1.0f;
  const float* taus = nullptr;
  int round = 0;
  // inference path: h0, read by the last round of the MLP-only network
  // (whose inner round is then skipped); NULL elsewhere
  const __nv_bfloat16* h_skip = nullptr;
};

cudaError_t launch_gnn_pack(const float* params, uint8_t* packed, cudaStream_t st);
// pull: f is a stored state (streamed first); b_only: ab receives B alone.
cudaError_t launch_gnn_encode(const float* f, bool pull, bool b_only, const Shape& s,
                              const uint8_t* packed, __nv_bfloat16* h0, __half* ab,
                              cudaStream_t st);
// mode 0: inner round; 1: last round + head + Eq. 3 collision; 2: last round + head -> y
cudaError_t launch_gnn_round(int mode, const RoundLaunch& rl, const Shape& s,
                             const uint8_t* packed, cudaStream_t st);

// Channel (walls beyond the first and last rows, force (force_x, 0), or
// (forces_x[b], 0) per lattice when forces_x is set): the network forward on
// pre-collision populations over the walled graph.  h0, h1 [N][64] BF16,
// ab0, ab1 [N][128] FP16, y [10][N]; h2, a0, a1 [N][64] BF16: the
// activations the backward reads, or NULL when the forward is for inference.
struct ChannelSaved {
  __nv_bfloat16* h0 = nullptr;
  __half* ab0 = nullptr;
  __nv_bfloat16* h1 = nullptr;
  __half* ab1 = nullptr;
  __nv_bfloat16* h2 = nullptr;
  __nv_bfloat16* a0 = nullptr;
  __nv_bfloat16* a1 = nullptr;
};
cudaError_t launch_gnn_forward_channel(const float* f_pre, const Shape& s, float force_x,
                                       const float* forces_x, const uint8_t* packed,
                                       const ChannelSaved& sv, float* y, cudaStream_t st);
// The channel's pull with bounce-back into f_pre, and Eq. 3 with Guo's
// source (relaxation time tau tau_adj) from the head output y.
cudaError_t launch_channel_pull(const float* fin, float* fpre, const Shape& s, cudaStream_t st);
cudaError_t launch_channel_gnn_collide(const float* fpre, const float* y, float* fout,
                                       const Shape& s, float tau, const float* taus, float gx,
                                       const uint8_t* packed, double* totals, cudaStream_t st);
// Restriction of a refined channel (odd factor m) to the coarse lattice:
// pulls the co-located fine nodes from the fine stored state (the
// pre-collision state of the next fine step), splits off the force part of
// the non-equilibrium populations and rescales the gradient part.
cudaError_t launch_channel_restrict(const float* f_fine, const Shape& fs, float* f_coarse,
                                    const Shape& cs, int m, float tau_f, const float* taus_f,
                                    float tau_c, const float* taus_c, float gx_f,
                                    const float* gxs_f, cudaStream_t st);

// The paper's Fig. 2 network (MLP-only variant) as one fused GNN-LBM step
// kernel (pull, features, 3 MMAs, heads, Eq. 3, store).  For any other
// network the kernel writes nothing (and with require_mlp raises ST_BLOB).
cudaError_t launch_gnn_mlp_step(const float* f_in, float* f_out, const Shape& s, float tau,
                                const float* taus, const uint8_t* packed, bool require_mlp,
                                cudaStream_t st);

struct LatDesc;
// The inference encoder of a message-passing network in the fused kernel's
// design (pull, features, two GELU layers, B = W_b h0; h0 BF16 and B FP16
// [N][64] in the chunked plane layout); returns at once for the MLP-only
// network.  The table form takes the nodes [base, base+count) of the lattices
// first .. first+n-1 of a device descriptor table.
cudaError_t launch_gnn_encode_fused(const float* f_in, const Shape& s, const uint8_t* packed,
                                    __nv_bfloat16* h0, __half* b, cudaStream_t st);
cudaError_t launch_gnn_encode_fused_table(const float* f_in, const LatDesc* lat, int first, int n,
                                          const int* hint, int64_t base, int64_t count, int64_t ps,
                                          const uint8_t* packed, __nv_bfloat16* h0, __half* b,
                                          cudaStream_t st);
cudaError_t launch_gnn_mlp_step_table(const float* f_in, float* f_out, const LatDesc* lat,
                                      int first, int n, const int* hint, int64_t base,
                                      int64_t count, int64_t ps, const uint8_t* packed,
                                      cudaStream_t st, int per_sm);
// GNN-LBM step (encoder, 2 rounds, head + Eq. 3) on the lattices first ..
// first+n-1 of a device descriptor table, whose nodes are [base, base+count)
// of population buffers with plane stride ps; hint: device int per 128-node
// block of the buffers, the lattice holding the block's first node (or
// NULL: binary search); ws: count * 512 bytes; per_sm: resident CTAs per SM
// of the persistent grids.
cudaError_t launch_gnn_step_table(const float* f_in, float* f_out, const LatDesc* lat, int first,
                                  int n, const int* hint, int64_t base, int64_t count, int64_t ps,
                                  const uint8_t* packed, __nv_bfloat16* ws, cudaStream_t st,
                                  int per_sm);

// Rows of per-CTA partial weight gradients (upper bound of the grid of every
// gradient kernel).
constexpr int GRAD_ROWS = 512;

struct BackwardLaunch {
  const float* f_pre = nullptr;            // [9][ps]
  const float* dy = nullptr;               // [10][N]
  const __nv_bfloat16* h0 = nullptr;       // saved activations
  const __nv_bfloat16* h1 = nullptr;
  const __nv_bfloat16* h2 = nullptr;
  const __nv_bfloat16* a0 = nullptr;
  const __nv_bfloat16* a1 = nullptr;
  const __half* ab0 = nullptr;             // FP16 edge terms
  const __half* ab1 = nullptr;
  float* dh[2] = {nullptr, nullptr};       // FP32 [N][64] ping-pong
  float* da = nullptr;                     // FP32 [N][64]
  float* G = nullptr;                      // FP32 [GRAD_ROWS][38922]
  float* grad = nullptr;                   // FP32 [38922]
  float* df = nullptr;                     // optional dL/df_pre [9][ps]
  // channel: the graph stops at the walls and the velocity feature carries
  // the force (fx, or fxs[b] per lattice)
  bool walls = false;
  float fx = 0.0f;
  const float* fxs = nullptr;
  // add the gradient to `grad` instead of overwriting it (rollout steps)
  bool accumulate = false;
};

cudaError_t launch_gnn_backward(const BackwardLaunch& bl, const Shape& s, const uint8_t* packed,
                                cudaStream_t st);
cudaError_t launch_collide_loss(const float* f_pre, const float* y, const float* tgt,
                                const Shape& s, float tau, const float* taus,
                                const uint8_t* packed, double* lossp, int* nblk, float* dy,
                                float* f_pred, cudaStream_t st, const float* lw = nullptr);
// The channel's loss: Eq. 3 with Guo's source for force (gx, 0) (gxs[b] per
// lattice when set) at the network's relaxation time, then Eq. 4.
cudaError_t launch_collide_loss_channel(const float* f_pre, const float* y, const float* tgt,
                                        const Shape& s, float tau, const float* taus, float gx,
                                        const float* gxs, const uint8_t* packed, double* lossp,
                                        int* nblk, float* dy, float* f_pred, cudaStream_t st,
                                        const float* lw = nullptr);
// Per-instance loss weights (weights.cu): w_b = mean_c D_c / D_b with D_b the
// mean squared one-step BGK residual of lattice b against its target.
int64_t pair_weights_ws(const Shape& s);
cudaError_t launch_pair_weights(const float* f_in, const float* tgt, const Shape& s, float tau,
                                const float* taus, float* w, void* ws, cudaStream_t st);
cudaError_t launch_loss_finish(const double* lossp, int nblk, double count, double* loss,
                               cudaStream_t st);
// Rollout loss: reverse mode of Eq. 3 from dL/df* = g_in + scale (f_post -
// tgt) (g_in nullable) to dL/dy [10][N] and the explicit part of dL/df_pre
// (dfd, planes of s.ps); and the adjoint of periodic streaming of a + b.
cudaError_t launch_collide_adjoint(const float* f_pre, const float* y, const float* f_post,
                                   const float* tgt, const float* g_in, const Shape& s, float tau,
                                   const float* taus, const uint8_t* packed, float scale,
                                   float* dy, float* dfd, cudaStream_t st);
cudaError_t launch_stream_adjoint_sum(const float* a, const float* b, float* out, const Shape& s,
                                      cudaStream_t st);
cudaError_t launch_adamw(float* theta, const float* g, float* m, float* v, float lr, float wd,
                         float b1, float b2, float eps, float bc1, float bc2, cudaStream_t st);

}  // namespace lbmgnn
