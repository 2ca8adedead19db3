// Internal launchers of the GNN kernels (forward, backward, training).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lbmgnn {

struct RoundLaunch {
  const __nv_bfloat16* h_in = nullptr;
  const __nv_bfloat16* ab_in = nullptr;
  __nv_bfloat16* h_out = nullptr;
  __nv_bfloat16* a_out = nullptr;
  __nv_bfloat16* ab_out = nullptr;
  float* y_out = nullptr;
  const float* f_post = nullptr;
  float* f_out = nullptr;
  float tau = 1.0f;
  const float* taus = nullptr;
  int round = 0;
};

cudaError_t launch_gnn_pack(const float* params, uint8_t* packed, cudaStream_t st);
cudaError_t launch_gnn_encode(const float* f, bool pull, const Shape& s, const uint8_t* packed,
                              __nv_bfloat16* h0, __nv_bfloat16* ab, cudaStream_t st);
// mode 0: inner round; 1: last round + head + Eq. 3 collision; 2: last round + head -> y
cudaError_t launch_gnn_round(int mode, const RoundLaunch& rl, const Shape& s,
                             const uint8_t* packed, cudaStream_t st);

}  // namespace lbmgnn
