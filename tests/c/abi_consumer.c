/* A plain C consumer of liblbmgnn.so through include/lbmgnn.h, with no
 * Python in the process: shows that the C ABI is usable as declared.
 *
 *   abi_consumer host          host-only calls (no GPU needed): status
 *                              strings, sizes, the Xavier starting parameters
 *   abi_consumer gpu OUT.bin   on the current CUDA device: a Taylor-Green
 *                              stack of 2 lattices of 24 x 20 nodes (Sec. 3.2),
 *                              7 BGK steps with totals (Eq. 1-2), then one
 *                              GNN-LBM step (Eq. 3) with the Xavier
 *                              parameters (seed 5, s_df 1e-2); OUT.bin gets
 *                              the BGK state (FP32 [9][N]), its totals (FP64
 *                              [5]) and the GNN-LBM state (FP32 [9][N])
 *
 * Prints one JSON line on stdout.  Exit status 0 when every call returned
 * LBM_OK, 1 otherwise (the failing call is named on stderr). */
#include <cuda_runtime_api.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lbmgnn.h"

#define CHECK(call)                                                              \
  do {                                                                           \
    int rc_ = (int)(call);                                                       \
    if (rc_ != 0) {                                                              \
      fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, lbm_status_string(rc_)); \
      return 1;                                                                  \
    }                                                                            \
  } while (0)

#define CUDA(call)                                                               \
  do {                                                                           \
    if ((call) != cudaSuccess) {                                                 \
      fprintf(stderr, "%s failed\n", #call);                                     \
      return 1;                                                                  \
    }                                                                            \
  } while (0)

static int host_part(void) {
  const lbm_shape s = {24, 20, 2, 0};
  const size_t np = gnn_param_count();
  float* theta = (float*)malloc(np * sizeof(float));
  if (!theta) return 1;
  CHECK(gnn_params_init_xavier(theta, 5, 1e-2f, 0));
  double sum = 0.0, sum_abs = 0.0;
  for (size_t i = 0; i < np; ++i) {
    sum += theta[i];
    sum_abs += fabs(theta[i]);
  }
  int abi = 0, layout = 0;
  CHECK(lbm_version(&abi, &layout));
  /* a NULL vector and an unknown variant are rejected */
  const int bad_null = gnn_params_init_xavier(NULL, 5, 1e-2f, 0);
  const int bad_variant = gnn_params_init_xavier(theta, 5, 1e-2f, 8);
  /* training entry points: workspace sizes, and argument errors found on the
   * host before any launch (an even refinement of the channel, K = 0) */
  const lbm_shape fine = {72, 60, 2, 0};
  const int bad_factor = lbm_restrict_channel((const float*)(uintptr_t)0x100000, fine,
                                              (float*)(uintptr_t)0x10000000, s, 2, 0.8f, NULL,
                                              0.7f, NULL, 1e-4f, NULL, NULL);
  const int bad_k = gnn_train_step_rollout((const float*)(uintptr_t)0x100000,
                                           (const float*)(uintptr_t)0x10000000, 0, s, 0.8f, NULL,
                                           theta, (void*)(uintptr_t)0x20000000, theta, theta, 1,
                                           1e-3f, 0.0f, (double*)(uintptr_t)0x30000000, NULL,
                                           (void*)(uintptr_t)0x40000000, 1u << 30, NULL);
  printf("{\"train_ws\": %zu, \"rollout_ws\": %zu, \"bad_factor\": %d, \"bad_k\": %d, ",
         gnn_train_workspace_bytes(s), gnn_rollout_workspace_bytes(s, 3), bad_factor, bad_k);
  printf("\"param_count\": %zu, \"trainable_count\": %zu, \"packed_bytes\": %zu, "
         "\"step_ws\": %zu, \"channel_ws\": %zu, \"host_ws\": %zu, \"saved_bytes\": %zu, "
         "\"xavier_sum\": %.17g, \"xavier_sum_abs\": %.17g, \"xavier_first\": %.9g, "
         "\"xavier_last\": %.9g, \"bad_null\": %d, \"bad_variant\": %d, "
         "\"status_ok\": \"%s\", \"status_tau\": \"%s\", \"abi\": %d, \"layout\": %d}\n",
         np, gnn_trainable_count(), gnn_packed_bytes(), gnn_step_workspace_bytes(s),
         gnn_channel_workspace_bytes(s), lbm_host_workspace_bytes(s), gnn_saved_bytes(s), sum, sum_abs, theta[0],
         theta[np - 1], bad_null, bad_variant, lbm_status_string(LBM_OK),
         lbm_status_string(LBM_ERR_TAU), abi, layout);
  free(theta);
  return 0;
}

static int gpu_part(const char* out_path) {
  const lbm_shape s = {24, 20, 2, 0};
  const size_t n = (size_t)s.nx * s.ny * s.nb;
  const size_t fbytes = 9 * n * sizeof(float);
  const double pi = 3.14159265358979323846;
  float *fa = NULL, *fb = NULL, *ft = NULL, *params = NULL;
  double* tot = NULL;
  void *packed = NULL, *ws = NULL;
  CUDA(cudaMalloc((void**)&fa, fbytes));
  CUDA(cudaMalloc((void**)&fb, fbytes));
  CUDA(cudaMalloc((void**)&ft, fbytes));
  CUDA(cudaMalloc((void**)&tot, 5 * sizeof(double)));
  CHECK(lbm_init_tgv(fa, s, 1.0, 0.05, 2 * pi / s.nx, 2 * pi / s.ny, 0, NULL));
  CHECK(lbm_step_bgk(fa, fb, ft, s, 0.7f, NULL, 7, tot, NULL));
  CHECK(lbm_get_status(NULL));

  const size_t np = gnn_param_count();
  float* theta = (float*)malloc(np * sizeof(float));
  if (!theta) return 1;
  CHECK(gnn_params_init_xavier(theta, 5, 1e-2f, 0));
  CUDA(cudaMalloc((void**)&params, np * sizeof(float)));
  CUDA(cudaMemcpy(params, theta, np * sizeof(float), cudaMemcpyHostToDevice));
  CUDA(cudaMalloc(&packed, gnn_packed_bytes()));
  CHECK(gnn_pack(params, packed, NULL));
  const size_t wsb = gnn_step_workspace_bytes(s);
  CUDA(cudaMalloc(&ws, wsb));
  /* GNN-LBM step of the BGK result: fb -> fa */
  CHECK(lbm_step_gnn(fb, fa, s, 0.7f, NULL, packed, NULL, ws, wsb, NULL));
  CHECK(lbm_get_status(NULL));
  /* GNN-LBM step of the channel (walls beyond rows 0 and ny-1, force 1e-4)
     of the BGK result: fb -> ft */
  const size_t wcb = gnn_channel_workspace_bytes(s);
  void* wc = NULL;
  CUDA(cudaMalloc(&wc, wcb));
  CHECK(lbm_step_gnn_channel(fb, ft, s, 0.7f, NULL, 1e-4f, packed, NULL, wc, wcb, NULL));
  CHECK(lbm_get_status(NULL));
  /* an aliased output is rejected before anything is launched */
  const int alias = lbm_step_bgk(fa, fa, NULL, s, 0.7f, NULL, 1, NULL, NULL);

  float* host = (float*)malloc(3 * fbytes);
  double th[5];
  if (!host) return 1;
  CUDA(cudaMemcpy(host, fb, fbytes, cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(th, tot, sizeof th, cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(host + 9 * n, fa, fbytes, cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(host + 18 * n, ft, fbytes, cudaMemcpyDeviceToHost));
  FILE* fh = fopen(out_path, "wb");
  if (!fh) return 1;
  const int ok = fwrite(host, 1, fbytes, fh) == fbytes && fwrite(th, 1, sizeof th, fh) == sizeof th &&
                 fwrite(host + 9 * n, 1, fbytes, fh) == fbytes &&
                 fwrite(host + 18 * n, 1, fbytes, fh) == fbytes;
  fclose(fh);
  if (!ok) return 1;
  printf("{\"nodes\": %zu, \"mass\": %.17g, \"alias\": %d}\n", n, th[0], alias);
  free(host);
  free(theta);
  cudaFree(wc);
  cudaFree(ws);
  cudaFree(packed);
  cudaFree(params);
  cudaFree(tot);
  cudaFree(ft);
  cudaFree(fb);
  cudaFree(fa);
  return 0;
}

int main(int argc, char** argv) {
  if (argc >= 2 && strcmp(argv[1], "host") == 0) return host_part();
  if (argc >= 3 && strcmp(argv[1], "gpu") == 0) return gpu_part(argv[2]);
  fprintf(stderr, "usage: abi_consumer host | gpu OUT.bin\n");
  return 2;
}
