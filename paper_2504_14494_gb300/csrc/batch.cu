// Batched runs: many lattices of uneven size and relaxation time, some with
// the BGK collision and some with the GNN-enhanced collision, advanced
// together.  A plan packs the lattices into one population buffer (BGK group
// first, then GNN group; plane stride = total nodes), keeps a device
// descriptor table, picks launch shapes with the autotuner, and records the
// whole multi-step run as one CUDA graph (per step: the batched BGK kernel on
// one branch, the GNN kernels on the other), replayed by a single launch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "gnn.cuh"
#include "gnn_launch.h"
#include "launch.h"
#include "trace.h"

using namespace lbmgnn;

namespace lbmgnn {

// The BGK group: pull-stream from the lattice's own nodes (periodic wrap),
// Eq. 1-2 with the lattice's tau, store.  Tile shape: a block of NT threads
// covers NT * NPT consecutive nodes, thread t the nodes t, t + NT, ... (each
// pass coalesced), so that NPT nodes' loads are in flight per thread.
template <int NT, int NPT>
__global__ void __launch_bounds__(NT) bgk_batch_kernel(const float* __restrict__ fin,
                                                       float* __restrict__ fout,
                                                       const LatDesc* __restrict__ lat, int nlat,
                                                       const int* __restrict__ hint, int64_t count,
                                                       int64_t ps, unsigned* stw) {
  const GeoTable geo{lat, 0, nlat, 0, count, ps, hint};
  const int64_t g0 = (int64_t)blockIdx.x * (NT * NPT) + threadIdx.x;
  float f[NPT][Q];
  int b[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int64_t g = g0 + k * NT;
    if (g < count) {
      const GeoPos p = geo.pos(g);
      b[k] = p.b;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        f[k][q] = __ldg(fin + q * ps + checked(geo_nbr(p, -ex(q), -ey(q)), 0, count, stw));
    }
  }
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int64_t g = g0 + k * NT;
    if (g < count) {
      bgk_collide(f[k], 1.0f / __ldg(&lat[b[k]].tau));
#pragma unroll
      for (int q = 0; q < Q; ++q) fout[q * ps + g] = f[k][q];
    }
  }
}

// Taylor-Green initial state of every lattice (per-lattice rho0, u0, kx, ky).
__global__ void __launch_bounds__(256) tgv_init_table_kernel(float* __restrict__ f,
                                                             const LatDesc* __restrict__ lat,
                                                             int nlat, int64_t count,
                                                             const double* __restrict__ prm,
                                                             int pc) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  const GeoTable geo{lat, 0, nlat, 0, count, count, nullptr};
  const GeoPos p = geo.pos(g);
  const double rho0 = prm[4 * p.b], u0 = prm[4 * p.b + 1], kx = prm[4 * p.b + 2],
               ky = prm[4 * p.b + 3];
  double sx, cx, sy, cy;
  sincos(kx * p.x, &sx, &cx);
  sincos(ky * p.y, &sy, &cy);
  const double ux = u0 * cx * sy, uy = -u0 * sx * cy;
  double rho = rho0;
  if (pc) rho = rho0 * (1.0 - 0.75 * u0 * u0 * ((cx * cx - sx * sx) + (cy * cy - sy * sy)));
  const double usq = ux * ux + uy * uy;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const double eu = ex(q) * ux + ey(q) * uy;
    const double w = q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    f[q * count + g] = (float)(w * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
  }
}

// ---- autotuner ---------------------------------------------------------------------
// Choices are cached per (kernel, SM count, size bucket = floor(log2 nodes)).
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;

std::string tune_key(const char* kernel, int64_t nodes) {
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= nodes) ++b;
  char buf[128];
  std::snprintf(buf, sizeof buf, "%s/sm%d/n2^%d", kernel, num_sms(), b);
  return buf;
}

// Times each candidate (one warm-up, then the best of three CUDA-event
// timings on `st`) and returns the fastest; cached.
template <typename Run>
int tune(const char* kernel, int64_t nodes, const std::vector<int>& cand, cudaStream_t st,
         Run run) {
  const std::string key = tune_key(kernel, nodes);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return cand[0];
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return cand[0];
  }
  int best = cand[0];
  float best_ms = 1e30f;
  for (int c : cand) {
    if (run(c) != cudaSuccess) continue;
    float t = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(a, st);
      run(c);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      t = std::min(t, ms);
    }
    if (t < best_ms) {
      best_ms = t;
      best = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}
}  // namespace

// Tile shapes of the batched BGK kernel the autotuner chooses from, encoded
// as threads per block * 10 + nodes per thread.
const std::vector<int> kBgkTiles = {1281, 1282, 1284, 2561, 2562, 2564, 5121, 5122};

template <int NT, int NPT>
static void bgk_batch_t(const float* fin, float* fout, const LatDesc* lat, int nlat,
                        const int* hint, int64_t count, int64_t ps, unsigned* stw,
                        cudaStream_t st) {
  const int64_t per = (int64_t)NT * NPT;
  bgk_batch_kernel<NT, NPT><<<(unsigned)((count + per - 1) / per), NT, 0, st>>>(
      fin, fout, lat, nlat, hint, count, ps, stw);
}

cudaError_t launch_bgk_batch(const float* fin, float* fout, const LatDesc* lat, int nlat,
                             const int* hint, int64_t count, int64_t ps, int tile,
                             cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  switch (tile) {
    case 1281: bgk_batch_t<128, 1>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
    case 1282: bgk_batch_t<128, 2>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
    case 1284: bgk_batch_t<128, 4>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
    case 2562: bgk_batch_t<256, 2>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
    case 2564: bgk_batch_t<256, 4>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
    case 5121: bgk_batch_t<512, 1>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
    case 5122: bgk_batch_t<512, 2>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
    default: bgk_batch_t<256, 1>(fin, fout, lat, nlat, hint, count, ps, stw, st); break;
  }
  return cudaGetLastError();
}

}  // namespace lbmgnn

// ---- plan ----------------------------------------------------------------------------
struct lbm_batch_plan {
  int device = 0;
  int n = 0, n_bgk = 0, n_gnn = 0;
  std::vector<int64_t> offset_of_input;  // first node of input lattice i
  LatDesc* d_lat = nullptr;               // sorted: BGK group, then GNN group
  int* d_hint = nullptr;                  // per 128-node block: lattice of its first node
  double* d_prm = nullptr;                // [n][4] TGV parameters (sorted order)
  std::vector<int> sorted_to_input;
  int64_t bgk_nodes = 0, gnn_nodes = 0, total = 0;
  int bgk_block = 0, gnn_per_sm = 0;  // tuned launch shapes (BGK: tile code, see kBgkTiles)
  // cached graph of one run configuration
  cudaStream_t cap = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int key_steps = -1;
};

namespace {

void plan_release(lbm_batch_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->d_lat) cudaFree(p->d_lat);
  if (p->d_hint) cudaFree(p->d_hint);
  if (p->d_prm) cudaFree(p->d_prm);
  delete p;
}

int64_t gnn_ws_bytes(const lbm_batch_plan* p) { return p->gnn_nodes * 512; }

// One step of every lattice: src -> dst.
cudaError_t plan_step(lbm_batch_plan* p, const float* src, float* dst, const uint8_t* packed,
                      __nv_bfloat16* ws, cudaStream_t s_bgk, cudaStream_t s_gnn) {
  cudaError_t e = cudaSuccess;
  if (p->n_bgk > 0) {
    e = launch_bgk_batch(src, dst, p->d_lat, p->n_bgk, p->d_hint, p->bgk_nodes, p->total,
                         p->bgk_block,
                         s_bgk);
    if (e != cudaSuccess) return e;
  }
  if (p->n_gnn > 0) {
    e = launch_gnn_step_table(src, dst, p->d_lat, p->n_bgk, p->n_gnn, p->d_hint, p->bgk_nodes,
                              p->gnn_nodes,
                              p->total, packed, ws, s_gnn, p->gnn_per_sm);
  }
  return e;
}

}  // namespace

extern "C" {

int lbm_batch_plan_create(const lbm_lattice_desc* lattices, int n, lbm_batch_plan** out) {
  LBM_TRACE("lbm_batch_plan_create");
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (!lattices || n < 1) return LBM_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    const auto& d = lattices[i];
    if (d.nx < 1 || d.ny < 1 || (int64_t)d.nx * d.ny >= (int64_t(1) << 31)) return LBM_ERR_SIZE;
    if (d.collision != LBM_COLLIDE_BGK && d.collision != LBM_COLLIDE_GNN) return LBM_ERR_ARG;
    if (!std::isfinite(d.tau) || !(d.tau > 0.5f)) return LBM_ERR_TAU;
  }
  auto* p = new lbm_batch_plan();
  p->n = n;
  p->offset_of_input.assign(n, 0);
  std::vector<LatDesc> table;
  int64_t off = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int want = pass == 0 ? LBM_COLLIDE_BGK : LBM_COLLIDE_GNN;
    for (int i = 0; i < n; ++i) {
      if (lattices[i].collision != want) continue;
      LatDesc d{off, lattices[i].nx, lattices[i].ny, lattices[i].tau, 0};
      table.push_back(d);
      p->sorted_to_input.push_back(i);
      p->offset_of_input[i] = off;
      off += (int64_t)lattices[i].nx * lattices[i].ny;
      if (pass == 0) {
        ++p->n_bgk;
        p->bgk_nodes = off;
      } else {
        ++p->n_gnn;
      }
    }
  }
  p->total = off;
  p->gnn_nodes = off - p->bgk_nodes;
  if (p->total > (int64_t(1) << 34)) {
    plan_release(p);
    return LBM_ERR_SIZE;
  }
  // lattice of the first node of every 128-node block
  std::vector<int> hint((size_t)((p->total + 127) / 128));
  for (size_t blk = 0, lo = 0; blk < hint.size(); ++blk) {
    const int64_t g = (int64_t)blk * 128;
    while (lo + 1 < table.size() && table[lo + 1].offset <= g) ++lo;
    hint[blk] = (int)lo;
  }
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaMalloc(&p->d_lat, sizeof(LatDesc) * n) != cudaSuccess ||
      cudaMalloc(&p->d_hint, sizeof(int) * hint.size()) != cudaSuccess ||
      cudaMemcpy(p->d_hint, hint.data(), sizeof(int) * hint.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMalloc(&p->d_prm, sizeof(double) * 4 * n) != cudaSuccess ||
      cudaMemcpy(p->d_lat, table.data(), sizeof(LatDesc) * n, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    plan_release(p);
    return LBM_ERR_CUDA;
  }
  *out = p;
  return LBM_OK;
}

void lbm_batch_plan_destroy(lbm_batch_plan* plan) { plan_release(plan); }

int64_t lbm_batch_nodes(const lbm_batch_plan* plan) { return plan ? plan->total : -1; }

int lbm_batch_offsets(const lbm_batch_plan* plan, int64_t* offsets) {
  LBM_TRACE("lbm_batch_offsets");
  if (!plan || !offsets) return LBM_ERR_ARG;
  std::memcpy(offsets, plan->offset_of_input.data(), sizeof(int64_t) * plan->n);
  return LBM_OK;
}

size_t lbm_batch_workspace_bytes(const lbm_batch_plan* plan) {
  return plan ? (size_t)gnn_ws_bytes(plan) : 0;
}

int lbm_batch_init_tgv(lbm_batch_plan* plan, float* f, const double* params,
                       int pressure_consistent, void* stream) {
  LBM_TRACE("lbm_batch_init_tgv");
  if (!plan || !f || !params) return LBM_ERR_ARG;
  std::vector<double> sorted(4 * (size_t)plan->n);
  for (int j = 0; j < plan->n; ++j)
    std::memcpy(&sorted[4 * j], params + 4 * plan->sorted_to_input[j], 4 * sizeof(double));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(plan->d_prm, sorted.data(), sizeof(double) * 4 * plan->n,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LBM_ERR_CUDA;
  tgv_init_table_kernel<<<(unsigned)((plan->total + 255) / 256), 256, 0, st>>>(
      f, plan->d_lat, plan->n, plan->total, plan->d_prm, pressure_consistent ? 1 : 0);
  return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int lbm_batch_run(lbm_batch_plan* plan, const float* f_in, float* f_out, float* f_tmp, int steps,
                  const void* packed, void* workspace, size_t ws_bytes, void* stream) {
  LBM_TRACE("lbm_batch_run");
  if (!plan || !f_in || !f_out || steps < 0) return LBM_ERR_ARG;
  if (steps > 1 && !f_tmp) return LBM_ERR_ARG;
  if (f_in == f_out || f_tmp == f_in || (f_tmp && f_tmp == f_out)) return LBM_ERR_ALIAS;
  if (plan->n_gnn > 0) {
    if (!packed) return LBM_ERR_ARG;
    if (!workspace || (int64_t)ws_bytes < gnn_ws_bytes(plan) ||
        (reinterpret_cast<uintptr_t>(workspace) & 15))
      return LBM_ERR_WORKSPACE;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return LBM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t bytes = 9 * plan->total * (int64_t)sizeof(float);
  if (steps == 0)
    return cudaMemcpyAsync(f_out, f_in, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess
               ? LBM_OK
               : LBM_ERR_CUDA;
  const uint8_t* pk = static_cast<const uint8_t*>(packed);
  auto* ws = static_cast<__nv_bfloat16*>(workspace);
  // Launch shapes: tuned once per size bucket (the timing runs write f_out).
  if (!plan->bgk_block) {
    plan->bgk_block = plan->n_bgk == 0 ? 2561 : tune("bgk_batch_tile", plan->bgk_nodes, kBgkTiles, st,
        [&](int c) {
          return launch_bgk_batch(f_in, f_out, plan->d_lat, plan->n_bgk, plan->d_hint,
                                  plan->bgk_nodes,
                                  plan->total, c, st);
        });
  }
  if (!plan->gnn_per_sm) {
    plan->gnn_per_sm = plan->n_gnn == 0 ? 2 : tune("gnn_step_table", plan->gnn_nodes, {1, 2}, st,
        [&](int c) {
          return launch_gnn_step_table(f_in, f_out, plan->d_lat, plan->n_bgk, plan->n_gnn,
                                       plan->d_hint, plan->bgk_nodes, plan->gnn_nodes, plan->total, pk, ws, st,
                                       c);
        });
  }
  const void* key[6] = {f_in, f_out, f_tmp, packed, workspace, nullptr};
  bool same = plan->exec && plan->key_steps == steps;
  for (int i = 0; i < 6 && same; ++i) same = key[i] == plan->key[i];
  if (!same) {
    if (plan->exec) {
      cudaGraphExecDestroy(plan->exec);
      plan->exec = nullptr;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(plan->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return LBM_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    const float* src = f_in;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
      const int left = steps - k;
      float* dst = (left % 2 == 1) ? f_out : f_tmp;
      e = cudaEventRecord(plan->ev_fork, plan->cap);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->side, plan->ev_fork, 0);
      if (e == cudaSuccess) e = plan_step(plan, src, dst, pk, ws, plan->cap, plan->side);
      if (e == cudaSuccess) e = cudaEventRecord(plan->ev_join, plan->side);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->cap, plan->ev_join, 0);
      src = dst;
    }
    const cudaError_t e2 = cudaStreamEndCapture(plan->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      return LBM_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&plan->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      plan->exec = nullptr;
      return LBM_ERR_CUDA;
    }
    std::memcpy(plan->key, key, sizeof key);
    plan->key_steps = steps;
  }
  return cudaGraphLaunch(plan->exec, st) == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

int lbm_autotune_save(const char* path) {
  LBM_TRACE("lbm_autotune_save");
  if (!path) return LBM_ERR_ARG;
  FILE* fh = std::fopen(path, "w");
  if (!fh) return LBM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::fprintf(fh, "{");
  bool first = true;
  for (const auto& kv : g_tune) {
    std::fprintf(fh, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  std::fprintf(fh, "\n}\n");
  std::fclose(fh);
  return LBM_OK;
}

int lbm_autotune_load(const char* path) {
  LBM_TRACE("lbm_autotune_load");
  if (!path) return LBM_ERR_ARG;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return LBM_ERR_ARG;
  std::string txt;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof buf, fh)) > 0) txt.append(buf, got);
  std::fclose(fh);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  size_t pos = 0;
  while ((pos = txt.find('"', pos)) != std::string::npos) {
    const size_t end = txt.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = txt.substr(pos + 1, end - pos - 1);
    const size_t colon = txt.find(':', end);
    if (colon == std::string::npos) break;
    g_tune[key] = std::atoi(txt.c_str() + colon + 1);
    pos = colon + 1;
  }
  return LBM_OK;
}

}  // extern "C"
