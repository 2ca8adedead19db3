// Channel (Poiseuille) flow, paper Sec. 3.1 Eq. 5: the BGK step with walls
// and a body force.  The paper names "Apply Boundary Conditions" (Fig. 1)
// without a scheme; this library uses halfway bounce-back walls at
// y = -1/2 and y = ny - 1/2 of every lattice (periodic in x) and Guo's
// forcing for a force (G, 0) per unit volume:
//   u = (sum f_i e_i + F/2) / rho,
//   f*_i = f_i - (f_i - f_i^eq)/tau + (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i].F
// In pull form the bounce-back reads f_i(x, y) = f*_opp(i)(x, y) whenever
// (x - e_ix, y - e_iy) lies outside the channel.
//
// The GNN-LBM step of the channel (Eq. 3 in place of the BGK relaxation)
// runs as pull (channel_pull_kernel) -> network on the walled graph
// (gnn_fwd.cu, GeoChannel) -> channel_gnn_collide_kernel, which relaxes with
// the network's time tau tau_adj, adds Guo's source with that same time and
// the correction Delta f.
//
// Training data of the channel network (Sec. 2.4 for this flow): the
// restriction of an m-times refined channel (odd m) that separates the
// force part of the non-equilibrium populations from the gradient part
// (channel_restrict_kernel).
#include "common.cuh"
#include "gnn.cuh"
#include "gnn_launch.h"
#include "launch.h"

namespace lbmgnn {

// Node n = (b, y, x): the nine populations pulled from the stored state with
// the channel's walls.
__device__ __forceinline__ void channel_pull(const float* __restrict__ fin, const Shape& s,
                                             int64_t nn, int x, int y, int64_t lat,
                                             float (&f)[Q], unsigned* stw) {
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int ys = y - ey(q);
    if (ys < 0 || ys >= s.ny) {
      f[q] = __ldg(fin + opp(q) * s.ps + nn);  // halfway bounce-back
    } else {
      int xs = x - ex(q);
      xs = xs < 0 ? xs + s.nx : (xs >= s.nx ? xs - s.nx : xs);
      f[q] = __ldg(fin + q * s.ps +
                   checked(lat + (int64_t)ys * s.nx + xs, 0, (int64_t)s.nb * s.ny * s.nx, stw));
    }
  }
}

// Block sums of the totals (mass, momentum, energy, non-finite count) of the
// written populations, one atomic per quantity and block.
__device__ __forceinline__ void channel_totals(const float (&f)[Q], bool on,
                                               double* __restrict__ totals, unsigned* stw) {
  double tt[5] = {0, 0, 0, 0, 0};
  if (on) {
    bool finite = true;
#pragma unroll
    for (int q = 0; q < Q; ++q) finite &= isfinite(f[q]);
    if (finite) {
      double r = 0.0, px = 0.0, py = 0.0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        r += f[q];
        if (ex(q)) px += ex(q) * (double)f[q];
        if (ey(q)) py += ey(q) * (double)f[q];
      }
      tt[0] = r;
      tt[1] = px;
      tt[2] = py;
      tt[3] = 0.5 * (px * px + py * py) / r;
    } else {
      tt[4] = 1.0;
    }
  }
  if (tt[4] != 0.0) raise_status(stw, ST_NONFINITE);
  __shared__ double red[8][5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tt[k] += __shfl_xor_sync(0xffffffffu, tt[k], o);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) red[threadIdx.x >> 5][k] = tt[k];
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double acc = 0.0;
    for (int i = 0; i < 8; ++i) acc += red[i][threadIdx.x];
    if (acc != 0.0) atomicAdd(totals + threadIdx.x, acc);
  }
}

// f_i - (f_i - f_i^eq(rho, u))/t + (1 - 1/(2t)) w_i [3 (e_i - u) + 9 (e_i.u) e_i].(gx, 0)
// with u the force-corrected velocity; t is tau (BGK) or tau tau_adj (Eq. 3).
__device__ __forceinline__ void channel_relax(float (&f)[Q], float t, float gx) {
  const float rho = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
  const float jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
  const float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const float inv = 1.0f / rho;
  const Moments m{rho, (jx + 0.5f * gx) * inv, jy * inv};
  const float usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy);
  const float omega = 1.0f / t, pre = 1.0f - 0.5f * omega;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float eu = float(ex(q)) * m.ux + float(ey(q)) * m.uy;
    const float src = pre * wq(q) * (3.0f * (float(ex(q)) - m.ux) + 9.0f * eu * float(ex(q))) * gx;
    f[q] = f[q] - omega * (f[q] - feq_i(q, m, usq15)) + src;
  }
}

struct NodeIdx {
  int64_t n, nn, lat;
  int x, y, b;
  bool on;
};
__device__ __forceinline__ NodeIdx node_idx(const Shape& s) {
  NodeIdx r;
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  r.n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  r.on = r.n < N;
  r.nn = r.on ? r.n : N - 1;
  r.x = (int)(r.nn % s.nx);
  const int64_t row = r.nn / s.nx;
  r.b = (int)(row / s.ny);
  r.y = (int)(row - (int64_t)r.b * s.ny);
  r.lat = (int64_t)r.b * s.ny * s.nx;
  return r;
}

template <bool TOTALS>
__global__ void __launch_bounds__(256) channel_step_kernel(const float* __restrict__ fin,
                                                           float* __restrict__ fout, Shape s,
                                                           float tau, const float* __restrict__ taus,
                                                           float gx, double* __restrict__ totals,
                                                           unsigned* stw) {
  const NodeIdx i = node_idx(s);
  float f[Q];
  channel_pull(fin, s, i.nn, i.x, i.y, i.lat, f, stw);
  channel_relax(f, taus ? __ldg(taus + i.b) : tau, gx);
  if (i.on) {
#pragma unroll
    for (int q = 0; q < Q; ++q) fout[q * s.ps + i.nn] = f[q];
  }
  if constexpr (TOTALS) channel_totals(f, i.on, totals, stw);
}

cudaError_t launch_channel_step(const float* fin, float* fout, const Shape& s, float tau,
                                const float* taus, float gx, double* totals, cudaStream_t st) {
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  unsigned* stw = status_word();
  if (totals && !stw) return cudaErrorInvalidDevice;
  const unsigned blocks = (unsigned)((N + 255) / 256);
  if (totals)
    channel_step_kernel<true><<<blocks, 256, 0, st>>>(fin, fout, s, tau, taus, gx, totals, stw);
  else
    channel_step_kernel<false><<<blocks, 256, 0, st>>>(fin, fout, s, tau, taus, gx, totals, stw);
  return cudaGetLastError();
}

// ---- GNN-LBM step of the channel ------------------------------------------------

// f_pre = stream(f_post) with the walls: the network's input (Fig. 2) and the
// populations that Eq. 3 relaxes.
__global__ void __launch_bounds__(256) channel_pull_kernel(const float* __restrict__ fin,
                                                           float* __restrict__ fpre, Shape s,
                                                           unsigned* stw) {
  const NodeIdx i = node_idx(s);
  float f[Q];
  channel_pull(fin, s, i.nn, i.x, i.y, i.lat, f, stw);
  if (i.on) {
#pragma unroll
    for (int q = 0; q < Q; ++q) fpre[q * s.ps + i.nn] = f[q];
  }
}

// Eq. 3 with Guo's source: f* = f - (f - f^eq)/(tau tau_adj) + S(tau tau_adj)
// + Delta f, from the head output y [10][N] (tau_adj and Delta f as in the
// periodic step: fixed-tau and conserving variants read from the image).
template <bool TOTALS>
__global__ void __launch_bounds__(256) channel_gnn_collide_kernel(
    const float* __restrict__ fpre, const float* __restrict__ y, float* __restrict__ fout,
    Shape s, float tau, const float* __restrict__ taus, float gx,
    const uint8_t* __restrict__ packed, double* __restrict__ totals, unsigned* stw) {
  if (!blob_ok(packed, stw)) return;
  const NodeIdx i = node_idx(s);
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const float* nrm = reinterpret_cast<const float*>(packed + K::NORM);
  const float sdf = __ldg(nrm + 24);
  const int variant = variant_of(nrm);
  float f[Q], d[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) f[q] = __ldg(fpre + q * s.ps + i.nn);
#pragma unroll
  for (int q = 0; q < Q; ++q) d[q] = sdf * __ldg(y + (int64_t)(1 + q) * N + i.nn);
  if (variant & VAR_CONSERVATIVE) conserve9(d);
  const float t = (taus ? __ldg(taus + i.b) : tau) * tau_adj_of(__ldg(y + i.nn), variant);
  channel_relax(f, t, gx);
#pragma unroll
  for (int q = 0; q < Q; ++q) f[q] += d[q];
  if (i.on) {
#pragma unroll
    for (int q = 0; q < Q; ++q) fout[q * s.ps + i.nn] = f[q];
  }
  if constexpr (TOTALS) channel_totals(f, i.on, totals, stw);
}

// ---- restriction of a refined channel --------------------------------------------

// Coarse node (b, J, I) <- fine node (b, m J + (m-1)/2, m I + (m-1)/2) (odd
// m: both lattices' walls lie halfway beyond their outer rows).  The fine
// node's populations are pulled from the fine stored state with the walls
// (its pre-collision state of the next step), and with u = (j + F_f/2)/rho,
//   P = (tau_f - 1/2) w_i [3 (e_i - u) + 9 (e_i.u) e_i].F_f   (force part),
//   G = f - f^eq - P                                          (gradient part),
//   f*_c = f^eq + (1 - 1/tau_c) m (tau_c / tau_f) G + P.
__global__ void __launch_bounds__(256) channel_restrict_kernel(
    const float* __restrict__ ff, Shape fs, float* __restrict__ fc, Shape cs, int m, float tau_f,
    const float* __restrict__ taus_f, float tau_c, const float* __restrict__ taus_c, float gx_f,
    const float* __restrict__ gxs_f, unsigned* stw) {
  const NodeIdx c = node_idx(cs);
  if (!c.on) return;
  const int o = (m - 1) / 2;
  const int xf = m * c.x + o, yf = m * c.y + o;
  const int64_t latf = (int64_t)c.b * fs.ny * fs.nx;
  const int64_t nf = latf + (int64_t)yf * fs.nx + xf;
  float f[Q];
  channel_pull(ff, fs, nf, xf, yf, latf, f, stw);
  const float tf = taus_f ? __ldg(taus_f + c.b) : tau_f;
  const float tc = taus_c ? __ldg(taus_c + c.b) : tau_c;
  const float gx = gxs_f ? __ldg(gxs_f + c.b) : gx_f;
  const float rho = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
  const float jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
  const float jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const float inv = 1.0f / rho;
  const Moments mo{rho, (jx + 0.5f * gx) * inv, jy * inv};
  const float usq15 = 1.5f * (mo.ux * mo.ux + mo.uy * mo.uy);
  const float kg = (1.0f - 1.0f / tc) * (float)m * (tc / tf), kp = tf - 0.5f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float fe = feq_i(q, mo, usq15);
    const float eu = float(ex(q)) * mo.ux + float(ey(q)) * mo.uy;
    const float p = kp * wq(q) * (3.0f * (float(ex(q)) - mo.ux) + 9.0f * eu * float(ex(q))) * gx;
    fc[q * cs.ps + c.n] = fe + kg * ((f[q] - fe) - p) + p;
  }
}

cudaError_t launch_channel_restrict(const float* f_fine, const Shape& fs, float* f_coarse,
                                    const Shape& cs, int m, float tau_f, const float* taus_f,
                                    float tau_c, const float* taus_c, float gx_f,
                                    const float* gxs_f, cudaStream_t st) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  const int64_t N = (int64_t)cs.nb * cs.ny * cs.nx;
  channel_restrict_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(
      f_fine, fs, f_coarse, cs, m, tau_f, taus_f, tau_c, taus_c, gx_f, gxs_f, stw);
  return cudaGetLastError();
}

cudaError_t launch_channel_pull(const float* fin, float* fpre, const Shape& s, cudaStream_t st) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  channel_pull_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(fin, fpre, s, stw);
  return cudaGetLastError();
}

cudaError_t launch_channel_gnn_collide(const float* fpre, const float* y, float* fout,
                                       const Shape& s, float tau, const float* taus, float gx,
                                       const uint8_t* packed, double* totals, cudaStream_t st) {
  unsigned* stw = status_word();
  if (!stw) return cudaErrorInvalidDevice;
  const int64_t N = (int64_t)s.nb * s.ny * s.nx;
  const unsigned blocks = (unsigned)((N + 255) / 256);
  if (totals)
    channel_gnn_collide_kernel<true>
        <<<blocks, 256, 0, st>>>(fpre, y, fout, s, tau, taus, gx, packed, totals, stw);
  else
    channel_gnn_collide_kernel<false>
        <<<blocks, 256, 0, st>>>(fpre, y, fout, s, tau, taus, gx, packed, totals, stw);
  return cudaGetLastError();
}

}  // namespace lbmgnn
