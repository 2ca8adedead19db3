/* lbmgnn.h -- C ABI of the GB300 (sm_103a) LBM-GNN library, liblbmgnn.so.
 *
 * The library advances D2Q9 lattice Boltzmann populations with the BGK
 * collision (paper Sec. 2.1, Eq. 1-2, Fig. 1) or with the GNN-enhanced
 * collision (Sec. 2.2-2.3, Eq. 3), and trains that network (Sec. 2.4, Eq. 4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers named f, f_in, f_out, ... are DEVICE pointers to caller-owned
 *    memory.  The library allocates nothing unless a call says so.
 *  - Population layout (SoA, q-major): the value of direction q at node (x, y)
 *    of lattice b is  f[q * plane_stride + (b * ny + y) * nx + x],  with
 *    0 <= q < 9, 0 <= b < nb.  plane_stride = 0 means nb * ny * nx.
 *  - D2Q9 order: e_0=(0,0); e_1..4=(1,0),(0,1),(-1,0),(0,-1);
 *    e_5..8=(1,1),(-1,1),(-1,-1),(1,-1); w = 4/9, 1/9 (x4), 1/36 (x4).
 *  - Stored state: the POST-collision populations f*(., n).  One step pulls
 *    f_i(x) = f*_i(x - e_i) with periodic wrap inside each lattice (streaming),
 *    collides, and stores f*(., n+1) at x.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on it; arguments are checked on the host before any launch.
 *  - Every call returns an int status: LBM_OK or a negative LBM_ERR_* code.
 *    Faults detected inside kernels (non-finite values, a device wait that
 *    gave up, an index that failed a bounds check) raise bits of a per-device
 *    status word, which lbm_get_status() reports and clears.
 *  - The library never aborts or prints.
 */
#ifndef LBMGNN_H
#define LBMGNN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,        /* NULL pointer, bad enum, nsteps < 0, ... */
  LBM_ERR_ALIAS = -2,      /* an output buffer aliases an input buffer */
  LBM_ERR_SIZE = -3,       /* nx, ny, nb or plane_stride out of range */
  LBM_ERR_TAU = -4,        /* tau <= 1/2 (negative viscosity) or not finite */
  LBM_ERR_BLOB = -5,       /* packed parameter image invalid (see gnn_pack) */
  LBM_ERR_CUDA = -6,       /* a CUDA runtime call failed */
  LBM_ERR_NONFINITE = -7,  /* a kernel produced a NaN or Inf population */
  LBM_ERR_TIMEOUT = -8,    /* a device-side wait gave up */
  LBM_ERR_BOUNDS = -9,     /* a gather index failed its bounds check (checked build) */
  LBM_ERR_WORKSPACE = -10  /* workspace missing or smaller than required */
};

typedef struct {
  int32_t nx, ny;        /* nodes per lattice in x and y, each >= 1 */
  int32_t nb;            /* number of stacked lattices, >= 1; nb*ny*nx <= 2^36 */
  int64_t plane_stride;  /* elements between planes (>= nb*ny*nx); 0 = nb*ny*nx */
} lbm_shape;

/* Human-readable name of a status code (static string). */
LBM_API const char* lbm_status_string(int status);

/* Versions of this library (no counterpart in the paper; host-only, no GPU
 * needed): *abi receives LBM_ABI_VERSION, the version of the calls and
 * structs declared here, *packed_layout the layout version of the packed
 * parameter image that gnn_pack writes and the kernels check.  Either
 * pointer may be NULL.  Returns LBM_OK. */
#define LBM_ABI_VERSION 1
#define LBM_PACKED_LAYOUT_VERSION 1
LBM_API int lbm_version(int* abi, int* packed_layout);

/* Waits for `stream`, then reads and clears the device status word of the
 * current device.  Returns LBM_OK, or the most severe of LBM_ERR_TIMEOUT,
 * LBM_ERR_BOUNDS, LBM_ERR_BLOB, LBM_ERR_NONFINITE raised since the last
 * call. */
LBM_API int lbm_get_status(void* stream);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * small kernel that waits on a device barrier nothing arrives on, with a
 * budget of max_cycles SM cycles (1 .. 2e9); the wait gives up, raises the
 * timeout bit and the kernel returns, exactly as the tensor-core kernels do
 * when a wait runs out.  The next lbm_get_status() then returns
 * LBM_ERR_TIMEOUT.  Nothing traps or hangs. */
LBM_API int lbm_selftest_wait_timeout(long long max_cycles, void* stream);

/* Taylor-Green vortex initial state (paper Sec. 3.2; the formula is this
 * library's reading): u_x = u0 cos(kx x) sin(ky y), u_y = -u0 sin(kx x)
 * cos(ky y) at integer node coordinates, rho = rho0 or, if
 * pressure_consistent, rho0 (1 - 3/4 u0^2 (cos 2kx x + cos 2ky y));
 * f = f^eq(rho, u) (Eq. 2), evaluated in FP64 and stored as FP32 in every
 * lattice of the stack.  f: device, 9 planes of shape s. */
LBM_API int lbm_init_tgv(float* f, lbm_shape s, double rho0, double u0, double kx, double ky,
                 int pressure_consistent, void* stream);

/* nsteps BGK steps (Eq. 1 with the equilibrium of Eq. 2, Fig. 1 loop):
 * pull-stream with periodic wrap, moments, f^eq, relaxation
 * f* = f - (f - f^eq)/tau, store.  One fused kernel per step.
 *   f_in   device, read only; the state after n steps.
 *   f_out  device; receives the state after n + nsteps steps.  != f_in.
 *   f_tmp  device ping-pong buffer of the same shape, required when
 *          nsteps > 1 (else may be NULL); distinct from f_in and f_out.
 *   tau    relaxation time (> 1/2) of every lattice, used when `taus` is NULL.
 *   taus   optional device float[nb]: per-lattice relaxation times.
 *   totals optional device double[5]; if given it is OVERWRITTEN with FP64
 *          sums over the final state: mass, x-momentum, y-momentum, kinetic
 *          energy 1/2 sum |rho u|^2/rho, and the number of nodes holding a
 *          non-finite value (such nodes are left out of the four sums).
 * nsteps == 0 copies f_in to f_out.  A non-finite output raises
 * LBM_ERR_NONFINITE in the status word only when totals are requested. */
LBM_API int lbm_step_bgk(const float* f_in, float* f_out, float* f_tmp, lbm_shape s, float tau,
                 const float* taus, int nsteps, double* totals, void* stream);

/* nsteps steps of the channel (Poiseuille) flow of paper Sec. 3.1: the BGK
 * step with walls and a body force.  The paper gives no wall or force scheme;
 * this library's reading: every lattice of the stack is a channel along x
 * (periodic in x) between walls halfway outside the first and last rows
 * (y = -1/2 and y = ny - 1/2, channel height H = ny), halfway bounce-back
 * (a population that would stream in from behind a wall is the node's own
 * opposite post-collision population), and Guo's forcing for a force
 * (force_x, 0) per unit volume: the velocity is u = (sum f_i e_i + F/2)/rho
 * and the collision adds (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i.u) e_i].F.
 * Steady state (rho = 1): u(y) = F/(2 nu) (y + 1/2)(ny - 1/2 - y) plus a
 * constant wall slip of O(F/nu) (Eq. 5).  Arguments, ping-pong and totals as
 * lbm_step_bgk (lbm_moments of the result returns sum f e / rho; add F/(2 rho)
 * for the velocity of the forced scheme). */
LBM_API int lbm_step_channel(const float* f_in, float* f_out, float* f_tmp, lbm_shape s, float tau,
                             const float* taus, float force_x, int nsteps, double* totals,
                             void* stream);

/* Bytes of the device workspace of lbm_step_bgk_host for shape s (two
 * population buffers, the totals and the per-lattice taus); 0 for a bad
 * shape. */
LBM_API size_t lbm_host_workspace_bytes(lbm_shape s);

/* lbm_step_bgk for a state held in HOST memory (Eq. 1-2, Fig. 1 loop):
 * copies f_in_host (host, populations of shape s in the device layout: 9
 * planes of plane_stride floats) to the device, advances nsteps >= 1 steps,
 * and copies the FP64 totals of the final state (as lbm_step_bgk) to
 * totals_host (host double[5], nullable) and the final state to f_out_host
 * (host, same layout, nullable).  taus_host: nullable host array of nb
 * per-lattice relaxation times (else tau for every lattice).
 *
 * The host-to-device copy runs on a second stream of the library's own in
 * 16 blocks of lattice rows (one 2D copy of the 9 planes per block);
 * the first step of a block is launched on `stream` as soon as the rows it
 * pulls from (y -+ 1 with periodic wrap) have arrived, so the copy overlaps
 * the step.  The final step is also launched by row blocks, and each block of
 * the final state is copied to f_out_host on a third stream as soon as its
 * kernel is done (overlapping the rest of the step and, for nsteps == 1, the
 * host-to-device copy of the remaining blocks).  Overlap needs page-locked
 * host memory; pageable memory works without it.  Asynchronous on `stream`: host outputs are valid, and host
 * inputs may be reused, once `stream` has completed the call's work.
 * workspace: device, 256-byte aligned, lbm_host_workspace_bytes(s) bytes, not
 * used by another call in flight on another stream.  Errors as lbm_step_bgk;
 * LBM_ERR_WORKSPACE for a missing, small or misaligned workspace. */
LBM_API int lbm_step_bgk_host(const float* f_in_host, float* f_out_host, lbm_shape s, float tau,
                              const float* taus_host, int nsteps, double* totals_host,
                              void* workspace, size_t ws_bytes, void* stream);

/* Macroscopic variables of a stored state (Fig. 1 'Compute macroscopic
 * variables'): rho = sum f_i, u = sum f_i e_i / rho per node (FP32 out,
 * node-major planes of nb*ny*nx values), and optional FP64 totals (as in
 * lbm_step_bgk).  Any of rho, ux, uy, totals may be NULL. */
LBM_API int lbm_moments(const float* f, lbm_shape s, float* rho, float* ux, float* uy,
                double* totals, void* stream);

/* ---------------------------------------------------------------------------
 * GNN-enhanced collision (paper Sec. 2.2-2.3, Fig. 2, Eq. 3)
 *
 * Network (this library's reading of Sec. 2.2, whose components the paper
 * names without formulas): features x = [f_0..f_8, rho, u_x, u_y] of the
 * pre-collision node, normalised (x - mu)/sigma; encoder 12-64-64 (Linear +
 * GELU twice); two message-passing rounds over the 8 lattice neighbours
 * j = i + e_k with m_ik = GELU(W_e [h_i; h_j; e_k] + b_e), a_i = sum_k m_ik,
 * h_i <- h_i + GELU(W_n [h_i; a_i] + b_n) (separate weights per round); head
 * y = W_h h + b_h (10 outputs); tau_adj = 1/2 + sigmoid(y_0) in (1/2, 3/2)
 * and Delta f_i = s_df y_{1+i} (Fig. 2 heads); f*_i = f_i - (f_i - f_i^eq) /
 * (tau tau_adj) + Delta f_i (Eq. 3).  GELU is the tanh form.
 *
 * Parameter vector (FP32, `params`), in this order:
 *   enc1.W[64][12] enc1.b[64] enc2.W[64][64] enc2.b[64]
 *   round 1: edge.W[64][130] edge.b[64] node.W[64][128] node.b[64]
 *   round 2: same shapes
 *   head.W[10][64] head.b[10]                     -> 38,922 trainable values
 *   mu[12] sigma[12] s_df variant                 -> 26 fixed values
 * Row-major W[out][in]; edge.W columns are [h_i (64) | h_j (64) | e_k (2)],
 * node.W columns are [h_i (64) | a_i (64)].
 * Weight matrices are used as BF16 (round to nearest even); biases and the
 * fixed values as FP32.  Dense layers run on the tensor cores with FP32
 * accumulation; activations are stored as BF16.
 * ------------------------------------------------------------------------- */

/* Number of floats of the parameter vector (38,948) and of its trainable
 * prefix (38,922).  The last value selects a variant of the network (sum of
 * flags, as a float): LBM_GNN_MLP_ONLY (1) is the paper's Fig. 2 network
 * (both encoder layers ReLU, no message passing, head on h0; the round
 * weights are unused and get zero gradients); LBM_GNN_CONSERVATIVE (2)
 * projects Delta f orthogonal to 1, e_x, e_y, so that Eq. 3 conserves mass
 * and momentum exactly like Eq. 1 (this library's option; the paper adds
 * Delta f unconstrained); LBM_GNN_FIXED_TAU (4) leaves the relaxation-time
 * head unused: tau_adj = 1 in Eq. 3 (the BGK relaxation time), the network
 * acts through Delta f alone and the head's first row gets zero gradients
 * (this library's option for training: a learned tau_adj multiplies the
 * relaxation of every non-equilibrium moment, i.e. it changes the
 * viscosity). */
enum { LBM_GNN_MLP_ONLY = 1, LBM_GNN_CONSERVATIVE = 2, LBM_GNN_FIXED_TAU = 4 };
LBM_API size_t gnn_param_count(void);
LBM_API size_t gnn_trainable_count(void);

/* Fills a parameter vector in HOST memory (gnn_param_count() floats) with a
 * starting point for training (Sec. 2.2 names the layers, not their
 * initialisation): every weight matrix Xavier-uniform, U(-b, b) with
 * b = sqrt(6 / (fan_in + fan_out)), every bias 0, drawn in parameter order
 * from a SplitMix64 stream seeded with `seed` (the same seed gives the same
 * vector on any machine); the input normaliser mu / sigma at the rest-state
 * populations (4/9, 1/9 x4, 1/36 x4) with a 10 % scale, rho 1 with scale
 * 0.01, u 0 with scale 0.01; the Delta f scale s_df (> 0, finite); and the
 * variant flags (0..7, see above).  Host-only: no GPU is needed.  Returns
 * LBM_ERR_ARG for a NULL vector, a bad s_df or unknown flags. */
LBM_API int gnn_params_init_xavier(float* params_host, uint64_t seed, float s_df, int variant);

/* Bytes of the packed device image of the parameters. */
LBM_API size_t gnn_packed_bytes(void);

/* Converts the FP32 parameter vector (device, gnn_param_count() floats) into
 * the packed image the kernels read (device, gnn_packed_bytes() bytes,
 * 16-byte aligned).  Re-run after every change of the parameters.
 * The image carries a validity word (layout version 1), written only when
 * the vector's fixed values are usable: every mu finite, every sigma and
 * s_df finite and > 0, variant one of 0..7; otherwise the pack raises
 * LBM_ERR_BLOB in the status word.  Every kernel that reads an image checks
 * the word first; given one without it (never packed, packed from invalid
 * fixed values, or another buffer) it computes and writes nothing (a loss
 * output becomes NaN) and raises LBM_ERR_BLOB in the status word. */
LBM_API int gnn_pack(const float* params, void* packed, void* stream);

/* Workspace bytes lbm_step_gnn needs for shape s (512 bytes per node: the
 * node states h and edge terms B = W_b h of the encoder and round 1). */
LBM_API size_t gnn_step_workspace_bytes(lbm_shape s);

/* One GNN-LBM step (Fig. 1 with 'Use GNN?' = yes): pull-stream f_in with
 * periodic wrap, run the network on the pre-collision state, apply Eq. 3 and
 * store f*(n+1) in f_out.
 *   f_in, f_out  device populations of shape s; f_out != f_in.
 *   tau / taus   as in lbm_step_bgk.
 *   packed       device image from gnn_pack.
 *   totals       optional device double[5] (as in lbm_step_bgk), of f_out.
 *   workspace    device scratch of ws_bytes >= gnn_step_workspace_bytes(s),
 *                16-byte aligned; contents undefined afterwards. */
LBM_API int lbm_step_gnn(const float* f_in, float* f_out, lbm_shape s, float tau,
                         const float* taus, const void* packed, double* totals,
                         void* workspace, size_t ws_bytes, void* stream);

/* One GNN-LBM step of the paper's Fig. 2 network (SimpleLBMGNN: the
 * MLP-only variant, LBM_GNN_MLP_ONLY set in the image) as a single fused
 * kernel: pull-stream, moments, features, Linear + ReLU twice and the heads
 * on the tensor cores, Eq. 3, store; 72 bytes of memory traffic per node and
 * no workspace.  lbm_step_gnn takes the same kernel for such an image (after
 * reading the variant on the device), at the cost of three more launches
 * that return at once.  Arguments and results as lbm_step_gnn.  An image of
 * a message-passing network is refused on the device: nothing is written
 * and LBM_ERR_BLOB is raised in the status word. */
LBM_API int lbm_step_gnn_mlp(const float* f_in, float* f_out, lbm_shape s, float tau,
                             const float* taus, const void* packed, double* totals,
                             void* stream);

/* Workspace bytes lbm_step_gnn_channel needs for shape s: the pre-collision
 * populations (rounded up to 256 bytes) and 808 bytes per node (node states,
 * edge terms and head output of the network); 0 for a bad shape. */
LBM_API size_t gnn_channel_workspace_bytes(lbm_shape s);

/* One GNN-LBM step of the channel flow of paper Sec. 3.1 (walls and body
 * force as in lbm_step_channel) with the collision of Eq. 3.  The paper does
 * not say how the network meets the walls; this library's reading: the
 * message-passing graph is the channel's own (periodic in x; a node next to
 * a wall has no neighbour beyond it, and that message is left out of the
 * sum), the velocity feature is the force-corrected one (sum f e + F/2)/rho,
 * and Guo's source is taken with the network's relaxation time:
 *   f* = f - (f - f^eq)/(tau tau_adj) + (1 - 1/(2 tau tau_adj)) w_i
 *        [3 (e_i - u) + 9 (e_i.u) e_i].F + Delta f,
 * f the populations pulled with halfway bounce-back.  With a network whose
 * heads give tau_adj = 1 and Delta f = 0 this is exactly lbm_step_channel.
 *   f_in, f_out  device populations of shape s; f_out != f_in.
 *   tau / taus   as in lbm_step_bgk; force_x finite.
 *   packed       device image from gnn_pack (any variant).
 *   totals       optional device double[5], of f_out.
 *   workspace    device scratch of ws_bytes >= gnn_channel_workspace_bytes(s),
 *                256-byte aligned; contents undefined afterwards.
 * Errors: LBM_ERR_ARG (null pointer, non-finite force, misaligned image),
 * LBM_ERR_SIZE, LBM_ERR_TAU, LBM_ERR_WORKSPACE, LBM_ERR_ALIAS; an invalid
 * image writes nothing and raises LBM_ERR_BLOB in the status word. */
LBM_API int lbm_step_gnn_channel(const float* f_in, float* f_out, lbm_shape s, float tau,
                                 const float* taus, float force_x, const void* packed,
                                 double* totals, void* workspace, size_t ws_bytes,
                                 void* stream);

/* Bytes of the activations gnn_forward saves for gnn_backward
 * (1,152 bytes per node), in this order: BF16 h0, h1, h2 [N][64] (node
 * states after the encoder and each round), BF16 a0, a1 [N][64] (aggregated
 * messages of each round), FP16 AB0, AB1 [N][128] (A = W_a h | B = W_b h of
 * each round).  Each tensor [N][F] is stored in planes of 8 values: value
 * (n, f) at element ((f / 8) * N + n) * 8 + f % 8 of the tensor. */
LBM_API size_t gnn_saved_bytes(lbm_shape s);

/* Network forward on PRE-collision populations f_pre (device, shape s):
 * writes the head output y (device FP32 [10][N], N = nb*ny*nx, plane o holds
 * output o of every node) and the saved activations (device, 16-byte
 * aligned, gnn_saved_bytes(s) bytes). */
LBM_API int gnn_forward(const float* f_pre, lbm_shape s, const void* packed, void* saved,
                        float* y, void* stream);

/* ---------------------------------------------------------------------------
 * Auxiliary lattice operations
 * ------------------------------------------------------------------------- */

/* Streaming alone (Fig. 1 'Streaming Step' with periodic wrap):
 * f_out_i(x) = f_in_i(x - e_i).  Turns a stored post-collision state into
 * the pre-collision populations of the next step.  f_out != f_in. */
LBM_API int lbm_stream(const float* f_in, float* f_out, lbm_shape s, void* stream);

/* Taylor-Green initial states (as lbm_init_tgv) with per-lattice parameters:
 * params is a device double[nb][4] = (rho0, u0, kx, ky) for every lattice. */
LBM_API int lbm_init_tgv_batch(float* f, lbm_shape s, const double* params,
                               int pressure_consistent, void* stream);

/* Restriction of an m-times refined post-collision state to the coarse
 * lattice (training data of Sec. 2.4, "high-resolution LBM simulations"; the
 * scheme is this library's reading): coarse node (X, Y) of lattice b takes
 * rho, u of fine node (m X, m Y); the non-equilibrium part of the fine
 * pre-collision state, (f*_f - f^eq)/(1 - 1/tau_f), is rescaled by
 * m tau_c / tau_f (Dupuis-Chopard) and re-relaxed:
 * f*_c = f^eq + (1 - 1/tau_c) f_neq_c.  fine = (m nx, m ny, nb) of coarse.
 * tau_f / taus_f and tau_c / taus_c: scalar or per-lattice device arrays. */
LBM_API int lbm_restrict(const float* f_fine, lbm_shape fine, float* f_coarse, lbm_shape coarse,
                         int factor, float tau_f, const float* taus_f, float tau_c,
                         const float* taus_c, void* stream);

/* Restriction of an m-times refined CHANNEL (Sec. 3.1 flow, lbm_step_channel
 * geometry; training data of Sec. 2.4 for the channel network; the scheme is
 * this library's reading): m odd, fine = (m nx, m ny, nb) of coarse; coarse
 * node (X, Y) of lattice b sits where fine node (m X + (m-1)/2,
 * m Y + (m-1)/2) does, so both lattices put the walls halfway beyond their
 * outer rows.  f_fine is the fine STORED state one fine step before the
 * sampled time: the fine node's populations are pulled from it with the
 * walls (its pre-collision state at the sampled time).  With the fine force
 * F_f = (force_x_f, 0) (forces_x_f: device FP32 [nb] per lattice, else NULL;
 * the coarse force is m F_f), u = (sum f e + F_f/2)/rho:
 *   P   = (tau_f - 1/2) w_i [3 (e_i - u) + 9 (e_i . u) e_i] . F_f  (force part,
 *         equal in both lattices' units),
 *   G   = f - f^eq(rho, u) - P                          (gradient part),
 *   f*_c = f^eq + (1 - 1/tau_c) m (tau_c / tau_f) G + P,
 * the coarse post-collision state at the sampled time.  tau_f / taus_f and
 * tau_c / taus_c as in lbm_restrict.  Errors: LBM_ERR_ARG (NULL buffer, even
 * or non-positive factor, non-finite scalar force), LBM_ERR_SIZE,
 * LBM_ERR_TAU, LBM_ERR_ALIAS (f_fine and f_coarse overlap). */
LBM_API int lbm_restrict_channel(const float* f_fine, lbm_shape fine, float* f_coarse,
                                 lbm_shape coarse, int factor, float tau_f, const float* taus_f,
                                 float tau_c, const float* taus_c, float force_x_f,
                                 const float* forces_x_f, void* stream);

/* ---------------------------------------------------------------------------
 * Training (Sec. 2.4, Eq. 4)
 * ------------------------------------------------------------------------- */

/* Workspace bytes of gnn_collide_loss. */
LBM_API size_t gnn_loss_workspace_bytes(lbm_shape s);

/* Eq. 3 on the pre-collision populations f_pre with head output y
 * (gnn_forward), then the loss of Eq. 4 against f_target, read as the mean
 * over nodes x 9 of (f*_pred - f*_target)^2.  Writes loss (device double[1]),
 * dL/dy (device FP32 [10][N], nullable) and f*_pred (nullable, populations of
 * shape s).  Deterministic. */
LBM_API int gnn_collide_loss(const float* f_pre, const float* y, const float* f_target,
                             lbm_shape s, float tau, const float* taus, const void* packed,
                             double* loss, float* dy, float* f_pred, void* workspace,
                             size_t ws_bytes, void* stream);

/* Workspace bytes of gnn_backward (3 x 256 bytes per node + 80 MB of
 * per-CTA gradient partials). */
LBM_API size_t gnn_backward_workspace_bytes(lbm_shape s);

/* Reverse mode of gnn_forward: given dL/dy (device FP32 [10][N]) and the
 * activations gnn_forward saved, writes dL/dparams (device FP32, the 38,922
 * trainable values in parameter order; gradients w.r.t. the BF16-rounded
 * weights as used) and, if df_pre is not NULL, dL/df_pre (populations of
 * shape s).  Recomputes every edge pre-activation instead of storing it.
 * Deterministic (no atomics on gradients). */
LBM_API int gnn_backward(const float* f_pre, lbm_shape s, const void* packed, const void* saved,
                         const float* dy, float* dparams, float* df_pre, void* workspace,
                         size_t ws_bytes, void* stream);

/* AdamW (decoupled weight decay) on the 38,922 trainable values, step >= 1:
 * theta <- theta (1 - lr wd) - lr mhat / (sqrt(vhat) + eps). */
LBM_API int gnn_adamw(float* params, const float* grads, float* m, float* v, int64_t step,
                      float lr, float wd, float beta1, float beta2, float eps, void* stream);

/* Workspace bytes of gnn_train_step (also gnn_train_step_weighted and
 * gnn_train_step_channel): 1,152 bytes of saved activations, 80 bytes of
 * head output and its gradient, 768 bytes of backward buffers per node, the
 * pre-collision populations (9 planes of plane_stride), the per-CTA gradient
 * partials (80 MB), the loss partials and the gradient. */
LBM_API size_t gnn_train_workspace_bytes(lbm_shape s);

/* One supervised step on nb training pairs (Sec. 2.4): f_in holds the
 * coarse post-collision states at step n, f_target those at n + 1; the
 * prediction is one GNN-LBM step (stream, network, Eq. 3) of f_in; loss
 * (Eq. 4) and its gradient, then AdamW (beta = 0.9, 0.999; eps = 1e-8) on
 * params (device FP32, updated in place, with adam_m / adam_v) and a repack
 * of `packed`.  loss: device double[1] (the loss before the update); grads:
 * optional device FP32 [38922] receiving the gradient. */
LBM_API int gnn_train_step(const float* f_in, const float* f_target, lbm_shape s, float tau,
                           const float* taus, float* params, void* packed, float* adam_m,
                           float* adam_v, int64_t step, float lr, float wd, double* loss,
                           float* grads, void* workspace, size_t ws_bytes, void* stream);

/* Per-instance weights of the training loss (this library's option; the
 * paper's Eq. 4 is the plain mean): for every lattice b of the stack of
 * training pairs, D_b = the mean over its nodes x 9 of the squared one-step
 * residual of the plain method, (BGK step of f_in) - f_target (Eq. 1-2 with
 * tau / taus), and weights[b] = mean_c(D_c) / D_b, capped at 1e4 (device
 * FP32 [nb]).  Weighting the loss by them makes every instance count by its
 * error relative to the method without the network, so that pairs of the
 * developed flow weigh as much as the start-up transient (whose residuals
 * are ~1e3 larger); the weighted loss of the zero network equals the plain
 * one.  workspace: device, lbm_pair_weights_workspace_bytes(s) bytes,
 * 16-byte aligned.  nb <= 65535.  Deterministic. */
LBM_API size_t lbm_pair_weights_workspace_bytes(lbm_shape s);
LBM_API int lbm_pair_weights(const float* f_in, const float* f_target, lbm_shape s, float tau,
                             const float* taus, float* weights, void* workspace,
                             size_t ws_bytes, void* stream);

/* gnn_train_step with the loss of Eq. 4 weighted per lattice:
 * L = 1/(9 N) sum_b lat_weights[b] sum_{nodes of b, q} (f*_pred - f*_target)^2
 * (lat_weights: device FP32 [nb], e.g. from lbm_pair_weights; all 1 gives
 * gnn_train_step).  Other arguments and results as gnn_train_step. */
LBM_API int gnn_train_step_weighted(const float* f_in, const float* f_target, lbm_shape s,
                                    float tau, const float* taus, const float* lat_weights,
                                    float* params, void* packed, float* adam_m, float* adam_v,
                                    int64_t step, float lr, float wd, double* loss,
                                    float* grads, void* workspace, size_t ws_bytes,
                                    void* stream);

/* K-step rollout training step (this library's option beyond Eq. 4, which
 * is its K = 1 case): K GNN-LBM steps (stream, network, Eq. 3) from the
 * stored coarse states f_in (shape s), loss = the mean over the K steps of
 * Eq. 4 against f_targets (device: target k, the refined run's restricted
 * state after k + 1 coarse steps, at f_targets + k * 9 * plane_stride, same
 * layout as f_in), its gradient by reverse mode through all K steps (the
 * adjoint of Eq. 3 including f^eq's dependence on rho and u, the network's
 * backward with dL/df_pre, the adjoint of streaming), then AdamW and a
 * repack as gnn_train_step.  1 <= K <= 64.  Workspace:
 * gnn_rollout_workspace_bytes(s, K) bytes, 16-byte aligned (per step the
 * pre- and post-collision populations, the saved activations and y: about
 * K x 1,270 bytes per node, plus gnn_backward's workspace).  Other
 * arguments, results and errors as gnn_train_step.  Deterministic. */
LBM_API size_t gnn_rollout_workspace_bytes(lbm_shape s, int K);
LBM_API int gnn_train_step_rollout(const float* f_in, const float* f_targets, int K, lbm_shape s,
                                   float tau, const float* taus, float* params, void* packed,
                                   float* adam_m, float* adam_v, int64_t step, float lr, float wd,
                                   double* loss, float* grads, void* workspace, size_t ws_bytes,
                                   void* stream);

/* gnn_train_step for the channel network (Sec. 3.1 flow): the prediction is
 * one lbm_step_gnn_channel step of f_in (pull with halfway bounce-back,
 * network on the walled graph with the forced velocity feature, Eq. 3 with
 * Guo's source at tau tau_adj), with force (force_x, 0), or (forces_x[b], 0)
 * per lattice when forces_x (device FP32 [nb]) is not NULL; lat_weights:
 * per-lattice loss weights (as gnn_train_step_weighted) or NULL for Eq. 4.
 * Workspace: gnn_train_workspace_bytes(s).  Other arguments and results as
 * gnn_train_step; LBM_ERR_ARG also for a non-finite scalar force. */
LBM_API int gnn_train_step_channel(const float* f_in, const float* f_target, lbm_shape s,
                                   float tau, const float* taus, float force_x,
                                   const float* forces_x, const float* lat_weights, float* params,
                                   void* packed, float* adam_m, float* adam_v, int64_t step,
                                   float lr, float wd, double* loss, float* grads,
                                   void* workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Batched runs of many lattices of uneven size (serving-style workload)
 *
 * A plan packs n lattices (any sizes, each with its own tau and collision)
 * into one population buffer: the BGK lattices first, then the GNN ones, in
 * input order within each group; plane stride = lbm_batch_nodes(plan).
 * lbm_batch_run advances every lattice `steps` steps (periodic wrap inside
 * each lattice) as ONE CUDA graph launch on `stream`: per step, a batched BGK
 * kernel over all BGK lattices and, concurrently on a second branch, the GNN
 * kernels over all GNN lattices.  The graph is recorded on the first call with
 * a given (buffers, steps) and replayed afterwards.  Launch shapes are chosen
 * on first use by the autotuner (each candidate timed with CUDA events, best
 * of three; cached per kernel, SM count and size bucket; lbm_autotune_save/
 * load persist the cache as JSON): the tile shape of the batched BGK kernel
 * (128, 256 or 512 threads per block x 1, 2 or 4 nodes per thread; cache
 * value = threads * 10 + nodes per thread) and the resident CTAs per SM of
 * the GNN kernels (1 or 2).  A GNN group whose network is the MLP-only one
 * runs the fused step kernel (one CTA of 4 tile groups per SM).
 * lbm_batch_plan_create allocates the plan's device tables (cudaMalloc) and
 * two streams; lbm_batch_plan_destroy frees them.
 * ------------------------------------------------------------------------- */
enum { LBM_COLLIDE_BGK = 0, LBM_COLLIDE_GNN = 1 };

typedef struct {
  int32_t nx, ny;     /* lattice size, each >= 1, nx * ny < 2^31 */
  int32_t collision;  /* LBM_COLLIDE_BGK or LBM_COLLIDE_GNN */
  float tau;          /* relaxation time, > 1/2 */
} lbm_lattice_desc;

typedef struct lbm_batch_plan lbm_batch_plan;

/* lattices: host array of n descriptors.  *plan receives the new plan. */
LBM_API int lbm_batch_plan_create(const lbm_lattice_desc* lattices, int n, lbm_batch_plan** plan);
LBM_API void lbm_batch_plan_destroy(lbm_batch_plan* plan);

/* Total nodes of the packed buffers (their plane stride); -1 for NULL. */
LBM_API int64_t lbm_batch_nodes(const lbm_batch_plan* plan);

/* First node of every input lattice in the packed buffers (host int64[n]). */
LBM_API int lbm_batch_offsets(const lbm_batch_plan* plan, int64_t* offsets);

/* Workspace bytes lbm_batch_run needs (512 per node of the GNN lattices). */
LBM_API size_t lbm_batch_workspace_bytes(const lbm_batch_plan* plan);

/* Taylor-Green initial state of every lattice (as lbm_init_tgv); params:
 * host double[n][4] = (rho0, u0, kx, ky) per input lattice.  f: packed. */
LBM_API int lbm_batch_init_tgv(lbm_batch_plan* plan, float* f, const double* params,
                               int pressure_consistent, void* stream);

/* `steps` steps of every lattice: f_in (read only) -> f_out, with f_tmp as
 * the ping-pong buffer when steps > 1 (all packed buffers, distinct).  packed:
 * gnn_pack image, workspace: lbm_batch_workspace_bytes (both only needed if
 * a lattice uses the GNN collision).  The first call of a plan runs the
 * autotuner, whose timing runs write f_out.  Call from the device the plan
 * was created on. */
LBM_API int lbm_batch_run(lbm_batch_plan* plan, const float* f_in, float* f_out, float* f_tmp,
                          int steps, const void* packed, void* workspace, size_t ws_bytes,
                          void* stream);

/* Write / read the autotuner's cache (JSON object "kernel/smN/n2^b": choice). */
LBM_API int lbm_autotune_save(const char* path);
LBM_API int lbm_autotune_load(const char* path);

/* ---------------------------------------------------------------------------
 * GNN-LBM step without caller-provided scratch
 *
 * The paper has no counterpart: this entry point exists for callers of this
 * library that cannot allocate device memory -- a host application whose own
 * allocator owns the device memory and forbids further allocations, a
 * real-time loop that may not allocate once running, or a binding with no way
 * to hand out a device buffer.  It computes exactly what lbm_step_gnn
 * computes, taking the 512 bytes of scratch per node from a fixed 16 MiB
 * array inside the library (held on every GPU that loads the library's device
 * code, until the process exits) instead of a workspace argument; it calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   - Lattices of more than LBM_STEP_GNN_NOALLOC_MAX_NODES nodes (nb*ny*nx)
 *     are rejected with LBM_ERR_SIZE before anything is launched.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.  A failed lookup returns LBM_ERR_CUDA.
 *   - All calls share the array, which keeps the previous call's contents;
 *     nothing in it needs to start at zero.  Calls that overlap on the GPU
 *     (different streams, several host threads) race on it: serialise them.
 * Other arguments, errors and results: as lbm_step_gnn. */
#define LBM_STEP_GNN_NOALLOC_MAX_NODES 32768
LBM_API int lbm_step_gnn_noalloc(const float* f_in, float* f_out, lbm_shape s, float tau,
                                 const float* taus, const void* packed, double* totals,
                                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBMGNN_H */
