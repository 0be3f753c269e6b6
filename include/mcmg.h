/*
 * mcmg.h -- C ABI of the B300-native McMg online solve.
 *
 * McMg (multi-channel multigrid) is a learned preconditioner for the
 * heterogeneous Helmholtz equation  -Laplace u - k(x)^2 (1 - i gamma) u = f
 * (Section 2.1, Eq. helm and the sponge equation), discretised with the 5-point
 * (2D) or 7-point (3D) finite-difference stencil (Eq. FDM_stencil).  A medium
 * is set up once (Algorithm 1: nonlinear setup networks produce cached
 * per-level features a_l, s_l); every later V-cycle (Algorithm 2) is linear in
 * its input residual and runs as fixed-coefficient stencil and channel-mixing
 * kernels.  The outer iteration is restarted flexible GMRES preconditioned by
 * one V-cycle per step (Section 3.3, Table 2 "GMRES+McMg").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Grids: shape n[0..dim-1] slowest axis first ((Ny, Nx) in 2D, (Nz, Ny, Nx)
 *   in 3D), x fastest.  The unit domain gives h = 1 / n[0].  All operators act
 *   on the h^2-scaled system (the equation multiplied by h^2); relative
 *   residuals are unchanged by that scaling.
 * - Complex numbers are interleaved (re, im): "c64" = two float32,
 *   "c128" = two float64.
 * - Multi-channel fields are channels-last: element (node p, channel c) of a
 *   C-channel field lives at index p * C + c.
 * - A batch of nrhs fields is stored contiguously, field k at offset
 *   k * nodes * C elements.
 * - "dev" pointers are CUDA device pointers on the context's device, 16-byte
 *   aligned; "host" pointers are ordinary host memory.  The caller owns every
 *   buffer it passes; the library never frees caller memory.  A handle owns its
 *   features, weights and workspaces until mcmg_destroy.
 * - Every call returns an mcmg_status.  Errors never cross the ABI as
 *   exceptions; mcmg_last_error() gives a thread-local message for the last
 *   failing call.  MCMG_ERR_CUDA means the CUDA context may be unusable.
 * - "stream" arguments are cudaStream_t values passed as void* (NULL = the
 *   legacy default stream).  Calls that take a stream are asynchronous on it.
 */
#ifndef MCMG_H
#define MCMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCMG_MAX_LEVELS 8

typedef struct mcmg_ctx_s* mcmg_ctx;
typedef struct mcmg_handle_s* mcmg_handle;

typedef enum {
  MCMG_OK = 0,
  MCMG_PENDING = 1,            /* mcmg_poll: the request has not finished   */
  MCMG_ERR_ARG = -1,           /* a NULL or out-of-range argument            */
  MCMG_ERR_SHAPE = -2,         /* grid or channel shape not supported        */
  MCMG_ERR_OOM = -3,           /* device memory or the HBM budget exhausted  */
  MCMG_ERR_CUDA = -4,          /* a CUDA runtime error                       */
  MCMG_ERR_NOT_CONVERGED = -5, /* max_iters reached above tolerance          */
  MCMG_ERR_TIMEOUT = -6,       /* a bounded wait ran out                     */
  MCMG_ERR_NUMERIC = -7,       /* NaN / Inf met in a residual                */
  MCMG_ERR_BUSY = -8           /* the server queue is full                   */
} mcmg_status;

typedef enum {
  MCMG_FP32 = 0,   /* channel mixing and stencils in FP32 (FFMA)               */
  MCMG_BF16 = 1,   /* channel mixing on tcgen05 tensor cores, BF16 operands,
                      FP32 accumulation; stencil arithmetic stays FP32        */
  MCMG_FP32_TC = 2 /* FP32-accurate channel mixing on tcgen05 tensor cores:
                      every FP32 operand split into two TF32 parts and three
                      TF32 products accumulated in FP32 (levels with C_l in
                      {8, 16}; other levels as MCMG_FP32)                     */
} mcmg_precision;

/* The medium: wave speed on the grid plus the sponge layer (Section 2.1).
 * The sponge occupies sponge_width cells on each side inside the grid; its
 * damping is gamma = gamma_max * (depth / sponge_width)^2 with depth the
 * distance in cells into the layer, the largest over the axes.              */
typedef struct {
  int dim;               /* 2 or 3                                           */
  int n[3];              /* grid shape, slowest axis first                   */
  const double* c;       /* host, wave speed per node (n[0]*...*n[dim-1])    */
  int sponge_width;      /* cells                                             */
  double gamma_max;      /* peak damping                                      */
} mcmg_medium;

/* Weights of one McMg model (Sections 3.1-3.2).  `blob` is a host array of
 * float64 in the order below; complex tensors take two doubles (re, im) per
 * entry, real tensors one.  C_l = channels[l], C' = channels[l+1],
 * T = 2*dim+1 stencil taps (centre, -x, +x, -y, +y, -z, +z), T3 = 3^dim
 * transfer taps indexed ((oz+1)*3+(oy+1))*3+(ox+1), and a mixing matrix
 * M[co][ci] maps input channel ci to output channel co.
 *
 *   f_lift weight  real [2*C_0][2][T3],  bias real [2*C_0]
 *   for l = 0 .. levels-1:
 *     W_l       complex [T][C_l][C_l]        neural PDE operator stencil
 *     K_A       complex [C_l][C_l]
 *     K_S       complex [C_l][C_l]
 *     W^(i)     complex [nu_pre+nu_post][C_l][C_l]   smoother, one per step
 *     f_s       real [2C_l][2C_l][T3], bias real [2C_l]
 *     if l < levels-1:
 *       R       complex [T3][C'][C_l]         restriction (stride-2 conv)
 *       P       complex [T3][C_l][C']         prolongation (transposed conv)
 *       f_a     real [2C'][2C_l][T3], bias real [2C']
 *   g_lift   complex [C_0]
 *   g_proj   complex [C_0]
 *
 * Setup features (Algorithm 1): the setup networks f_lift, f_s, f_a are one
 * 3^d convolution + bias + exact GELU each, on real channel pairs; the input
 * is m = ((kh)^2, (kh)^2 gamma).  Channel 0 of a_l, s_l is replaced by
 * feat_sl times the classical shifted-Laplacian coefficients
 * a = -(sl_shift) q_l, s = 1/(2 dim 4^(-l) + a) when feat_sl != 0, where q_1 =
 * (kh)^2 (1 - i gamma) and q_{l+1} is its full-weighting restriction; every
 * other entry is feat_eps times the network output.                         */
typedef struct {
  int levels;                          /* L, 1 .. MCMG_MAX_LEVELS            */
  int channels[MCMG_MAX_LEVELS];       /* each in {1, 2, 4, 8, 16, 32, 64}    */
  int nu_pre[MCMG_MAX_LEVELS];         /* pre-smoothing steps per level      */
  int nu_post[MCMG_MAX_LEVELS];        /* post-smoothing steps (last = 0)    */
  double feat_sl, feat_eps;            /* feature blend, see above           */
  double sl_shift_re, sl_shift_im;     /* (beta1, beta2) of Eq. csl_shift    */
  int precision;                       /* mcmg_precision                     */
  const double* blob;                  /* host, see layout above             */
  size_t blob_len;                     /* number of doubles in blob          */
} mcmg_weights;

typedef struct {
  double tol;        /* relative residual target ||f - A u|| / ||f||          */
  int restart_m;     /* Krylov vectors per FGMRES cycle                       */
  int max_iters;     /* cap on V-cycle applications (0 = 20 * n[0])          */
  int nrhs;          /* right-hand sides solved together (independent systems)*/
  int flags;         /* MCMG_SOLVE_* bits                                     */
  void* stream;      /* cudaStream_t the solve runs on (NULL = the handle's
                        own stream); the call still returns only when done.
                        The solve reads f and u only after all work enqueued
                        on this stream (NULL: on the legacy default stream)
                        before the call; mcmg_submit marks that point at
                        submission and the server orders the request after it */
} mcmg_solve_opts;

#define MCMG_SOLVE_STATIONARY 1  /* u <- u + MG(f - A u) instead of FGMRES
                                    (Eq. mcmg_iteration); restart_m is
                                    ignored; mcmg_solve only (the server
                                    refuses it with MCMG_ERR_ARG)             */
#define MCMG_SOLVE_BORN 2        /* Born+McMg: u <- u + MG(G(f - A u)) with G
                                    = (-Delta_h - k0^2)^{-1} applied by FFT
                                    with the discrete-Laplacian symbol
                                    (Appendix, Born-series variant and
                                    discrete Green operator; periodic modes).
                                    q0 = (k0 h)^2: Re q0 halfway between the
                                    extremes of Re q, Im q0 = -max|q - Re q0|.
                                    restart_m ignored; mcmg_solve only.  The
                                    first Born solve on a handle builds an FFT
                                    plan (cuFFT allocates its workspace outside
                                    the HBM budget).                          */

typedef struct {
  int iters;                 /* V-cycle applications (max over the rhs)      */
  int restarts;              /* FGMRES cycles started                        */
  double rel_residual;       /* true FP64 ||f - A u|| / ||f|| (max over rhs) */
  double t_solve_s;          /* wall time of the solve                       */
  int converged;             /* 1 when every rhs met tol                     */
} mcmg_solve_info;

/* ---- context -------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory all handles of this context may hold (0 = no bound); setup
 * and the server's admission refuse work beyond it with MCMG_ERR_OOM.        */
mcmg_status mcmg_ctx_create(int device, size_t hbm_budget_bytes, mcmg_ctx* out);
mcmg_status mcmg_ctx_destroy(mcmg_ctx ctx);
/* Bytes currently held by the context's handles.                            */
mcmg_status mcmg_ctx_memory(mcmg_ctx ctx, size_t* used_bytes);

/* ---- setup (Algorithm 1) -------------------------------------------------- */

/* Build a handle for one medium: uploads the medium, computes q = (kh)^2
 * (1 - i gamma) with k = omega / c and h = 1/n[0], runs the setup networks on
 * the device and caches a_l, s_l for every level, and converts the weights to
 * the device layouts.  Grid sizes must be divisible by 2^(levels-1) with the
 * coarsest grid at least 2 nodes per axis, and the grid below 2^31 nodes
 * (else MCMG_ERR_SHAPE).  Blocks until the setup is complete.                */
mcmg_status mcmg_setup(mcmg_ctx ctx, const mcmg_medium* medium, double omega,
                       const mcmg_weights* weights, mcmg_handle* out);
mcmg_status mcmg_destroy(mcmg_handle h);

/* ---- V-cycle (Algorithm 2) ------------------------------------------------ */

/* e = MG(r) for nrhs scalar residuals.  r, e: dev c64 [nrhs][nodes];
 * they may not overlap.  Asynchronous on `stream`.                           */
mcmg_status mcmg_vcycle(mcmg_handle h, const void* r_dev_c64, void* e_dev_c64,
                        int nrhs, void* stream);

/* ---- solve ---------------------------------------------------------------- */

/* Solve A u = f for opts->nrhs right-hand sides with FGMRES(restart_m)
 * preconditioned by one V-cycle per step (or the stationary iteration with
 * MCMG_SOLVE_STATIONARY).  f: dev c128 [nrhs][nodes]; u: dev c128, holds the
 * initial guess on entry (zero = the paper's setting) and the solution on
 * return.  Krylov orthogonalisation, the Hessenberg least-squares update and
 * the true residual run in FP64 on the device.  Synchronous.  Returns
 * MCMG_ERR_NOT_CONVERGED (with info filled) when max_iters is reached.       */
mcmg_status mcmg_solve(mcmg_handle h, const void* f_dev_c128, void* u_dev_c128,
                       const mcmg_solve_opts* opts, mcmg_solve_info* info);

/* As mcmg_solve, with f and u in HOST memory: the library copies f to the
 * device and u back (the copies are part of the call).                      */
mcmg_status mcmg_solve_host(mcmg_handle h, const void* f_host_c128, void* u_host_c128,
                            const mcmg_solve_opts* opts, mcmg_solve_info* info);

/* ---- serving -------------------------------------------------------------- */

/* Queue a solve on the context's server.  f, u as in mcmg_solve (device
 * memory, kept alive by the caller until the ticket completes).  The server
 * admits queued requests while the HBM budget allows, advances every admitted
 * request one FGMRES step per round, and overlaps their work on the device.
 * Returns MCMG_ERR_BUSY when the queue is full.  Thread-safe.                */
mcmg_status mcmg_submit(mcmg_ctx ctx, mcmg_handle h, const void* f_dev_c128,
                        void* u_dev_c128, const mcmg_solve_opts* opts, uint64_t* ticket);
/* Cross-request batching of the server (not in the paper; serving): with it
 * on (the default), the requests whose V-cycles are due in the same round and
 * whose handles share weights and level layout run those V-cycles as one
 * cohort, every smoothing step and residual of a level one tensor-core launch
 * over all their fields (each field with its own grid and medium); results
 * are the same as alone.  enable: 1 on, 0 off, -1 unchanged.  rounds /
 * members (may be NULL): cohort V-cycles run so far and the requests they
 * held, summed.  Thread-safe.                                               */
mcmg_status mcmg_server_batching(mcmg_ctx ctx, int enable, uint64_t* rounds, uint64_t* members);

/* MCMG_PENDING until the request finished; then its final status, with info
 * filled.  A finished ticket is forgotten after the first non-pending poll.  */
mcmg_status mcmg_poll(mcmg_ctx ctx, uint64_t ticket, mcmg_solve_info* info);
/* Run the server until every submitted request has finished.                */
mcmg_status mcmg_drain(mcmg_ctx ctx);

/* ---- single steps of the path (used by tests and diagnostics) ------------- */

/* Wait for the device and read the handle's error word: 0 = fine; non-zero
 * means a bounded wait inside a kernel ran out (1: a tensor-core MMA, 2: a
 * bulk copy of mixing weights; that kernel released its resources and
 * skipped its output).  mcmg_solve reports the same condition as
 * MCMG_ERR_TIMEOUT.                                                          */
mcmg_status mcmg_device_error(mcmg_handle h, int* code);

/* y = h^2 A x (Eq. FDM_stencil with the sponge).  fp64 = 0: x, y dev c64;
 * fp64 = 1: x, y dev c128.  nrhs fields.                                     */
mcmg_status mcmg_apply_A(mcmg_handle h, const void* x_dev, void* y_dev, int fp64,
                         int nrhs, void* stream);

/* Copy the cached feature of `level` (0-based): which = 0 -> a_l, 1 -> s_l,
 * into out_dev (dev c64 [nodes_l][C_l]).                                     */
mcmg_status mcmg_get_feature(mcmg_handle h, int level, int which, void* out_dev);

/* r_1 = g_lift(r):  r dev c64 [nrhs][nodes], r1 dev c64 [nrhs][nodes][C_0].  */
mcmg_status mcmg_lift(mcmg_handle h, const void* r_dev, void* r1_dev, int nrhs, void* stream);
/* e = g_proj(e_1):  e1 dev c64 [nrhs][nodes][C_0], e dev c64 [nrhs][nodes].  */
mcmg_status mcmg_project(mcmg_handle h, const void* e1_dev, void* e_dev, int nrhs, void* stream);

/* One smoothing step of Section 3.2 on `level`:
 *   e_out = e_in + S^(step)(r - A_l(e_in)),   step 0-based into W^(i).
 * e_in = NULL means e_in = 0.  All dev c64 [nrhs][nodes_l][C_l]; e_out may
 * not overlap e_in.                                                          */
mcmg_status mcmg_smooth(mcmg_handle h, int level, int step, const void* r_dev,
                        const void* e_in_dev, void* e_out_dev, int nrhs, void* stream);

/* The residual of Algorithm 2 on `level`:  t = r - A_l(e)  (the input of the
 * restriction).  r, e, t: dev c64 [nrhs][nodes_l][C_l]; t may not overlap e.
 * Enqueued on `stream`.                                                      */
mcmg_status mcmg_residual(mcmg_handle h, int level, const void* r_dev, const void* e_dev,
                          void* t_dev, int nrhs, void* stream);

/* r_coarse = R_l(r - A_l(e)) for level < levels-1.  r, e: dev c64
 * [nrhs][nodes_l][C_l]; r_coarse: dev c64 [nrhs][nodes_{l+1}][C_{l+1}].       */
mcmg_status mcmg_residual_restrict(mcmg_handle h, int level, const void* r_dev,
                                   const void* e_dev, void* r_coarse_dev, int nrhs,
                                   void* stream);

/* e += P_l(e_coarse) for level < levels-1.                                   */
mcmg_status mcmg_prolong_add(mcmg_handle h, int level, const void* e_coarse_dev,
                             void* e_dev, int nrhs, void* stream);

/* The background Green operator of the Born-series variant (Appendix, the
 * discrete Green operator; Eq. discrete_symbol), in place:
 *   x <- IDFT( DFT(x) / (sum_a 4 sin^2(pi m_a / N_a) - q0) ),
 * the discrete Laplacian's symbol on periodic modes, q0 = (k0 h)^2 with
 * Re q0 halfway between the extremes of Re q and Im q0 = -max|q - Re q0|.
 * x: dev c128 [nodes_0] (grid order, x fastest).  The DFT is this library's
 * own FFT, so every axis must be a power of two of at most 4096 cells
 * (else MCMG_ERR_SHAPE).  Enqueued on `stream`; the first call on a handle
 * prepares the symbols (synchronous).                                        */
mcmg_status mcmg_apply_G(mcmg_handle h, void* x_dev, void* stream);

/* Raw coarse-basis response (Eq. coarse_basis, Section 3.4):
 *   Psi = g_proj(P_1 P_2 ... P_level (delta_alpha)),
 * delta_alpha the one-hot latent field at node `node` (linear index on that
 * level's grid, x fastest) and channel `channel` of `level` (1 <= level <
 * levels).  out_dev: dev c64 [nodes_0].  Enqueued on `stream`; uses the
 * handle's V-cycle workspace, so it must not overlap an mcmg_vcycle or
 * single-step call on another stream.  MCMG_ERR_ARG for an out-of-range
 * level, node or channel.                                                     */
mcmg_status mcmg_coarse_basis(mcmg_handle h, int level, long long node, int channel,
                              void* out_dev, void* stream);

/* Classical Gram-Schmidt with one re-orthogonalisation (CGS2) against k
 * basis vectors, FP64 accumulation:  h = V^H w, w -= V h (twice, h summed),
 * norm = ||w||.  V: dev c64 [k][n]; w: dev c64 [n], updated in place;
 * h_host: host c128 [k]; norm_host: host double.  Synchronous.               */
mcmg_status mcmg_cgs2(mcmg_handle h, const void* V_dev, int k, size_t n, void* w_dev,
                      double* h_host, double* norm_host);

/* mcmg_cgs2 for callers that cannot allocate device memory.  The paper has no
 * counterpart; this entry point exists for callers that must not call
 * cudaMalloc: code running under another framework's fixed memory budget or
 * allocator, and call sites that cannot afford the device-wide
 * synchronisation that cudaMalloc / cudaFree can cause.  It allocates nothing:
 * its scratch (about 1.2 MB) is a static device array that every GPU which
 * loads this library holds until the process exits.  Same arguments and
 * results as mcmg_cgs2, with k at most 64 (larger k returns MCMG_ERR_ARG), no
 * handle, and the caller's stream (NULL = legacy default stream).  V and w
 * must be device memory of the current device (else MCMG_ERR_ARG).  The call
 * is synchronous: it copies the results to the host and synchronises the
 * stream before returning, so it must not be issued on a stream that is being
 * captured.  The first call on a device looks up the array's device address
 * with that device current.  All calls share the one array, so calls that
 * overlap on the GPU race; nothing carries over from one call to the next.   */
mcmg_status mcmg_cgs2_noalloc(const void* V_dev, int k, size_t n, void* w_dev,
                              double* h_host, double* norm_host, void* stream);

/* Kernel shapes of the V-cycle operations (tuning and test access; the
 * paper has no counterpart).  op: 0 smoothing step, 1 residual r - A_l(e),
 * 2 restriction R_l, 3 prolongation P_l (ops 2 and 3 exist for
 * level < levels-1).  Each has several interchangeable kernels and thread
 * shapes with the same results up to FP32 rounding order; setup times them
 * on every level and keeps the fastest.  The last three shapes of ops 2 and
 * 3 run on the tensor cores of tensor-core handles (MCMG_BF16,
 * MCMG_FP32_TC), with that handle's mixing precision: count-3 is the
 * transfer per parity class, where its input has 16, 32 or 64 channels (a
 * restriction also 8) and its output as many, half or twice as many;
 * count-2 (prolongation only) computes all parity classes of a coarse tile
 * at once, where C_{l+1} is 16, 32 or 64, C_l = C_{l+1} or C_{l+1} / 2 and
 * 2^d x 2 C_l <= 256; count-1 (restriction only) stages the fine lines in
 * shared memory, where C_l = 8, C_{l+1} is 8 or 16 and the coarse x extent
 * is a multiple of 32.
 *   mcmg_kernel_shape_count: number of shapes of op (indices 0 .. count-1),
 *                            0 for an unknown op.
 *   mcmg_get_kernel_shape:   the shape `level` uses for op (*shape).
 *   mcmg_set_kernel_shape:   use `shape` from now on, or -1 for setup's
 *                            choice; MCMG_ERR_SHAPE (nothing changed) if the
 *                            shape cannot run on this level's channels.
 * A change applies to later calls; captured V-cycle graphs are re-captured
 * at their next use.  Call only while no solve or request on this handle is
 * in flight.  Op 0 on a level that runs on the tensor cores (BF16 handles,
 * C_l >= 8) is not affected.                                                  */
int mcmg_kernel_shape_count(int op);
mcmg_status mcmg_get_kernel_shape(mcmg_handle h, int level, int op, int* shape);
mcmg_status mcmg_set_kernel_shape(mcmg_handle h, int level, int op, int shape);

/* Measurement aid (the paper has no counterpart): the FP32 fused
 * multiply-add rate of the current device in TFLOP/s, timed with CUDA events
 * on `stream` over a loop of independent FFMA chains (about 5 ms of work).
 * It is the roofline denominator of the CUDA-core FP32 kernels.  Synchronous. */
mcmg_status mcmg_fp32_ffma_tflops(void* stream, double* tflops);

/* Number of kernel launches the library has issued in this process (a
 * captured graph counts as its kernel nodes).  For launch accounting.        */
uint64_t mcmg_kernel_launches(void);

/* Thread-local message of the last failing call on this thread.              */
const char* mcmg_last_error(void);
/* Library version string.                                                    */
const char* mcmg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MCMG_H */
