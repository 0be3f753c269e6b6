// Internal declarations shared by the McMg CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mcmg.h"

namespace mcmg {

// ---------------------------------------------------------------- complex ---
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a b with every rounding explicit, so that kernels computing the same
// product (the lift in its own kernel and inside the level-0 step) agree bit
// for bit whatever the compiler contracts elsewhere
__device__ __forceinline__ float2 cmul_rn(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)),
                     __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__host__ __device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}

// ------------------------------------------------------- launch counting ---
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ----------------------------------------------------------------- errors ---
void set_error(const char* fmt, ...);
mcmg_status cuda_fail(cudaError_t e, const char* what);

#define MCMG_CUDA(call)                                              \
  do {                                                               \
    cudaError_t _e = (call);                                         \
    if (_e != cudaSuccess) return ::mcmg::cuda_fail(_e, #call);      \
  } while (0)

#define MCMG_CHECK_LAUNCH(what)                                      \
  do {                                                               \
    ::mcmg::count_launch();                                          \
    cudaError_t _e = cudaGetLastError();                             \
    if (_e != cudaSuccess) return ::mcmg::cuda_fail(_e, what);       \
  } while (0)

#define MCMG_TRY(expr)                                               \
  do {                                                               \
    mcmg_status _s = (expr);                                         \
    if (_s != MCMG_OK) return _s;                                    \
  } while (0)

// ------------------------------------------------------------------- grid ---
struct Grid {
  int d;            // 2 or 3
  int nx, ny, nz;   // nz = 1 in 2D
  __host__ __device__ long long nodes() const { return (long long)nx * ny * nz; }
  __host__ __device__ Grid coarse() const { return Grid{d, nx / 2, ny / 2, d == 3 ? nz / 2 : 1}; }
};

// Read-only per-level state: features and weights.  Mixing matrices are
// stored transposed, M^T[ci][co], so consecutive output channels are
// contiguous.
struct Level {
  Grid g;
  int C = 0, Cn = 0;          // channels here and on the next coarser level
  int nu_pre = 0, nu_post = 0;
  float2* a = nullptr;        // [nodes][C]
  float2* s = nullptr;        // [nodes][C]
  float2* Wt = nullptr;       // [T][C][C]
  float2* KAt = nullptr;      // [C][C]
  float2* KSt = nullptr;      // [C][C]
  float2* Wsmt = nullptr;     // [nsteps][C][C]
  float2* Rt = nullptr;       // [T3][C][Cn]
  float2* Pt = nullptr;       // [T3][Cn][C]
  bool use_ts = false;        // smoothing step and residual on tcgen05, TMEM A operands
  int ts_prec = -1;           // MCMG_BF16 or MCMG_FP32_TC when use_ts
  const uint4* ts_mats = nullptr;  // weight matrices in the operand layout of ts_prec
  // restriction (Cn x C) and prolongation (C x Cn) tap matrices in the same
  // layout, for the tensor-core transfers (null where those do not apply)
  const uint4* ts_R = nullptr;
  const uint4* ts_P = nullptr;
  // per coarse source offset s in {0,1}^d: the prolongation matrices of all
  // 2^d parity classes stacked (zero where a class does not read s)
  const uint4* ts_Pb = nullptr;
  // restriction from 8 channels, per stage (o_y, o_z): [R_o | R_o' | R_o'']
  // over o_x = -1, 0, +1 (Cn x 24), for the line-staged kernel
  const uint4* ts_R3 = nullptr;
  // signatures of the arithmetic of one smoothing step (stencil, K_A, K_S,
  // W^(i)) and of the residual (stencil, K_A), with precision and C: launches
  // of different handles may be batched when these agree
  uint64_t ssig[2 * 8 + 1] = {};
  uint64_t rsig = 0;
  // CUDA-core kernel shape per operation in use (0 smoothing step, 1 residual,
  // 2 restriction, 3 prolongation) and the autotuner's choice
  int shape[4] = {-1, -1, -1, -1};
  int tuned[4] = {-1, -1, -1, -1};
  int* err = nullptr;         // device view of the handle's error word
};

// One field of a batched tensor-core launch: its own grid and features
// (fields of several requests at the same level, same weights).  first: the
// first tile (item) of the field in the launch, a prefix sum of tiles.
struct TsField {
  const float2* r;
  const float2* e_in;
  float2* out;
  const float2* a;
  const float2* s;
  long long nodes;
  int nx, ny, nz, tiles, first;
};

// tensor-core smoothing step and residual with A operands in tensor memory
// (kernels_ts.cu); mode as launch_smooth
bool ts_supported(int C, int prec);
mcmg_status launch_smooth_ts(const Level& L, int step, const float2* r, const float2* e_in,
                             float2* out, int mode, int nrhs, cudaStream_t st);
// The same over nf fields given by descriptors in device memory (fields_dev,
// their host copy fields_host for the shapes): L supplies the weights, C and
// the dimension; every field's e_in is null exactly when has_e is false.
mcmg_status launch_smooth_ts_fields(const Level& L, int step, const TsField* fields_dev,
                                    const TsField* fields_host, int nf, bool has_e, int mode,
                                    cudaStream_t st);
// Level 0 of a one-field V-cycle with the lift folded into the step's read
// of r and, when z_cell is set (smoothing steps), the projection into its
// write: r_cell and z_cell are device cells holding the scalar input and
// output addresses.  Available where ts_fused_io_supported(L).
bool ts_fused_io_supported(const Level& L);
mcmg_status launch_smooth_ts_io(const Level& L, int step, const float2* const* r_cell,
                                const float2* lift, const float2* e_in, float2* out,
                                float2* const* z_cell, const float2* proj, int mode,
                                cudaStream_t st);
// complex C x C matrix -> its real 2C x 2C block form as a B operand: BF16
// (4C^2 values), or TF32 hi and lo halves (2 * 4C^2 floats)
void pack_ts_bf16(const float2* Mc, int C, uint16_t* out);
void pack_ts_tf32(const float2* Mc, int C, float* out);

// tensor-core restriction (restrict_ true: r_c = R t) and prolongation
// (e += P e_c) of level L (kernels_xts.cu): available on tensor-core levels
// whose input side has at least 16 channels.  src, dst: nrhs fields each.
bool xts_supported(const Level& L, bool restrict_);
mcmg_status launch_transfer_ts(const Level& L, bool restrict_, const float2* src, float2* dst,
                               int nrhs, cudaStream_t st);
// complex Cout x Cin matrix [co][ci] -> real block form (2 Cout x 2 Cin) as
// a B operand: BF16 (4 Cout Cin values) or TF32 hi and lo (2 * 4 Cout Cin)
void pack_ts_rect(const float2* Mc, int Cout, int Cin, bool tf32, void* out);
// block prolongation (kernels_xts.cu): all parity classes of a coarse tile
// in one pass; available where xts_block_pair(d, C_n, C) holds
bool xts_block_pair(int d, int Cn, int C);
bool xts_block_supported(const Level& L);
mcmg_status launch_prolong_block_ts(const Level& L, const float2* ec, float2* e, int nrhs,
                                    cudaStream_t st);
// restriction from 8 channels with the fine lines staged in shared memory
// (kernels_xts.cu): tensor-core levels with C = 8, C_n in {8, 16} and a
// coarse x extent that is a multiple of 32
bool xts_lines_pair(int C, int Cn, int cx);
bool xts_lines_supported(const Level& L);
mcmg_status launch_restrict_lines_ts(const Level& L, const float2* src, float2* dst, int nrhs,
                                     cudaStream_t st);

// Launchers used by the V-cycle (kernels_vcycle.cu), asynchronous on `st`.
// mode 0: e_out = e_in + S^(step)(r - A e_in); mode 1: e_out = r - A e_in.
mcmg_status launch_smooth(const Level& L, int step, const float2* r, const float2* e_in,
                          float2* e_out, int mode, int nrhs, cudaStream_t st);
mcmg_status launch_restrict(const Level& L, const float2* t, float2* rc, int nrhs,
                            cudaStream_t st);
// Time the thread shapes of the CUDA-core smoothing kernel on level L and keep
// the fastest per mode (r, e, out: scratch fields of nodes * C elements).
mcmg_status autotune_smooth(Level& L, float2* r, float2* e, float2* out, cudaStream_t st);
// Transfer shapes of level L (fine, coarse: scratch fields), timed at setup.
mcmg_status autotune_transfer(Level& L, float2* fine, float2* coarse, cudaStream_t st);
// Number of kernel shapes of an operation (0 smoothing step, 1 residual,
// 2 restriction, 3 prolongation), and whether one can run on level L.
int kernel_shape_count(int op);
bool kernel_shape_valid(const Level& L, int op, int shape);
mcmg_status launch_prolong_add(const Level& L, const float2* ec, float2* e, int nrhs,
                               cudaStream_t st);
mcmg_status launch_lift(const float2* r, const float2* lift, float2* r1, int C, long long nodes,
                        int nrhs, cudaStream_t st);
mcmg_status launch_project(const float2* e1, const float2* proj, float2* e, int C,
                           long long nodes, int nrhs, cudaStream_t st);
mcmg_status launch_lift_gather(const float2* const* srcs, const float2* lift, float2* r1, int C,
                               long long nodes, int count, cudaStream_t st);
mcmg_status launch_project_scatter(const float2* e1, const float2* proj, float2* const* dsts, int C,
                                   long long nodes, int count, cudaStream_t st);

// helmholtz (kernels_helm.cu)
mcmg_status launch_make_q(const double* c_dev, double omega, int width, double gamma_max,
                          const Grid& g, float2* q32, double2* q64, cudaStream_t st);
mcmg_status launch_apply_A32(const float2* q, const float2* x, float2* y, const Grid& g,
                             int nrhs, cudaStream_t st);
mcmg_status launch_apply_A64(const double2* q, const double2* x, double2* y, const Grid& g,
                             int nrhs, cudaStream_t st);
// complex64 x, FP64 arithmetic, complex128 y
// w = A x for the Arnoldi step: x complex64, w complex double-float
// (float4 per node: re hi, re lo, im hi, im lo), coefficients from qdf
mcmg_status launch_apply_A_arnoldi(const float4* qdf, const float2* x, float4* w, const Grid& g,
                                   cudaStream_t st);
// qdf from q64 (once, at setup)
mcmg_status launch_make_qdf(const double2* q64, float4* qdf, const Grid& g, cudaStream_t st);
mcmg_status launch_residual64(const double2* q, const double2* f, const double2* x, double2* r,
                              double* part, int nblk, const Grid& g, int nrhs, cudaStream_t st);

// setup (kernels_setup.cu)
mcmg_status launch_setup_input(const double2* q64, float* m, const Grid& g, cudaStream_t st);
mcmg_status launch_conv3_gelu(const float* in, int cin, float* out, int cout, const float* w,
                              const float* b, const Grid& gin, int stride, cudaStream_t st);
mcmg_status launch_fw_restrict_q(const double2* qf, double2* qc, const Grid& gf, cudaStream_t st);
mcmg_status launch_assemble_features(const float* net_a, const float* net_s, const double2* ql,
                                     float2* a, float2* s, int C, const Grid& g, int level,
                                     double feat_sl, double feat_eps, double beta_re,
                                     double beta_im, cudaStream_t st);

// Device allocations tracked against a context budget.
struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
};

}  // namespace mcmg

struct mcmg_handle_s;

namespace mcmg {

// Per-execution V-cycle workspace (one per synchronous user / server request).
struct VWork {
  int nrhs = 0;
  float2* r[MCMG_MAX_LEVELS] = {};
  float2* e[MCMG_MAX_LEVELS] = {};
  float2* e2[MCMG_MAX_LEVELS] = {};
  float2* t[MCMG_MAX_LEVELS] = {};
  cudaGraphExec_t graph = nullptr;   // the level sequence for nrhs fields, captured once
  float2* e1 = nullptr;              // buffer holding e_1 after the graph
  unsigned long long graph_kernels = 0;  // kernel nodes in the graph
  // graphs of the level sequence for fewer fields (batched solves), by count
  std::map<int, std::pair<cudaGraphExec_t, unsigned long long>> sub;
  unsigned shape_gen = 0;            // handle's shape generation the graphs were captured at
  // one-field V-cycles with the lift and projection folded into level 0:
  // cells[0] = the scalar input r, cells[1] = the scalar output e, written
  // before each launch of a graph captured that way (graph_fused)
  float2** cells = nullptr;
  bool graph_fused = false;
  DevArena arena;
};

mcmg_status vwork_create(mcmg_handle_s* h, int nrhs, VWork** out);
void vwork_destroy(mcmg_handle_s* h, VWork* w);
// e = MG(r) on stream st using workspace w.
mcmg_status vcycle_run(mcmg_handle_s* h, VWork* w, const float2* r, float2* e, int nrhs,
                       cudaStream_t st);
// Batched V-cycle over `count` <= w->nrhs fields: field k reads srcs[k] and
// writes dsts[k] (device arrays of device pointers).
mcmg_status vcycle_run_batch(mcmg_handle_s* h, VWork* w, const float2* const* srcs,
                             float2* const* dsts, int count, cudaStream_t st);

// Resumable FGMRES(m) for one right-hand side (krylov.cu).
struct Krylov;
mcmg_status krylov_create(mcmg_handle_s* h, int m, Krylov** out, bool own_vcycle_work = true);
void krylov_destroy(mcmg_handle_s* h, Krylov* k);
// Start a solve of A u = f (device c128).  Enqueues work on st.
mcmg_status krylov_begin(Krylov* k, const double2* f, double2* u, const mcmg_solve_opts& o,
                         cudaStream_t st);
// Advance: if the last enqueued work has finished, read its results and
// enqueue the next stage.  *done = 1 when the solve has finished.
// blocking = true waits for the enqueued work instead of polling.
mcmg_status krylov_advance(Krylov* k, bool blocking, int* done);
void krylov_info(const Krylov* k, mcmg_solve_info* info, mcmg_status* final_status);
int krylov_m(const Krylov* k);
// The stationary iteration u <- u + MG(f - A u), synchronous, on a Krylov workspace.
// Born+McMg: u <- u + MG(G(f - A u)), synchronous, on a Krylov workspace.
mcmg_status born_run(Krylov* k, const double2* f, double2* u, const mcmg_solve_opts& o,
                     cudaStream_t st, mcmg_solve_info* info, mcmg_status* final_status);
mcmg_status stationary_run(Krylov* k, const double2* f, double2* u, const mcmg_solve_opts& o,
                           cudaStream_t st, mcmg_solve_info* info, mcmg_status* final_status);
cudaStream_t krylov_stream(const Krylov* k);   // the solve's private stream
// FGMRES(m) for several right-hand sides of one medium: every round batches
// the V-cycles of all members that need one into a single launch per level;
// Arnoldi, restarts and convergence stay per member.
struct KrylovBlock;
mcmg_status block_create(mcmg_handle_s* h, int m, int nb, KrylovBlock** out);
void block_destroy(mcmg_handle_s* h, KrylovBlock* b);
mcmg_status block_begin(KrylovBlock* b, const double2* f, double2* u, const mcmg_solve_opts& o);
// As krylov_advance, for the whole block (one round per call).
mcmg_status block_advance(KrylovBlock* b, bool blocking, int* done);
// The same round in two halves around a V-cycle run by the caller:
// block_poll reads the last round's results (once its work has finished;
// *count = -1 while it runs) and stages, on the block's stream, the device
// pointer arrays of the *count members that need a V-cycle; after the caller
// has run that V-cycle (block_vcycle_io: workspace, source and destination
// arrays), block_after_vcycle enqueues their Arnoldi steps.
mcmg_status block_poll(KrylovBlock* b, bool blocking, int* done, int* count);
mcmg_status block_after_vcycle(KrylovBlock* b);
void block_vcycle_io(KrylovBlock* b, VWork** w, const float2* const** srcs, float2* const** dsts);
void block_info(const KrylovBlock* b, mcmg_solve_info* info, mcmg_status* final_status);
int block_size(const KrylovBlock* b);
cudaStream_t block_stream(const KrylovBlock* b);   // the block solve's private stream
int block_m(const KrylovBlock* b);
// CGS2 on caller buffers (used by mcmg_cgs2).
mcmg_status cgs2_once(mcmg_handle_s* h, const float2* V, int k, long long n, float2* w,
                      double* h_host, double* norm_host, cudaStream_t st);

mcmg_status dev_alloc(mcmg_handle_s* h, DevArena& a, void** p, size_t bytes);
void arena_free(mcmg_handle_s* h, DevArena& a);

}  // namespace mcmg

struct mcmg_ctx_s;

struct mcmg_handle_s {
  mcmg_ctx_s* ctx = nullptr;
  int device = 0;
  int L = 0;
  int precision = MCMG_FP32;
  mcmg::Grid g0;
  float2* q32 = nullptr;        // (kh)^2 (1 - i gamma), c64 [nodes]
  double2* q64 = nullptr;       // same, c128
  // (2d - Re q, Im q) as double-float pairs (hi, lo, hi, lo): the Arnoldi
  // operator's coefficients without FP64 arithmetic per application
  float4* qdf = nullptr;
  float2* lift = nullptr;       // [C0]
  float2* proj = nullptr;       // [C0]
  mcmg::Level lv[MCMG_MAX_LEVELS];
  mcmg::DevArena arena;         // features, weights
  mcmg::VWork* work = nullptr;  // for mcmg_vcycle / mcmg_solve
  mcmg::Krylov* kry = nullptr;  // for mcmg_solve, one right-hand side
  mcmg::KrylovBlock* blk = nullptr;  // for mcmg_solve, several right-hand sides
  cudaStream_t stream = nullptr;
  std::mutex mu;                // serialises synchronous use of work / kry
  int* err_host = nullptr;      // error word, mapped pinned (bounded waits that ran out)
  int* err_dev = nullptr;
  unsigned shape_gen = 0;       // bumped when a smoothing shape is overridden
  uint64_t wsig = 0;            // signature of the weights and level layout (batching key)
  // Born-series variant (born.cu): per-axis Laplacian symbols and FFT
  // twiddles, q0
  bool born_ready = false;
  double* born_sym[3] = {};
  double2* born_tw[3] = {};
  double born_q0r = 0.0, born_q0i = 0.0;
};

namespace mcmg {
// Green operator of the Born-series variant (born.cu): symbols, twiddles and
// q0 once per handle; x <- G x in place (x: c128 [nodes_0]) on st.
mcmg_status born_prepare(mcmg_handle_s* h);
mcmg_status born_apply_G(mcmg_handle_s* h, double2* x, cudaStream_t st);
void born_release(mcmg_handle_s* h);
}  // namespace mcmg
