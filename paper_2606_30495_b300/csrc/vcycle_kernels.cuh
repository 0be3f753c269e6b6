// Kernel parameter blocks and device helpers shared by the V-cycle kernel
// translation units (kernels_vcycle.cu, kernels_smooth_rt.cu,
// kernels_transfer_rt.cu).
#pragma once
#include <utility>

#include "mcmg_internal.cuh"

namespace mcmg {

// Programmatic dependent launch.  The V-cycle's kernels are launched so that
// each may start while its predecessor drains: a kernel first lets its own
// dependents launch, reads only setup-time data (weights, features) before
// pdl_wait(), and touches fields written by earlier kernels only after it.
// pdl_wait() returns once every prerequisite grid has completed and its
// memory is visible; both are no-ops in a kernel launched without the
// attribute.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define MCMG_LAUNCH_PDL(kernel, grid, block, smem, st, ...)                      \
  do {                                                                          \
    cudaError_t _e = ::mcmg::launch_pdl(kernel, grid, block, smem, st, __VA_ARGS__); \
    if (_e != cudaSuccess) return ::mcmg::cuda_fail(_e, #kernel);              \
  } while (0)

template <int C, int TN_, int CO_>
struct Tile {
  static constexpr int CO = CO_;
  static constexpr int CG = C / CO;
  static constexpr int G = 256 / CG;
  static constexpr int TN = TN_;
  static constexpr int NB = G * TN;
};

static constexpr size_t kMaxSmem = 227 * 1024;

// Register-tiled K-split geometry (k_smooth_rt): CG = C / CO channel groups,
// KS = C / KQ K-groups and NG node groups fill a 256-thread block; a block
// covers NB = NG * TN nodes.
template <int C, int TN, int CO, int KQ>
struct RtTile {
  static constexpr int CG = CO <= C && C % CO == 0 ? C / CO : 0;
  static constexpr int KS = KQ <= C && C % KQ == 0 ? C / KQ : 0;
  static constexpr int NG = CG * KS > 0 && CG * KS <= 256 ? 256 / (CG * KS) : 0;
  static constexpr int NB = NG * TN;
  static constexpr bool valid = NG >= 1 && CG * KS * NG == 256;
};

struct SmoothParams {
  const float2* r;
  const float2* e_in;   // null: e = 0 (first pre-smoothing step)
  float2* e_out;
  const float2* a;
  const float2* s;
  const float2* Wt;     // [T][C][C]
  const float2* KAt;
  const float2* KSt;
  const float2* Wst;    // W^(i) for this step, [C][C]
  int nx, ny, nz;
  long long nodes;
  int* err;             // handle's error word (bounded waits that ran out)
};

__device__ __forceinline__ void node_xyz(long long n, int nx, int ny, int& x, int& y, int& z) {
  x = (int)(n % nx);
  long long rest = n / nx;
  y = (int)(rest % ny);
  z = (int)(rest / ny);
}

// The same for node indices below 2^31 (every grid; checked at setup).
__device__ __forceinline__ void node_xyz32(int n, int nx, int ny, int& x, int& y, int& z) {
  const int rest = n / nx;
  x = n - rest * nx;
  y = rest % ny;
  z = rest / ny;
}

// CO consecutive complex values (one float2, or two float4 for CO = 4).
template <int CO>
__device__ __forceinline__ void ldc(const float2* __restrict__ q, float2 (&v)[CO]) {
  if constexpr (CO == 1) {
    v[0] = __ldg(q);
  } else {
    static_assert(CO == 4, "CO is 1 or 4");
    const float4* q4 = reinterpret_cast<const float4*>(q);
    const float4 a = __ldg(q4), b = __ldg(q4 + 1);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
  }
}

template <int CO>
__device__ __forceinline__ void stc(float2* q, const float2 (&v)[CO]) {
  if constexpr (CO == 1) {
    q[0] = v[0];
  } else {
    float4* q4 = reinterpret_cast<float4*>(q);
    q4[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    q4[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
  }
}

struct TransferParams {
  const float2* src;
  float2* dst;
  const float2* Wt;    // [T3][cin][CO]
  int cin;
  int fx, fy, fz;      // fine grid
  int cx, cy, cz;      // coarse grid
  long long src_nodes, dst_nodes;
};

template <int CI, int CO, int TN, int CV, int KQ>
struct XTile {
  static constexpr int CG = CV <= CO && CO % CV == 0 ? CO / CV : 0;
  static constexpr int KS = KQ <= CI && CI % KQ == 0 ? CI / KQ : 0;
  static constexpr int NG = CG * KS > 0 && CG * KS <= 256 ? 256 / (CG * KS) : 0;
  static constexpr int NB = NG * TN;
  static constexpr bool valid = NG >= 1 && CG * KS * NG == 256 && CI % 2 == 0;
};

// Register-tiled smoothing step (kernels_smooth_rt.cu): shape (tn, co, kq)
// on C channels in D dimensions; MCMG_ERR_SHAPE if it is not built.
// bulk: the variant that stages each mixing matrix in shared memory with
// bulk asynchronous copies.
mcmg_status smooth_rt_launch(const SmoothParams& p, int C, int D, int mode, int tn, int co, int kq,
                             bool bulk, int nrhs, cudaStream_t st);
// Shared memory of the register-tiled smoothing step (0: the shape cannot run).
size_t rt_smem(int C, int D, int tn, int co, int kq, bool bulk);
// Register-tiled restriction (restrict_) or prolongation-add between Cf fine
// and Cc coarse channels (kernels_transfer_rt.cu).
mcmg_status transfer_rt_launch(const TransferParams& p, int Cf, int Cc, int D, bool restrict_,
                               int tn, int cv, int kq, int nrhs, cudaStream_t st);

}  // namespace mcmg
