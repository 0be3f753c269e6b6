// The discrete Helmholtz operator with the sponge layer (Section 2.1,
// Eq. helm, the sponge equation and Eq. FDM_stencil), in the h^2-scaled form
//   (h^2 A u)_p = 2d u_p - sum_{neighbours q} u_q - q_p u_p,
//   q_p = (k_p h)^2 (1 - i gamma_p),  k = omega / c,  h = 1 / n[0],
// with zero values outside the grid.  Pure streaming kernels: one thread per
// node, neighbours through L1/L2.
#include "mcmg_internal.cuh"

namespace mcmg {

__global__ void k_make_q(const double* __restrict__ c, double omega, double h, int width,
                         double gamma_max, Grid g, float2* __restrict__ q32,
                         double2* __restrict__ q64) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long N = g.nodes();
  if (n >= N) return;
  int x = (int)(n % g.nx);
  long long rest = n / g.nx;
  int y = (int)(rest % g.ny);
  int z = (int)(rest / g.ny);
  int idx[3] = {x, y, z};
  int ext[3] = {g.nx, g.ny, g.nz};
  double depth = 0.0;
  for (int a = 0; a < g.d; ++a) {
    double i = idx[a];
    double d1 = fmax(fmax((double)width - i, i - (double)(ext[a] - 1 - width)), 0.0);
    depth = fmax(depth, d1);
  }
  double gam = width > 0 ? gamma_max * (depth / width) * (depth / width) : 0.0;
  double kh = omega * h / c[n];
  double kh2 = kh * kh;
  double2 q = make_double2(kh2, -kh2 * gam);
  q64[n] = q;
  q32[n] = make_float2((float)q.x, (float)q.y);
}

mcmg_status launch_make_q(const double* c_dev, double omega, int width, double gamma_max,
                          const Grid& g, float2* q32, double2* q64, cudaStream_t st) {
  long long N = g.nodes();
  int threads = 256;
  unsigned blocks = (unsigned)((N + threads - 1) / threads);
  // the paper's unit domain: h = 1 / n[0], n[0] the slowest axis
  double h = 1.0 / (g.d == 3 ? g.nz : g.ny);
  k_make_q<<<blocks, threads, 0, st>>>(c_dev, omega, h, width, gamma_max, g, q32, q64);
  MCMG_CHECK_LAUNCH("make_q");
  return MCMG_OK;
}

template <typename T>
struct CTraits;
template <>
struct CTraits<float2> {
  using R = float;
  static __device__ __forceinline__ float2 mk(R a, R b) { return make_float2(a, b); }
};
template <>
struct CTraits<double2> {
  using R = double;
  static __device__ __forceinline__ double2 mk(R a, R b) { return make_double2(a, b); }
};

// y = h^2 A x for nrhs fields (gridDim.y = rhs index); X is the input type,
// C2 the arithmetic and output type (complex64 in -> complex128 out promotes).
template <typename C2, typename X2 = C2>
__global__ void k_apply_A(const C2* __restrict__ q, const X2* __restrict__ x, C2* __restrict__ y,
                          Grid g) {
  using R = typename CTraits<C2>::R;
  long long N = g.nodes();
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  size_t off = (size_t)blockIdx.y * N;
  const X2* xx = x + off;
  int ix = (int)(n % g.nx);
  long long rest = n / g.nx;
  int iy = (int)(rest % g.ny);
  int iz = (int)(rest / g.ny);
  X2 u = xx[n];
  C2 qq = q[n];
  R dg = (R)(2 * g.d);
  // (2d - q) u
  R re = (dg - qq.x) * (R)u.x + qq.y * (R)u.y;
  R im = (dg - qq.x) * (R)u.y - qq.y * (R)u.x;
  long long sxy = (long long)g.nx * g.ny;
  if (ix > 0) { X2 v = xx[n - 1]; re -= (R)v.x; im -= (R)v.y; }
  if (ix < g.nx - 1) { X2 v = xx[n + 1]; re -= (R)v.x; im -= (R)v.y; }
  if (iy > 0) { X2 v = xx[n - g.nx]; re -= (R)v.x; im -= (R)v.y; }
  if (iy < g.ny - 1) { X2 v = xx[n + g.nx]; re -= (R)v.x; im -= (R)v.y; }
  if (g.d == 3) {
    if (iz > 0) { X2 v = xx[n - sxy]; re -= (R)v.x; im -= (R)v.y; }
    if (iz < g.nz - 1) { X2 v = xx[n + sxy]; re -= (R)v.x; im -= (R)v.y; }
  }
  y[off + n] = CTraits<C2>::mk(re, im);
}

mcmg_status launch_apply_A32(const float2* q, const float2* x, float2* y, const Grid& g,
                             int nrhs, cudaStream_t st) {
  long long N = g.nodes();
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)nrhs);
  k_apply_A<float2><<<grid, 256, 0, st>>>(q, x, y, g);
  MCMG_CHECK_LAUNCH("apply_A32");
  return MCMG_OK;
}

mcmg_status launch_apply_A64(const double2* q, const double2* x, double2* y, const Grid& g,
                             int nrhs, cudaStream_t st) {
  long long N = g.nodes();
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)nrhs);
  k_apply_A<double2><<<grid, 256, 0, st>>>(q, x, y, g);
  MCMG_CHECK_LAUNCH("apply_A64");
  return MCMG_OK;
}

// ---- w = h^2 A x for a complex64 x in double-float arithmetic --------------
// The Arnoldi product of the Krylov loop.  FP64 arithmetic runs at a small
// fraction of the FP32 rate on this part, so the operator is evaluated as
// double-float (an unevaluated sum hi + lo of two FP32 values, 48 significand
// bits) and the result stays double-float: (2d - Re q) and Im q come split
// from a table made once at setup, their products with the FP32 x are exact
// up to the lo * lo term (Dekker's product through the FMA), sums use Knuth's
// two-sum.  Relative error ~2^-44 of the largest term, far below the FP32
// rounding already in x; no FP64 instruction per node.
namespace {
struct DFh {
  float hi, lo;
};
__device__ __forceinline__ DFh dfh_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ void dfh_add(DFh& x, DFh y) {
  const DFh s = dfh_two_sum(x.hi, y.hi);
  const float lo = __fadd_rn(__fadd_rn(s.lo, x.lo), y.lo);
  const float hi = __fadd_rn(s.hi, lo);
  x = {hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}
__device__ __forceinline__ void dfh_add(DFh& x, float y) { dfh_add(x, DFh{y, 0.f}); }
// a * (bh + bl) for an FP32 a
__device__ __forceinline__ DFh dfh_mul(float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  return {p, __fmaf_rn(a, bl, __fmaf_rn(a, bh, -p))};
}
__device__ __forceinline__ DFh dfh_split(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
}  // namespace

__global__ void k_make_qdf(const double2* __restrict__ q, float4* __restrict__ qdf, int d,
                           long long n) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double2 qq = q[p];
  const DFh a = dfh_split((double)(2 * d) - qq.x);   // 2d - Re q
  const DFh b = dfh_split(qq.y);                      // Im q
  qdf[p] = make_float4(a.hi, a.lo, b.hi, b.lo);
}

mcmg_status launch_make_qdf(const double2* q64, float4* qdf, const Grid& g, cudaStream_t st) {
  const long long n = g.nodes();
  k_make_qdf<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(q64, qdf, g.d, n);
  MCMG_CHECK_LAUNCH("make_qdf");
  return MCMG_OK;
}

// IT: index type (32-bit below 2^31 nodes)
template <typename IT>
__global__ void __launch_bounds__(256) k_apply_A_arnoldi(const float4* __restrict__ qdf,
                                                         const float2* __restrict__ x,
                                                         float4* __restrict__ y, Grid g) {
  const IT N = (IT)g.nodes();
  const IT n = (IT)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const IT rest = n / g.nx;
  const int ix = (int)(n - rest * g.nx);
  const int iy = (int)(rest % g.ny);
  const int iz = (int)(rest / g.ny);
  const float2 u = x[n];
  const float4 c = qdf[n];
  // (2d - q) u = (a ur + b ui) + i (a ui - b ur), a = 2d - Re q, b = Im q
  DFh re = dfh_mul(u.x, c.x, c.y), im = dfh_mul(u.y, c.x, c.y);
  dfh_add(re, dfh_mul(u.y, c.z, c.w));
  dfh_add(im, dfh_mul(-u.x, c.z, c.w));
  const IT sxy = (IT)g.nx * g.ny;
  auto sub = [&](float2 v) {
    dfh_add(re, -v.x);
    dfh_add(im, -v.y);
  };
  if (ix > 0) sub(x[n - 1]);
  if (ix < g.nx - 1) sub(x[n + 1]);
  if (iy > 0) sub(x[n - g.nx]);
  if (iy < g.ny - 1) sub(x[n + g.nx]);
  if (g.d == 3) {
    if (iz > 0) sub(x[n - sxy]);
    if (iz < g.nz - 1) sub(x[n + sxy]);
  }
  y[n] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

mcmg_status launch_apply_A_arnoldi(const float4* qdf, const float2* x, float4* w, const Grid& g,
                                   cudaStream_t st) {
  const long long N = g.nodes();
  const unsigned grid = (unsigned)((N + 255) / 256);
  if (N < (1ll << 31))
    k_apply_A_arnoldi<int><<<grid, 256, 0, st>>>(qdf, x, w, g);
  else
    k_apply_A_arnoldi<long long><<<grid, 256, 0, st>>>(qdf, x, w, g);
  MCMG_CHECK_LAUNCH("apply_A_arnoldi");
  return MCMG_OK;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r = f - A x in FP64; part[(rhs * nblk + block) * 2 + {0, 1}] = partial sums
// of |r|^2 and |f|^2 over the block's grid-stride range (fixed order).
__global__ void __launch_bounds__(256) k_residual64(const double2* __restrict__ q,
                                                    const double2* __restrict__ f,
                                                    const double2* __restrict__ x,
                                                    double2* __restrict__ r,
                                                    double* __restrict__ part, Grid g) {
  long long N = g.nodes();
  size_t off = (size_t)blockIdx.y * N;
  const double2* xx = x + off;
  double rr = 0.0, ff = 0.0;
  long long sxy = (long long)g.nx * g.ny;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    int ix = (int)(n % g.nx);
    long long rest = n / g.nx;
    int iy = (int)(rest % g.ny);
    int iz = (int)(rest / g.ny);
    double2 u = xx[n], qq = q[n];
    double dg = 2.0 * g.d;
    double re = (dg - qq.x) * u.x + qq.y * u.y;
    double im = (dg - qq.x) * u.y - qq.y * u.x;
    if (ix > 0) { double2 v = xx[n - 1]; re -= v.x; im -= v.y; }
    if (ix < g.nx - 1) { double2 v = xx[n + 1]; re -= v.x; im -= v.y; }
    if (iy > 0) { double2 v = xx[n - g.nx]; re -= v.x; im -= v.y; }
    if (iy < g.ny - 1) { double2 v = xx[n + g.nx]; re -= v.x; im -= v.y; }
    if (g.d == 3) {
      if (iz > 0) { double2 v = xx[n - sxy]; re -= v.x; im -= v.y; }
      if (iz < g.nz - 1) { double2 v = xx[n + sxy]; re -= v.x; im -= v.y; }
    }
    double2 fv = f[off + n];
    double2 rv = make_double2(fv.x - re, fv.y - im);
    r[off + n] = rv;
    rr += rv.x * rv.x + rv.y * rv.y;
    ff += fv.x * fv.x + fv.y * fv.y;
  }
  __shared__ double s_rr[8], s_ff[8];
  rr = warp_sum(rr);
  ff = warp_sum(ff);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s_rr[w] = rr; s_ff[w] = ff; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += s_rr[i]; b += s_ff[i]; }
    size_t k = ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 2;
    part[k] = a;
    part[k + 1] = b;
  }
}

mcmg_status launch_residual64(const double2* q, const double2* f, const double2* x, double2* r,
                              double* part, int nblk, const Grid& g, int nrhs, cudaStream_t st) {
  dim3 grid((unsigned)nblk, (unsigned)nrhs);
  k_residual64<<<grid, 256, 0, st>>>(q, f, x, r, part, g);
  MCMG_CHECK_LAUNCH("residual64");
  return MCMG_OK;
}

}  // namespace mcmg
