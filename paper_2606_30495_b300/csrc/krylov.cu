// Flexible GMRES(m) on the device (the outer iteration of GMRES+McMg,
// Section 3.3 and Table 2, in Saad's flexible right-preconditioned form).
//
// Precision split: the Krylov basis V and the preconditioned vectors Z are
// complex64 (the V-cycle's input and output precision).  The Arnoldi work
// vector w = A z_j is formed in double-float from the complex64 z_j (an
// unevaluated sum hi + lo of two FP32 values per real number, 48 significand
// bits: FP64-class on the FP32 units, which on this part run many times the
// FP64 rate) and stays double-float through Gram-Schmidt; every inner
// product, update and norm accumulates in double-float and the block
// partials in FP64.  The Hessenberg matrix, Givens rotations and the
// least-squares solve are FP64 on the host, fed by the step's inner products
// (mirrored to mapped memory).  The solution u and the true residual f - A u
// (at every restart) are complex128.
// Forming A z in FP32 would lose up to ||A|| ||z|| / ||A z|| times the FP32
// rounding, which for an indefinite Helmholtz operator and a preconditioned
// z is large enough to separate the implicit and true residuals.
// Orthogonalisation is classical Gram-Schmidt with one re-orthogonalisation
// (CGS2) in one sweep over the basis: the sweep returns h1 = V^H w and the
// Gram row V^H v_j, the second pass h2 = V^H (w - V h1) = -(V^H V - I) h1 is
// formed from the kept Gram matrix, and one update applies h1 + h2.  The
// basis is complex64, so V^H V - I (its storage rounding) is what the second
// pass has to remove; the sweep's double-float dots are far below it.
// (mcmg_cgs2 keeps the explicit two-pass form for its callers.)
//
// The solve is a resumable state machine so that a server can interleave many
// solves on separate streams: every stage enqueues device work, records an
// event, and the host reads the few scalars it needs (inner products, norms)
// from mapped pinned memory once the event has completed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <type_traits>

#include "mcmg_internal.cuh"

namespace mcmg {

constexpr int KV = 8;         // vectors per block in the multi-dot
constexpr int RED_T = 256;    // threads per reduction block

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
__device__ __forceinline__ void store_w(float2* p, double re, double im) {
  *p = make_float2((float)re, (float)im);
}
__device__ __forceinline__ void store_w(double2* p, double re, double im) {
  *p = make_double2(re, im);
}

// ---- double-float arithmetic ----------------------------------------------
// FP64 arithmetic on this part runs at a small fraction of the FP32 rate, so
// the Gram-Schmidt inner products and updates carry FP64-class precision as
// double-float numbers: an unevaluated sum hi + lo of two FP32 values (48
// significand bits).  Products of an FP32 value and a double-float are exact
// up to the lo * lo term through the FMA (Dekker's product); sums use Knuth's
// two-sum.  The correctly rounded intrinsics keep the compiler from fusing
// or reassociating the error-free transformations.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// x += y
__device__ __forceinline__ void df_add(DF& x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  const float lo = __fadd_rn(__fadd_rn(s.lo, x.lo), y.lo);
  const float hi = __fadd_rn(s.hi, lo);
  x = {hi, __fsub_rn(lo, __fsub_rn(hi, s.hi))};
}
// a * (bh + bl) for an FP32 a
__device__ __forceinline__ DF df_mul(float a, float bh, float bl) {
  const float p = __fmul_rn(a, bh);
  return {p, __fmaf_rn(a, bl, __fmaf_rn(a, bh, -p))};
}
__device__ __forceinline__ DF df_from(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ DF df_from(float v) { return {v, 0.f}; }
// real and imaginary part of a complex w as double-float: float2 and double2
// values are converted, float4 ones (re hi, re lo, im hi, im lo) already are
__device__ __forceinline__ DF df_re(float2 w) { return {w.x, 0.f}; }
__device__ __forceinline__ DF df_im(float2 w) { return {w.y, 0.f}; }
__device__ __forceinline__ DF df_re(double2 w) { return df_from(w.x); }
__device__ __forceinline__ DF df_im(double2 w) { return df_from(w.y); }
__device__ __forceinline__ DF df_re(float4 w) { return {w.x, w.y}; }
__device__ __forceinline__ DF df_im(float4 w) { return {w.z, w.w}; }
__device__ __forceinline__ double df_to(DF x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ DF df_shfl_xor(DF x, int o) {
  return {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}
// x^2 for a double-float x (the lo^2 term, 2^-48 relative, dropped)
__device__ __forceinline__ DF df_sq(DF x) { return df_mul(x.hi, x.hi, __fmul_rn(2.f, x.lo)); }

// part[(bx * ktot + i) * 2 + {0,1}] = sum over this block's range of conj(v_i) w,
// v_i = V[i * ldv + .] for i < k, v_k = w when ktot = k + 1.  Double-float
// accumulation; block partials in a fixed order, written as FP64.
template <typename WT>
__global__ void __launch_bounds__(RED_T) k_multidot(const float2* __restrict__ V, long long ldv,
                                                    int k, int ktot, const WT* __restrict__ w,
                                                    long long n, double* __restrict__ part) {
  const int i0 = blockIdx.y * KV;
  DF ar[KV], ai[KV];
#pragma unroll
  for (int i = 0; i < KV; ++i) ar[i] = ai[i] = DF{0.f, 0.f};
  // two elements per iteration, every load issued before the arithmetic, so
  // that twice as many loads are in flight per thread
  const long long stride = (long long)gridDim.x * RED_T;
  auto accumulate = [&](const WT wv, const float2 (&vv)[KV]) {
    const DF wx = df_re(wv), wy = df_im(wv);
#pragma unroll
    for (int i = 0; i < KV; ++i) {
      const int ii = i0 + i;
      if (ii < k) {
        const float2 v = vv[i];
        // conj(v) w = (vx wx + vy wy) + i (vx wy - vy wx)
        df_add(ar[i], df_mul(v.x, wx.hi, wx.lo));
        df_add(ar[i], df_mul(v.y, wy.hi, wy.lo));
        df_add(ai[i], df_mul(v.x, wy.hi, wy.lo));
        df_add(ai[i], df_mul(-v.y, wx.hi, wx.lo));
      } else if (ii < ktot) {  // |w|^2
        df_add(ar[i], df_sq(wx));
        df_add(ar[i], df_sq(wy));
      }
    }
  };
  long long p = (long long)blockIdx.x * RED_T + threadIdx.x;
  for (; p + stride < n; p += 2 * stride) {
    const WT wa = w[p], wb = w[p + stride];
    float2 va[KV], vb[KV];
#pragma unroll
    for (int i = 0; i < KV; ++i) {
      const int ii = i0 + i < k ? i0 + i : 0;
      va[i] = V[(long long)ii * ldv + p];
      vb[i] = V[(long long)ii * ldv + p + stride];
    }
    accumulate(wa, va);
    accumulate(wb, vb);
  }
  if (p < n) {
    const WT wa = w[p];
    float2 va[KV];
#pragma unroll
    for (int i = 0; i < KV; ++i) {
      const int ii = i0 + i < k ? i0 + i : 0;
      va[i] = V[(long long)ii * ldv + p];
    }
    accumulate(wa, va);
  }
  // 2 KV values per thread: through shared memory, warp q sums values 2q, 2q+1
  static_assert(2 * KV == 2 * (RED_T / 32), "one warp per pair of values");
  __shared__ DF sh[2 * KV][RED_T];
#pragma unroll
  for (int i = 0; i < KV; ++i) {
    sh[2 * i][threadIdx.x] = ar[i];
    sh[2 * i + 1][threadIdx.x] = ai[i];
  }
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int val = 2 * wid + c;
    DF acc = sh[val][lane];
#pragma unroll
    for (int q = 1; q < RED_T / 32; ++q) df_add(acc, sh[val][lane + 32 * q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) df_add(acc, df_shfl_xor(acc, o));
    const int vec = i0 + val / 2;
    if (lane == 0 && vec < ktot) part[((size_t)blockIdx.x * ktot + vec) * 2 + (val & 1)] = df_to(acc);
  }
}

// One pass over the basis for Arnoldi step j (double-float w): for every
// basis vector i <= j, a_i = conj(v_i) w and b_i = conj(v_i) v_j (a row of the
// Gram matrix V^H V), and |w|^2.  Partials part[(bx * width + idx) * 2 + {0,1}]
// with width = 2j + 3: idx i -> a_i, j + 1 -> |w|^2, j + 2 + i -> b_i.
// a_i and |w|^2 accumulate in double-float.  b_i only has to resolve the
// basis' storage rounding (~6e-8) to well below it: each thread sums its few
// dozen products in FP32 (error ~1e-13 of the unit norms), and the thread
// partials are added in double-float.  Each warp sums its values by shuffles
// and warp partials are added in warp order, so the result does not depend
// on scheduling.
__global__ void __launch_bounds__(RED_T, 2) k_multidot_gram(const float2* __restrict__ V, long long ldv,
                                                         int j, const float4* __restrict__ w,
                                                         long long n, double* __restrict__ part) {
  const int k = j + 1, width = 2 * j + 3;
  const int i0 = blockIdx.y * KV;
  DF ar[KV], ai[KV];
  float br[KV], bi[KV];
#pragma unroll
  for (int i = 0; i < KV; ++i) {
    ar[i] = ai[i] = DF{0.f, 0.f};
    br[i] = bi[i] = 0.f;
  }
  const float2* vj = V + (long long)j * ldv;
  auto accumulate = [&](const float4 wv, const float2 uj, const float2 (&vv)[KV]) {
    const DF wx{wv.x, wv.y}, wy{wv.z, wv.w};
#pragma unroll
    for (int i = 0; i < KV; ++i) {
      const int ii = i0 + i;
      if (ii < k) {
        const float2 v = vv[i];
        // conj(v) w = (vx wx + vy wy) + i (vx wy - vy wx)
        df_add(ar[i], df_mul(v.x, wx.hi, wx.lo));
        df_add(ar[i], df_mul(v.y, wy.hi, wy.lo));
        df_add(ai[i], df_mul(v.x, wy.hi, wy.lo));
        df_add(ai[i], df_mul(-v.y, wx.hi, wx.lo));
        // conj(v) v_j in FP32 per thread
        br[i] = __fmaf_rn(v.x, uj.x, __fmaf_rn(v.y, uj.y, br[i]));
        bi[i] = __fmaf_rn(v.x, uj.y, __fmaf_rn(-v.y, uj.x, bi[i]));
      } else if (ii == k) {  // |w|^2
        df_add(ar[i], df_sq(wx));
        df_add(ar[i], df_sq(wy));
      }
    }
  };
  // two elements per iteration, every load issued before the arithmetic
  const long long stride = (long long)gridDim.x * RED_T;
  long long p = (long long)blockIdx.x * RED_T + threadIdx.x;
  for (; p + stride < n; p += 2 * stride) {
    const float4 wa = w[p], wb = w[p + stride];
    const float2 ua = vj[p], ub = vj[p + stride];
    float2 va[KV], vb[KV];
#pragma unroll
    for (int i = 0; i < KV; ++i) {
      const int ii = i0 + i < k ? i0 + i : 0;
      va[i] = V[(long long)ii * ldv + p];
      vb[i] = V[(long long)ii * ldv + p + stride];
    }
    accumulate(wa, ua, va);
    accumulate(wb, ub, vb);
  }
  if (p < n) {
    const float4 wa = w[p];
    const float2 ua = vj[p];
    float2 va[KV];
#pragma unroll
    for (int i = 0; i < KV; ++i) {
      const int ii = i0 + i < k ? i0 + i : 0;
      va[i] = V[(long long)ii * ldv + p];
    }
    accumulate(wa, ua, va);
  }
  // 4 KV values per thread: warp sums by shuffles, then the warps in order
  __shared__ DF sh[4 * KV][RED_T / 32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto warp_reduce = [&](DF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) df_add(v, df_shfl_xor(v, o));
    return v;
  };
#pragma unroll
  for (int i = 0; i < KV; ++i) {
    const DF r0 = warp_reduce(ar[i]), r1 = warp_reduce(ai[i]);
    const DF r2 = warp_reduce(DF{br[i], 0.f}), r3 = warp_reduce(DF{bi[i], 0.f});
    if (lane == 0) {
      sh[4 * i][wid] = r0;
      sh[4 * i + 1][wid] = r1;
      sh[4 * i + 2][wid] = r2;
      sh[4 * i + 3][wid] = r3;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 * KV) {
    const int val = threadIdx.x;
    DF acc = sh[val][0];
#pragma unroll
    for (int q = 1; q < RED_T / 32; ++q) df_add(acc, sh[val][q]);
    const int ii = i0 + val / 4, comp = val & 1;
    const bool second = (val & 2) != 0;       // b_i
    int idx = -1;
    if (!second && ii <= k) idx = ii;          // a_i, or |w|^2 at ii == k
    if (second && ii < k) idx = j + 2 + ii;
    if (idx >= 0) part[((size_t)blockIdx.x * width + idx) * 2 + comp] = df_to(acc);
  }
}

// Second Gram-Schmidt pass from the Gram matrix (one block, FP64):
// red[0..j] = h1 = V^H w, red[j+1] = |w|^2, red[j+2+i] = v_i^H v_j.  Row j of
// G = V^H V is stored (Gd[j][i] = v_i^H v_j, i <= j), then
// h2 = V^H (w - V h1) = -(G - I) h1, which the two-pass form would compute
// from a second sweep over the basis.  d1 / d2 (and the host mirror) get h1
// with |w|^2 and h2; dsum = h1 + h2 is the update's coefficient vector.
__global__ void k_gram_correct(const double2* __restrict__ red, int j, int ldg,
                               double2* __restrict__ Gd, double2* __restrict__ d1,
                               double2* __restrict__ d2, double2* __restrict__ dsum,
                               double2* __restrict__ mir, int m) {
  const int t = threadIdx.x;
  for (int i = t; i <= j; i += blockDim.x) Gd[(size_t)j * ldg + i] = red[j + 2 + i];
  __syncthreads();
  for (int l = t; l <= j; l += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int q = 0; q <= j; ++q) {
      // G[l][q] = v_l^H v_q: stored as row max(l, q)
      double2 g;
      if (l <= q) {
        g = Gd[(size_t)q * ldg + l];
      } else {
        const double2 c = Gd[(size_t)l * ldg + q];
        g = make_double2(c.x, -c.y);
      }
      if (l == q) g.x -= 1.0;
      const double2 h = red[q];
      sr += g.x * h.x - g.y * h.y;
      si += g.x * h.y + g.y * h.x;
    }
    const double2 h1 = red[l], h2 = make_double2(-sr, -si);
    d1[l] = h1;
    d2[l] = h2;
    dsum[l] = make_double2(h1.x + h2.x, h1.y + h2.y);
    if (mir) {
      mir[l] = h1;
      mir[m + 2 + l] = h2;
    }
  }
  if (t == 0) {
    d1[j + 1] = red[j + 1];
    if (mir) mir[j + 1] = red[j + 1];
  }
}

// Block-wide sum of two doubles (fixed order: per-thread strided partials,
// warp shuffles, then warps in order).  Result valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double a, double b) {
  __shared__ double sh[2][RED_T / 32];
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][wid] = a; sh[1][wid] = b; }
  __syncthreads();
  double ra = 0.0, rb = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < RED_T / 32; ++q) { ra += sh[0][q]; rb += sh[1][q]; }
  return make_double2(ra, rb);
}

// out[i] = sum_b part[(b * width + i) * 2 + {0,1}]; one block per output i.
// out_host (mapped host memory, may be null) receives a copy.
__global__ void __launch_bounds__(RED_T) k_reduce_parts(const double* __restrict__ part, int nblk,
                                                        int width, double2* __restrict__ out,
                                                        double2* out_host) {
  const int i = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += RED_T) {
    a += part[((size_t)q * width + i) * 2];
    b += part[((size_t)q * width + i) * 2 + 1];
  }
  const double2 r = block_sum2(a, b);
  if (threadIdx.x == 0) {
    out[i] = r;
    if (out_host) out_host[i] = r;
  }
}

// w -= sum_{i<k} h_i V_i (double-float accumulation per element, the
// difference taken in w's precision); part[bx] = sum |w|^2 over the block's
// elements.  h is split into double-float pairs once per block, in dynamic
// shared memory (k * 16 bytes).
template <typename WT>
__global__ void __launch_bounds__(RED_T) k_update(const float2* __restrict__ V, long long ldv, int k,
                                                  const double2* __restrict__ hc,
                                                  WT* __restrict__ w, long long n,
                                                  double* __restrict__ part) {
  extern __shared__ DF hs[];   // [k][2]
  for (int i = threadIdx.x; i < k; i += RED_T) {
    const double2 hh = hc[i];
    hs[2 * i] = df_from(hh.x);
    hs[2 * i + 1] = df_from(hh.y);
  }
  __syncthreads();
  DF nn{0.f, 0.f};
  for (long long p = (long long)blockIdx.x * RED_T + threadIdx.x; p < n;
       p += (long long)gridDim.x * RED_T) {
    DF sr{0.f, 0.f}, si{0.f, 0.f};
    // h v = (hx vx - hy vy) + i (hx vy + hy vx); four basis vectors loaded
    // before their arithmetic (same order of accumulation as one at a time)
    auto acc = [&](const float2 v, int i) {
      const DF hx = hs[2 * i], hy = hs[2 * i + 1];
      df_add(sr, df_mul(v.x, hx.hi, hx.lo));
      df_add(sr, df_mul(-v.y, hy.hi, hy.lo));
      df_add(si, df_mul(v.y, hx.hi, hx.lo));
      df_add(si, df_mul(v.x, hy.hi, hy.lo));
    };
    int i = 0;
    for (; i + 4 <= k; i += 4) {
      float2 v4[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v4[q] = V[(long long)(i + q) * ldv + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc(v4[q], i + q);
    }
    for (; i < k; ++i) acc(V[(long long)i * ldv + p], i);
    if constexpr (std::is_same<WT, float4>::value) {
      // double-float w: the difference and the norm without FP64
      const float4 wv = w[p];
      DF wr{wv.x, wv.y}, wi{wv.z, wv.w};
      df_add(wr, DF{-sr.hi, -sr.lo});
      df_add(wi, DF{-si.hi, -si.lo});
      w[p] = make_float4(wr.hi, wr.lo, wi.hi, wi.lo);
      df_add(nn, df_sq(wr));
      df_add(nn, df_sq(wi));
    } else {
      const double2 wd = to_d2(w[p]);
      store_w(w + p, wd.x - df_to(sr), wd.y - df_to(si));
      const double2 o = to_d2(w[p]);
      df_add(nn, df_sq(df_from(o.x)));
      df_add(nn, df_sq(df_from(o.y)));
    }
  }
  __shared__ DF sh[RED_T / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) df_add(nn, df_shfl_xor(nn, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    DF a = sh[0];
    for (int q = 1; q < RED_T / 32; ++q) df_add(a, sh[q]);
    part[blockIdx.x] = df_to(a);
  }
}

// Launch of k_update with its shared memory for k coefficients.
template <typename WT>
static mcmg_status launch_update(const float2* V, long long ldv, int k, const double2* hc, WT* w,
                                 long long n, double* part, int nblk, cudaStream_t st) {
  const size_t smem = (size_t)k * 2 * sizeof(DF);
  if (smem > 227 * 1024) {
    set_error("Gram-Schmidt against %d vectors exceeds shared memory", k);
    return MCMG_ERR_SHAPE;
  }
  if (smem > 48 * 1024)
    MCMG_CUDA(cudaFuncSetAttribute(k_update<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  k_update<WT><<<nblk, RED_T, smem, st>>>(V, ldv, k, hc, w, n, part);
  MCMG_CHECK_LAUNCH("update");
  return MCMG_OK;
}

__global__ void __launch_bounds__(RED_T) k_reduce_scalar(const double* __restrict__ part, int nblk,
                                                         double* out, double* out_host) {
  double a = 0.0;
  for (int q = threadIdx.x; q < nblk; q += RED_T) a += part[q];
  const double2 r = block_sum2(a, 0.0);
  if (threadIdx.x == 0) {
    *out = r.x;
    if (out_host) *out_host = r.x;
  }
}

// Residual partials [nblk][2] -> rr, ff
__global__ void __launch_bounds__(RED_T) k_reduce_res(const double* __restrict__ part, int nblk,
                                                      double* __restrict__ dsc,
                                                      double* __restrict__ stat_rr) {
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += RED_T) { a += part[2 * q]; b += part[2 * q + 1]; }
  const double2 r = block_sum2(a, b);
  if (threadIdx.x == 0) {
    dsc[0] = r.x;
    dsc[1] = r.y;
    stat_rr[0] = r.x;
    stat_rr[1] = r.y;
  }
}

// v0 = r / beta (to complex64)
// The scalar of a scaling kernel, computed once per block (FP64 square roots
// and divisions run at a small fraction of the FP32 rate on this part).
__device__ __forceinline__ double block_inv_sqrt(const double* v) {
  __shared__ double inv;
  if (threadIdx.x == 0) {
    const double b = sqrt(*v);
    inv = b > 0.0 ? 1.0 / b : 0.0;
  }
  __syncthreads();
  return inv;
}

__device__ __forceinline__ double block_sqrt(const double* v) {
  __shared__ double root;
  if (threadIdx.x == 0) root = sqrt(*v);
  __syncthreads();
  return root;
}

__global__ void k_start_cycle(const double2* __restrict__ r, const double* __restrict__ dsc,
                              float2* __restrict__ v0, long long n) {
  const double inv = block_inv_sqrt(dsc);
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) {
    const double2 v = r[p];
    v0[p] = make_float2((float)(v.x * inv), (float)(v.y * inv));
  }
}

struct Stat {
  double rr, ff;  // |f - A u|^2, |f|^2 at the last restart
};

// v_{j+1} = w / sqrt(nrm2), rounded to complex64 (FP32 arithmetic on the
// double-float parts: the result is FP32 anyway)
__global__ void k_scale(const float4* __restrict__ w, const double* __restrict__ dsc,
                        float2* __restrict__ v, long long n) {
  const float inv = (float)block_inv_sqrt(dsc + 3);
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float4 x = w[p];
  v[p] = make_float2(__fmaf_rn(x.x, inv, x.y * inv), __fmaf_rn(x.z, inv, x.w * inv));
}

// Stationary step: u += beta * z, beta = ||r|| (the V-cycle ran on r / beta).
__global__ void k_stationary_update(const float2* __restrict__ z, const double* __restrict__ dsc,
                                    double2* __restrict__ u, long long n) {
  const double beta = block_sqrt(dsc);
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float2 zz = z[p];
  const double2 o = u[p];
  u[p] = make_double2(o.x + beta * zz.x, o.y + beta * zz.y);
}

// u += sum_{i<k} y_i Z_i (complex128 accumulate)
// (double-float accumulation: y is split once per block into shared memory,
// the products with the FP32 z are exact up to lo * lo, and only the final
// sum is added to u in FP64)
__global__ void k_update_x(const float2* __restrict__ Z, long long ldz, int k,
                           const double2* __restrict__ y, double2* __restrict__ u, long long n) {
  constexpr int CH = 64;                 // coefficients staged per chunk
  __shared__ DF ys[2 * CH];
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < n;
  DF sr{0.f, 0.f}, si{0.f, 0.f};
  for (int base = 0; base < k; base += CH) {
    const int cnt = k - base < CH ? k - base : CH;
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const double2 yy = y[base + i];
      ys[2 * i] = df_from(yy.x);
      ys[2 * i + 1] = df_from(yy.y);
    }
    __syncthreads();
    if (!live) continue;
    for (int i = 0; i < cnt; ++i) {
      const float2 z = Z[(long long)(base + i) * ldz + p];
      const DF yx = ys[2 * i], yy = ys[2 * i + 1];
      // y z = (yx zx - yy zy) + i (yx zy + yy zx)
      df_add(sr, df_mul(z.x, yx.hi, yx.lo));
      df_add(sr, df_mul(-z.y, yy.hi, yy.lo));
      df_add(si, df_mul(z.y, yx.hi, yx.lo));
      df_add(si, df_mul(z.x, yy.hi, yy.lo));
    }
  }
  if (!live) return;
  const double2 o = u[p];
  u[p] = make_double2(o.x + df_to(sr), o.y + df_to(si));
}

// ---------------------------------------------------------------------------
struct Krylov {
  mcmg_handle_s* h = nullptr;
  int m = 0;
  long long n = 0;
  int nblk = 0;
  VWork* vw = nullptr;
  float2* V = nullptr;
  float2* Z = nullptr;
  float4* w = nullptr;      // Arnoldi work vector, complex double-float
  double2* r64 = nullptr;
  double* part = nullptr;
  double2* d1 = nullptr;
  double2* d2 = nullptr;
  double2* dsum = nullptr;          // h1 + h2, the update's coefficients
  double2* red = nullptr;           // reduced one-pass dots: 2m + 3 values
  double2* Gd = nullptr;            // rows of the Gram matrix V^H V, (m+1) x (m+1)
  double2* y = nullptr;             // device copy of the least-squares solution
  // Host side of the Arnoldi process (FP64): Hessenberg columns, Givens
  // rotations, rotated right-hand side, and the least-squares solution.
  std::vector<std::complex<double>> Hh, sn, g;
  std::vector<double> cs;
  double2* y_h = nullptr;           // pinned staging of y
  // per Arnoldi step j, mapped: [0, m+2) first-pass dots (with |w|^2 last),
  // [m+2, 2m+4) second-pass dots, [2m+4].x = ||w||^2 after Gram-Schmidt
  double2* mir_h = nullptr;
  double2* mir_d = nullptr;
  int mir_stride = 0;
  double* dsc = nullptr;
  Stat* stat_h = nullptr;   // mapped pinned: the restart residual
  Stat* stat_d = nullptr;
  cudaEvent_t ev = nullptr;         // restart residual ready
  cudaEvent_t evs[2] = {};          // Arnoldi step j ready: evs[j & 1]
  cudaStream_t st = nullptr;        // stream of the current solve
  cudaStream_t own = nullptr;       // the solve's private stream (server use)
  DevArena arena;
  // solve state
  const double2* f = nullptr;
  double2* u = nullptr;
  mcmg_solve_opts o{};
  enum Phase { IDLE, WAIT_RES, WAIT_STEP, NEED_STEP, DONE } phase = IDLE;
  int j = 0, iters = 0, restarts = 0, max_iters = 0;
  int enq = 0;                      // Arnoldi steps enqueued in this cycle (j <= enq - 1 <= j + 1)
  double fnorm = 0.0, rel = 0.0;
  bool converged = false;
  mcmg_status final = MCMG_OK;
  std::chrono::steady_clock::time_point t0;
  double t_solve = 0.0;
};

// Blocks of the grid-stride reductions: about one element per thread, at
// most eight blocks per SM (the update and multi-dot loops over the basis are
// serial per element, so parallelism over elements hides their latency).
constexpr int RED_MAX_BLK = 148 * 8;

static int red_blocks(long long n) {
  long long b = (n + RED_T - 1) / RED_T;
  long long cap = RED_MAX_BLK;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

mcmg_status krylov_create(mcmg_handle_s* h, int m, Krylov** out, bool own_vcycle_work) {
  Krylov* k = new Krylov();
  k->h = h;
  k->m = m;
  k->n = h->g0.nodes();
  k->nblk = red_blocks(k->n);
  const long long n = k->n;
  auto A = [&](void** p, size_t b) { return dev_alloc(h, k->arena, p, b); };
  mcmg_status s = MCMG_OK;
  if ((s = A((void**)&k->V, sizeof(float2) * (size_t)(m + 1) * n)) ||
      (s = A((void**)&k->Z, sizeof(float2) * (size_t)m * n)) ||
      (s = A((void**)&k->w, sizeof(float4) * (size_t)n)) ||
      (s = A((void**)&k->r64, sizeof(double2) * (size_t)n)) ||
      (s = A((void**)&k->part, sizeof(double) * 2 * (size_t)k->nblk * (2 * m + 3))) ||
      (s = A((void**)&k->d1, sizeof(double2) * (m + 2))) ||
      (s = A((void**)&k->d2, sizeof(double2) * (m + 2))) ||
      (s = A((void**)&k->dsum, sizeof(double2) * (m + 2))) ||
      (s = A((void**)&k->red, sizeof(double2) * (2 * m + 3))) ||
      (s = A((void**)&k->Gd, sizeof(double2) * (size_t)(m + 1) * (m + 1))) ||
      (s = A((void**)&k->y, sizeof(double2) * (m + 1))) ||
      (s = A((void**)&k->dsc, sizeof(double) * 8))) {
    krylov_destroy(h, k);
    return s;
  }
  if (own_vcycle_work && (s = vwork_create(h, 1, &k->vw)) != MCMG_OK) {
    krylov_destroy(h, k);
    return s;
  }
  k->Hh.assign((size_t)m * (m + 1), 0.0);
  k->sn.assign(m + 1, 0.0);
  k->g.assign(m + 2, 0.0);
  k->cs.assign(m + 1, 0.0);
  k->mir_stride = 2 * m + 5;
  cudaError_t e = cudaHostAlloc((void**)&k->stat_h, sizeof(Stat), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&k->stat_d, k->stat_h, 0);
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&k->mir_h, sizeof(double2) * (size_t)m * k->mir_stride,
                      cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&k->mir_d, k->mir_h, 0);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&k->y_h, sizeof(double2) * (m + 1), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&k->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&k->evs[0], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&k->evs[1], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&k->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    krylov_destroy(h, k);
    return cuda_fail(e, "krylov_create");
  }
  *out = k;
  return MCMG_OK;
}

void krylov_destroy(mcmg_handle_s* h, Krylov* k) {
  if (!k) return;
  if (k->vw) vwork_destroy(h, k->vw);
  arena_free(h, k->arena);
  if (k->stat_h) cudaFreeHost(k->stat_h);
  if (k->mir_h) cudaFreeHost(k->mir_h);
  if (k->y_h) cudaFreeHost(k->y_h);
  if (k->ev) cudaEventDestroy(k->ev);
  for (cudaEvent_t e : k->evs)
    if (e) cudaEventDestroy(e);
  if (k->own) cudaStreamDestroy(k->own);
  delete k;
}

// Enqueue r = f - A u and its norms; the host reads them at WAIT_RES.
static mcmg_status enqueue_restart(Krylov* k) {
  mcmg_handle_s* h = k->h;
  MCMG_TRY(launch_residual64(h->q64, k->f, k->u, k->r64, k->part, k->nblk, h->g0, 1, k->st));
  k_reduce_res<<<1, RED_T, 0, k->st>>>(k->part, k->nblk, k->dsc, &k->stat_d->rr);
  MCMG_CHECK_LAUNCH("reduce_res");
  MCMG_CUDA(cudaEventRecord(k->ev, k->st));
  k->phase = Krylov::WAIT_RES;
  return MCMG_OK;
}

// The Arnoldi part of step j once z_j = MG(v_j) is in Z: w = A z_j, CGS2,
// Givens, v_{j+1}.  No event.
static mcmg_status enqueue_arnoldi(Krylov* k, int j) {
  mcmg_handle_s* h = k->h;
  const long long n = k->n;
  float2* zj = k->Z + (size_t)j * n;
  MCMG_TRY(launch_apply_A_arnoldi(h->qdf, zj, k->w, h->g0, k->st));
  double2* mir = k->mir_d + (size_t)j * k->mir_stride;
  // one sweep over the basis: h1 = V^H w, |w|^2 and the Gram row V^H v_j;
  // the second pass's coefficients from the Gram matrix; one update
  const int width = 2 * j + 3;
  dim3 grid((unsigned)k->nblk, (unsigned)((j + 2 + KV - 1) / KV));
  k_multidot_gram<<<grid, RED_T, 0, k->st>>>(k->V, n, j, k->w, n, k->part);
  MCMG_CHECK_LAUNCH("multidot_gram");
  k_reduce_parts<<<width, RED_T, 0, k->st>>>(k->part, k->nblk, width, k->red, nullptr);
  MCMG_CHECK_LAUNCH("reduce_parts");
  k_gram_correct<<<1, 64, 0, k->st>>>(k->red, j, k->m + 1, k->Gd, k->d1, k->d2, k->dsum, mir,
                                      k->m);
  MCMG_CHECK_LAUNCH("gram_correct");
  MCMG_TRY(launch_update(k->V, n, j + 1, k->dsum, k->w, n, k->part, k->nblk, k->st));
  k_reduce_scalar<<<1, RED_T, 0, k->st>>>(k->part, k->nblk, k->dsc + 3,
                                          &mir[2 * k->m + 4].x);
  MCMG_CHECK_LAUNCH("reduce_scalar");
  if (j + 1 <= k->m) {
    k_scale<<<(unsigned)((n + 255) / 256), 256, 0, k->st>>>(k->w, k->dsc, k->V + (size_t)(j + 1) * n, n);
    MCMG_CHECK_LAUNCH("scale");
  }
  k->phase = Krylov::WAIT_STEP;
  return MCMG_OK;
}

// One Arnoldi step j: z_j = MG(v_j), then the Arnoldi part; event evs[j & 1].
static mcmg_status enqueue_step(Krylov* k, int j) {
  const long long n = k->n;
  MCMG_TRY(vcycle_run(k->h, k->vw, k->V + (size_t)j * n, k->Z + (size_t)j * n, 1, k->st));
  MCMG_TRY(enqueue_arnoldi(k, j));
  MCMG_CUDA(cudaEventRecord(k->evs[j & 1], k->st));
  k->enq = j + 1;
  return MCMG_OK;
}

// Step j + 1 may be enqueued before the host has read step j's results: it
// needs only v_{j+1}, produced on the device in stream order, and its own
// outputs (z_{j+1}, v_{j+2}, its mirrored inner products) are read only if
// the cycle continues past step j.  So the device never waits for the host
// between steps; a cycle that stops early wastes one step.
static bool may_run_ahead(const Krylov* k, int step) {
  return step < k->m && k->iters + (step - k->j) + 1 <= k->max_iters;
}

// Host side of Arnoldi step j (after its event): Hessenberg column j from the
// step's mirrored inner products, the previous Givens rotations applied to
// it, the new rotation, and the rotated right-hand side g.  Returns
// |g_{j+1}| (the least-squares residual norm), h_{j+1,j} and ||A z_j||.
static void host_givens(Krylov* k, int j, double* res, double* hn, double* w0) {
  using cd = std::complex<double>;
  const int m = k->m;
  std::vector<double2> buf(k->mir_stride);
  std::memcpy(buf.data(), (const void*)(k->mir_h + (size_t)j * k->mir_stride),
              sizeof(double2) * k->mir_stride);
  const double2* d1 = buf.data();
  const double2* d2 = buf.data() + (m + 2);
  const double hnv = std::sqrt(std::max(buf[2 * m + 4].x, 0.0));
  cd* col = k->Hh.data() + (size_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = cd(d1[i].x + d2[i].x, d1[i].y + d2[i].y);
  col[j + 1] = cd(hnv, 0.0);
  for (int i = 0; i < j; ++i) {   // [c, s; -conj(s), c] applied to (h_i, h_{i+1})
    const cd h0 = col[i], h1 = col[i + 1];
    col[i] = k->cs[i] * h0 + k->sn[i] * h1;
    col[i + 1] = -std::conj(k->sn[i]) * h0 + k->cs[i] * h1;
  }
  const cd a = col[j], b = col[j + 1];
  const double aa = std::abs(a), bb = std::abs(b), rho = std::hypot(aa, bb);
  double c;
  cd sv;
  if (aa == 0.0) {
    c = 0.0;
    sv = 1.0;
  } else {
    c = aa / rho;
    sv = (a / aa) * std::conj(b) / rho;
  }
  k->cs[j] = c;
  k->sn[j] = sv;
  col[j] = c * a + sv * b;
  col[j + 1] = 0.0;
  const cd gj = k->g[j];
  k->g[j + 1] = -std::conj(sv) * gj;
  k->g[j] = c * gj;
  *res = std::abs(k->g[j + 1]);
  *hn = hnv;
  *w0 = std::sqrt(std::max(d1[j + 1].x, 0.0));
}

// y = R^{-1} g for the kk x kk upper triangle of the rotated Hessenberg
// matrix (host, FP64), staged in pinned memory.
static void host_backsolve(Krylov* k, int kk) {
  using cd = std::complex<double>;
  const int m = k->m;
  std::vector<cd> gw(k->g.begin(), k->g.begin() + kk), y(kk);
  for (int i = kk - 1; i >= 0; --i) {
    y[i] = gw[i] / k->Hh[(size_t)i * (m + 1) + i];
    for (int l = 0; l < i; ++l) gw[l] -= k->Hh[(size_t)i * (m + 1) + l] * y[i];
  }
  for (int i = 0; i < kk; ++i) k->y_h[i] = make_double2(y[i].real(), y[i].imag());
}

static mcmg_status enqueue_finish_cycle(Krylov* k, int kk) {
  host_backsolve(k, kk);
  MCMG_CUDA(cudaMemcpyAsync(k->y, k->y_h, sizeof(double2) * kk, cudaMemcpyHostToDevice, k->st));
  k_update_x<<<(unsigned)((k->n + 255) / 256), 256, 0, k->st>>>(k->Z, k->n, kk, k->y, k->u, k->n);
  MCMG_CHECK_LAUNCH("update_x");
  k->restarts += 1;
  return enqueue_restart(k);
}

mcmg_status krylov_begin(Krylov* k, const double2* f, double2* u, const mcmg_solve_opts& o,
                         cudaStream_t st) {
  k->f = f;
  k->u = u;
  k->o = o;
  k->st = st;
  k->iters = 0;
  k->restarts = 0;
  k->j = 0;
  k->converged = false;
  k->final = MCMG_OK;
  k->fnorm = -1.0;
  k->max_iters = o.max_iters > 0 ? o.max_iters : 20 * (k->h->g0.d == 3 ? k->h->g0.nz : k->h->g0.ny);
  k->t0 = std::chrono::steady_clock::now();
  return enqueue_restart(k);
}

static void finish(Krylov* k, bool conv, mcmg_status s) {
  k->converged = conv;
  k->final = s;
  k->phase = Krylov::DONE;
  k->t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - k->t0).count();
}

mcmg_status krylov_advance(Krylov* k, bool blocking, int* done) {
  *done = 0;
  if (k->phase == Krylov::DONE) {
    *done = 1;
    return MCMG_OK;
  }
  cudaEvent_t ev = k->phase == Krylov::WAIT_RES ? k->ev : k->evs[k->j & 1];
  if (blocking) {
    MCMG_CUDA(cudaEventSynchronize(ev));
  } else {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaErrorNotReady) return MCMG_OK;
    if (e != cudaSuccess) return cuda_fail(e, "krylov event");
  }
  if (k->h->err_host && *(volatile int*)k->h->err_host) {
    set_error("a bounded wait in a device kernel ran out (code %d)", *k->h->err_host);
    finish(k, false, MCMG_ERR_TIMEOUT);
    *done = 1;
    return MCMG_OK;
  }
  if (k->phase == Krylov::WAIT_RES) {
    Stat st;
    std::memcpy(&st, (const void*)k->stat_h, sizeof(Stat));
    if (k->fnorm < 0.0) k->fnorm = std::sqrt(st.ff);
    const double beta = std::sqrt(st.rr);
    if (!std::isfinite(beta)) {
      k->rel = beta;
      finish(k, false, MCMG_ERR_NUMERIC);
      *done = 1;
      return MCMG_OK;
    }
    k->rel = k->fnorm > 0.0 ? beta / k->fnorm : 0.0;
    if (k->fnorm == 0.0 || k->rel <= k->o.tol) {
      finish(k, true, MCMG_OK);
      *done = 1;
      return MCMG_OK;
    }
    if (k->iters >= k->max_iters) {
      finish(k, false, MCMG_ERR_NOT_CONVERGED);
      *done = 1;
      return MCMG_OK;
    }
    k_start_cycle<<<(unsigned)((k->n + 255) / 256), 256, 0, k->st>>>(k->r64, k->dsc, k->V, k->n);
    MCMG_CHECK_LAUNCH("start_cycle");
    std::fill(k->g.begin(), k->g.end(), 0.0);
    k->g[0] = beta;
    k->j = 0;
    k->phase = Krylov::WAIT_STEP;
    MCMG_TRY(enqueue_step(k, 0));
    if (may_run_ahead(k, 1)) MCMG_TRY(enqueue_step(k, 1));
    return MCMG_OK;
  }
  // WAIT_STEP: step j has finished (step j + 1 may be queued behind it)
  double res, hn, w0;
  host_givens(k, k->j, &res, &hn, &w0);
  k->iters += 1;
  const double est = res / k->fnorm;
  if (!std::isfinite(est)) {
    finish(k, false, MCMG_ERR_NUMERIC);
    *done = 1;
    return MCMG_OK;
  }
  const bool stop = est <= k->o.tol || hn <= 1e-14 * w0 || k->j + 1 >= k->m ||
                    k->iters >= k->max_iters;
  if (stop) return enqueue_finish_cycle(k, k->j + 1);
  k->j += 1;
  if (k->enq <= k->j) MCMG_TRY(enqueue_step(k, k->j));
  if (k->enq == k->j + 1 && may_run_ahead(k, k->j + 1)) MCMG_TRY(enqueue_step(k, k->j + 1));
  return MCMG_OK;
}

int krylov_m(const Krylov* k) { return k->m; }
cudaStream_t krylov_stream(const Krylov* k) { return k->own; }

void krylov_info(const Krylov* k, mcmg_solve_info* info, mcmg_status* final_status) {
  if (info) {
    info->iters = k->iters;
    info->restarts = k->restarts;
    info->rel_residual = k->rel;
    info->t_solve_s = k->t_solve;
    info->converged = k->converged ? 1 : 0;
  }
  if (final_status) *final_status = k->final;
}

// The stationary McMg iteration (Eq. mcmg_iteration): r = f - A u in FP64,
// u <- u + MG(r), until ||r|| / ||f|| <= tol or max_iters V-cycles.  The
// V-cycle runs on r / ||r|| (it is linear) so the complex64 input stays in
// range.  Synchronous.
mcmg_status stationary_run(Krylov* k, const double2* f, double2* u, const mcmg_solve_opts& o,
                           cudaStream_t st, mcmg_solve_info* info, mcmg_status* final_status) {
  mcmg_handle_s* h = k->h;
  const long long n = k->n;
  const int max_iters = o.max_iters > 0 ? o.max_iters : 20 * (h->g0.d == 3 ? h->g0.nz : h->g0.ny);
  const auto t0 = std::chrono::steady_clock::now();
  double fnorm = -1.0, rel = 0.0;
  int it = 0;
  mcmg_status fs = MCMG_OK;
  bool conv = false;
  for (;; ++it) {
    MCMG_TRY(launch_residual64(h->q64, f, u, k->r64, k->part, k->nblk, h->g0, 1, st));
    k_reduce_res<<<1, RED_T, 0, st>>>(k->part, k->nblk, k->dsc, &k->stat_d->rr);
    MCMG_CHECK_LAUNCH("reduce_res");
    MCMG_CUDA(cudaStreamSynchronize(st));
    Stat sv;
    std::memcpy(&sv, (const void*)k->stat_h, sizeof(Stat));
    if (fnorm < 0.0) fnorm = std::sqrt(sv.ff);
    rel = fnorm > 0.0 ? std::sqrt(sv.rr) / fnorm : 0.0;
    if (!std::isfinite(rel)) { fs = MCMG_ERR_NUMERIC; break; }
    if (rel <= o.tol) { conv = true; break; }
    if (it >= max_iters) { fs = MCMG_ERR_NOT_CONVERGED; break; }
    if (h->err_host && *(volatile int*)h->err_host) { fs = MCMG_ERR_TIMEOUT; break; }
    k_start_cycle<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(k->r64, k->dsc, k->V, n);
    MCMG_CHECK_LAUNCH("start_cycle");
    MCMG_TRY(vcycle_run(h, k->vw, k->V, k->Z, 1, st));
    k_stationary_update<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(k->Z, k->dsc, u, n);
    MCMG_CHECK_LAUNCH("stationary_update");
  }
  if (info) {
    info->iters = it;
    info->restarts = 0;
    info->rel_residual = rel;
    info->converged = conv ? 1 : 0;
    info->t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  *final_status = fs;
  return MCMG_OK;
}


// part[bx] = sum |x|^2 over the block's elements (FP64)
__global__ void __launch_bounds__(RED_T) k_norm2_parts(const double2* __restrict__ x, long long n,
                                                       double* __restrict__ part) {
  double a = 0.0;
  for (long long p = (long long)blockIdx.x * RED_T + threadIdx.x; p < n;
       p += (long long)gridDim.x * RED_T) {
    const double2 v = x[p];
    a += v.x * v.x + v.y * v.y;
  }
  const double2 r = block_sum2(a, 0.0);
  if (threadIdx.x == 0) part[blockIdx.x] = r.x;
}

// Born+McMg (Appendix, Born-series variant): r = f - A u in FP64, the
// Born-series residual G r (FFT, born.cu), u <- u + MG(G r) with the V-cycle
// run on G r / ||G r|| (it is linear).  Stops on ||f - A u|| / ||f|| like
// the stationary iteration.  Synchronous.
mcmg_status born_run(Krylov* k, const double2* f, double2* u, const mcmg_solve_opts& o,
                     cudaStream_t st, mcmg_solve_info* info, mcmg_status* final_status) {
  mcmg_handle_s* h = k->h;
  const long long n = k->n;
  MCMG_TRY(born_prepare(h));
  const int max_iters = o.max_iters > 0 ? o.max_iters : 20 * (h->g0.d == 3 ? h->g0.nz : h->g0.ny);
  const auto t0 = std::chrono::steady_clock::now();
  double fnorm = -1.0, rel = 0.0;
  int it = 0;
  mcmg_status fs = MCMG_OK;
  bool conv = false;
  for (;; ++it) {
    MCMG_TRY(launch_residual64(h->q64, f, u, k->r64, k->part, k->nblk, h->g0, 1, st));
    k_reduce_res<<<1, RED_T, 0, st>>>(k->part, k->nblk, k->dsc, &k->stat_d->rr);
    MCMG_CHECK_LAUNCH("reduce_res");
    MCMG_CUDA(cudaStreamSynchronize(st));
    Stat sv;
    std::memcpy(&sv, (const void*)k->stat_h, sizeof(Stat));
    if (fnorm < 0.0) fnorm = std::sqrt(sv.ff);
    rel = fnorm > 0.0 ? std::sqrt(sv.rr) / fnorm : 0.0;
    if (!std::isfinite(rel)) { fs = MCMG_ERR_NUMERIC; break; }
    if (rel <= o.tol) { conv = true; break; }
    if (it >= max_iters) { fs = MCMG_ERR_NOT_CONVERGED; break; }
    if (h->err_host && *(volatile int*)h->err_host) { fs = MCMG_ERR_TIMEOUT; break; }
    MCMG_TRY(born_apply_G(h, k->r64, st));                       // G (f - A u)
    k_norm2_parts<<<k->nblk, RED_T, 0, st>>>(k->r64, n, k->part);
    MCMG_CHECK_LAUNCH("norm2_parts");
    k_reduce_scalar<<<1, RED_T, 0, st>>>(k->part, k->nblk, k->dsc, nullptr);   // dsc[0]
    MCMG_CHECK_LAUNCH("reduce_scalar");
    k_start_cycle<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(k->r64, k->dsc, k->V, n);
    MCMG_CHECK_LAUNCH("start_cycle");
    MCMG_TRY(vcycle_run(h, k->vw, k->V, k->Z, 1, st));
    k_stationary_update<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(k->Z, k->dsc, u, n);
    MCMG_CHECK_LAUNCH("stationary_update");
  }
  if (info) {
    info->iters = it;
    info->restarts = 0;
    info->rel_residual = rel;
    info->converged = conv ? 1 : 0;
    info->t_solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  *final_status = fs;
  return MCMG_OK;
}


// ---------------------------------------------------------------------------
// Block of right-hand sides of one medium.
// ---------------------------------------------------------------------------
struct KrylovBlock {
  mcmg_handle_s* h = nullptr;
  int nb = 0, m = 0;
  std::vector<Krylov*> ks;
  VWork* vw = nullptr;              // nb fields
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  float2** ptr_h = nullptr;          // pinned: [0, nb) sources, [nb, 2nb) destinations
  float2** ptr_d = nullptr;
  DevArena arena;
  std::chrono::steady_clock::time_point t0;
  double t_solve = 0.0;
};

cudaStream_t block_stream(const KrylovBlock* b) { return b->st; }

int block_size(const KrylovBlock* b) { return b->nb; }
int block_m(const KrylovBlock* b) { return b->m; }

mcmg_status block_create(mcmg_handle_s* h, int m, int nb, KrylovBlock** out) {
  KrylovBlock* b = new KrylovBlock();
  b->h = h;
  b->nb = nb;
  b->m = m;
  mcmg_status s = MCMG_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->ptr_h, sizeof(float2*) * 2 * nb, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    block_destroy(h, b);
    return cuda_fail(e, "block_create");
  }
  if ((s = dev_alloc(h, b->arena, (void**)&b->ptr_d, sizeof(float2*) * 2 * nb)) ||
      (s = vwork_create(h, nb, &b->vw))) {
    block_destroy(h, b);
    return s;
  }
  for (int k = 0; k < nb; ++k) {
    Krylov* kr = nullptr;
    if ((s = krylov_create(h, m, &kr, false)) != MCMG_OK) {
      block_destroy(h, b);
      return s;
    }
    b->ks.push_back(kr);
  }
  *out = b;
  return MCMG_OK;
}

void block_destroy(mcmg_handle_s* h, KrylovBlock* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  for (Krylov* k : b->ks) krylov_destroy(h, k);
  if (b->vw) vwork_destroy(h, b->vw);
  arena_free(h, b->arena);
  if (b->ptr_h) cudaFreeHost(b->ptr_h);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

mcmg_status block_begin(KrylovBlock* b, const double2* f, double2* u, const mcmg_solve_opts& o) {
  const size_t N = (size_t)b->h->g0.nodes();
  b->t0 = std::chrono::steady_clock::now();
  for (int k = 0; k < b->nb; ++k)
    MCMG_TRY(krylov_begin(b->ks[k], f + k * N, u + k * N, o, b->st));
  MCMG_CUDA(cudaEventRecord(b->ev, b->st));
  return MCMG_OK;
}

// Read one member's results of the last round and decide its next stage.
static mcmg_status member_process(Krylov* k) {
  Stat st;
  std::memcpy(&st, (const void*)k->stat_h, sizeof(Stat));
  if (k->h->err_host && *(volatile int*)k->h->err_host) {
    set_error("a bounded wait in a device kernel ran out (code %d)", *k->h->err_host);
    finish(k, false, MCMG_ERR_TIMEOUT);
    return MCMG_OK;
  }
  if (k->phase == Krylov::WAIT_RES) {
    if (k->fnorm < 0.0) k->fnorm = std::sqrt(st.ff);
    const double beta = std::sqrt(st.rr);
    if (!std::isfinite(beta)) {
      k->rel = beta;
      finish(k, false, MCMG_ERR_NUMERIC);
      return MCMG_OK;
    }
    k->rel = k->fnorm > 0.0 ? beta / k->fnorm : 0.0;
    if (k->fnorm == 0.0 || k->rel <= k->o.tol) {
      finish(k, true, MCMG_OK);
      return MCMG_OK;
    }
    if (k->iters >= k->max_iters) {
      finish(k, false, MCMG_ERR_NOT_CONVERGED);
      return MCMG_OK;
    }
    k_start_cycle<<<(unsigned)((k->n + 255) / 256), 256, 0, k->st>>>(k->r64, k->dsc, k->V, k->n);
    MCMG_CHECK_LAUNCH("start_cycle");
    std::fill(k->g.begin(), k->g.end(), 0.0);
    k->g[0] = beta;
    k->j = 0;
    k->phase = Krylov::NEED_STEP;
    return MCMG_OK;
  }
  if (k->phase == Krylov::WAIT_STEP) {
    double res, hn, w0;
    host_givens(k, k->j, &res, &hn, &w0);
    k->iters += 1;
    const double est = res / k->fnorm;
    if (!std::isfinite(est)) {
      finish(k, false, MCMG_ERR_NUMERIC);
      return MCMG_OK;
    }
    const bool stop = est <= k->o.tol || hn <= 1e-14 * w0 || k->j + 1 >= k->m ||
                      k->iters >= k->max_iters;
    if (stop) return enqueue_finish_cycle(k, k->j + 1);   // -> WAIT_RES
    k->j += 1;
    k->phase = Krylov::NEED_STEP;
  }
  return MCMG_OK;
}

mcmg_status block_poll(KrylovBlock* b, bool blocking, int* done, int* count) {
  *done = 0;
  *count = -1;                         // -1: the last round is still running
  if (blocking) {
    MCMG_CUDA(cudaEventSynchronize(b->ev));
  } else {
    cudaError_t e = cudaEventQuery(b->ev);
    if (e == cudaErrorNotReady) return MCMG_OK;
    if (e != cudaSuccess) return cuda_fail(e, "block event");
  }
  for (Krylov* k : b->ks)
    if (k->phase == Krylov::WAIT_RES || k->phase == Krylov::WAIT_STEP) MCMG_TRY(member_process(k));
  // the members that need a V-cycle this round, in member order
  int n = 0;
  for (Krylov* k : b->ks)
    if (k->phase == Krylov::NEED_STEP) {
      b->ptr_h[n] = k->V + (size_t)k->j * k->n;
      b->ptr_h[b->nb + n] = k->Z + (size_t)k->j * k->n;
      ++n;
    }
  if (n > 0) {
    MCMG_CUDA(cudaMemcpyAsync(b->ptr_d, b->ptr_h, sizeof(float2*) * n, cudaMemcpyHostToDevice,
                              b->st));
    MCMG_CUDA(cudaMemcpyAsync(b->ptr_d + b->nb, b->ptr_h + b->nb, sizeof(float2*) * n,
                              cudaMemcpyHostToDevice, b->st));
  }
  *count = n;
  bool all = true;
  for (Krylov* k : b->ks) all = all && k->phase == Krylov::DONE;
  if (all) {
    MCMG_CUDA(cudaStreamSynchronize(b->st));
    b->t_solve = std::chrono::duration<double>(std::chrono::steady_clock::now() - b->t0).count();
    *done = 1;
  }
  return MCMG_OK;
}

mcmg_status block_after_vcycle(KrylovBlock* b) {
  for (Krylov* k : b->ks)
    if (k->phase == Krylov::NEED_STEP) MCMG_TRY(enqueue_arnoldi(k, k->j));
  MCMG_CUDA(cudaEventRecord(b->ev, b->st));
  return MCMG_OK;
}

void block_vcycle_io(KrylovBlock* b, VWork** w, const float2* const** srcs, float2* const** dsts) {
  *w = b->vw;
  *srcs = b->ptr_d;
  *dsts = b->ptr_d + b->nb;
}

mcmg_status block_advance(KrylovBlock* b, bool blocking, int* done) {
  int count = 0;
  MCMG_TRY(block_poll(b, blocking, done, &count));
  if (*done || count < 0) return MCMG_OK;
  if (count > 0) MCMG_TRY(vcycle_run_batch(b->h, b->vw, b->ptr_d, b->ptr_d + b->nb, count, b->st));
  return block_after_vcycle(b);
}

void block_info(const KrylovBlock* b, mcmg_solve_info* info, mcmg_status* final_status) {
  mcmg_solve_info agg{};
  agg.converged = 1;
  mcmg_status worst = MCMG_OK;
  for (const Krylov* k : b->ks) {
    agg.iters = std::max(agg.iters, k->iters);
    agg.restarts = std::max(agg.restarts, k->restarts);
    agg.rel_residual = std::max(agg.rel_residual, k->rel);
    agg.converged &= k->converged ? 1 : 0;
    if (k->final != MCMG_OK && worst == MCMG_OK) worst = k->final;
  }
  agg.t_solve_s = b->t_solve;
  if (info) *info = agg;
  if (final_status) *final_status = worst;
}

mcmg_status cgs2_once(mcmg_handle_s* h, const float2* V, int kv, long long n, float2* w,
                      double* h_host, double* norm_host, cudaStream_t st) {
  DevArena ar;
  int nblk = red_blocks(n);
  double* part = nullptr;
  double2 *d1 = nullptr, *d2 = nullptr;
  double* dsc = nullptr;
  mcmg_status s;
  if ((s = dev_alloc(h, ar, (void**)&part, sizeof(double) * 2 * (size_t)nblk * (kv + 1))) ||
      (s = dev_alloc(h, ar, (void**)&d1, sizeof(double2) * (kv + 1))) ||
      (s = dev_alloc(h, ar, (void**)&d2, sizeof(double2) * (kv + 1))) ||
      (s = dev_alloc(h, ar, (void**)&dsc, sizeof(double) * 2))) {
    arena_free(h, ar);
    return s;
  }
  auto run = [&]() -> mcmg_status {
    dim3 grid((unsigned)nblk, (unsigned)((kv + KV - 1) / KV));
    for (int pass = 0; pass < 2; ++pass) {
      double2* dd = pass == 0 ? d1 : d2;
      k_multidot<float2><<<grid, RED_T, 0, st>>>(V, n, kv, kv, w, n, part);
      MCMG_CHECK_LAUNCH("multidot");
      k_reduce_parts<<<kv, RED_T, 0, st>>>(part, nblk, kv, dd, nullptr);
      MCMG_CHECK_LAUNCH("reduce_parts");
      MCMG_TRY(launch_update(V, n, kv, dd, w, n, part, nblk, st));
    }
    k_reduce_scalar<<<1, RED_T, 0, st>>>(part, nblk, dsc, nullptr);
    MCMG_CHECK_LAUNCH("reduce_scalar");
    std::vector<double2> a(kv), b(kv);
    double nrm2 = 0.0;
    MCMG_CUDA(cudaMemcpyAsync(a.data(), d1, sizeof(double2) * kv, cudaMemcpyDeviceToHost, st));
    MCMG_CUDA(cudaMemcpyAsync(b.data(), d2, sizeof(double2) * kv, cudaMemcpyDeviceToHost, st));
    MCMG_CUDA(cudaMemcpyAsync(&nrm2, dsc, sizeof(double), cudaMemcpyDeviceToHost, st));
    MCMG_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < kv; ++i) {
      h_host[2 * i] = a[i].x + b[i].x;
      h_host[2 * i + 1] = a[i].y + b[i].y;
    }
    *norm_host = std::sqrt(nrm2);
    return MCMG_OK;
  };
  s = run();
  cudaStreamSynchronize(st);
  arena_free(h, ar);
  return s;
}

// ---------------------------------------------------------------------------
// CGS2 without any allocation, for callers that cannot allocate device memory.
//
// Its scratch (multi-dot partial sums, the two coefficient vectors, the norm)
// lives in the file-scope array below, which every GPU that loads this
// library holds until the process exits.  Host code must not pass the array's
// name to a kernel: on the host that name is only a stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (on the first
// call made with that device current) and cached.  All calls share the array:
// calls that overlap on the GPU race, and each call writes every scratch entry
// it reads before reading it, so nothing depends on an earlier call's contents.
// ---------------------------------------------------------------------------
constexpr int NOALLOC_MAX_K = 64;                       // basis vectors per call
constexpr int NOALLOC_MAX_BLK = RED_MAX_BLK;            // the red_blocks() cap
constexpr size_t NOALLOC_PART = 2ull * NOALLOC_MAX_BLK * NOALLOC_MAX_K;
constexpr size_t NOALLOC_DOUBLES = NOALLOC_PART + 4ull * NOALLOC_MAX_K + 8;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// h = d1 + d2 (k entries), written as (re, im) pairs into out.
__global__ void k_sum_coeffs(const double2* __restrict__ d1, const double2* __restrict__ d2, int k,
                             double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) {
    out[2 * i] = d1[i].x + d2[i].x;
    out[2 * i + 1] = d1[i].y + d2[i].y;
  }
}

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {};                 // per device ordinal

static mcmg_status noalloc_scratch(double** out) {
  int dev = 0;
  MCMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range", dev);
    return MCMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return MCMG_OK;
}

}  // namespace mcmg

mcmg_status mcmg_cgs2_noalloc(const void* V_dev, int k, size_t n, void* w_dev, double* h_host,
                              double* norm_host, void* stream) {
  using namespace mcmg;
  if (!V_dev || !w_dev || !h_host || !norm_host || n < 1) {
    set_error("NULL pointer or empty vector");
    return MCMG_ERR_ARG;
  }
  if (k < 1 || k > NOALLOC_MAX_K) {
    set_error("mcmg_cgs2_noalloc takes 1..%d basis vectors, got %d", NOALLOC_MAX_K, k);
    return MCMG_ERR_ARG;
  }
  int dev = 0;
  MCMG_CUDA(cudaGetDevice(&dev));
  for (const void* p : {V_dev, (const void*)w_dev}) {
    // both vectors must live on the current device: the scratch and the
    // kernels belong to it, and a peer pointer would be read across the link
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
      set_error("mcmg_cgs2_noalloc: V and w must be device memory of the current device %d", dev);
      return MCMG_ERR_ARG;
    }
  }
  double* base = nullptr;
  MCMG_TRY(noalloc_scratch(&base));
  cudaStream_t st = (cudaStream_t)stream;
  const long long nn = (long long)n;
  const int nblk = red_blocks(nn);
  if (nblk > NOALLOC_MAX_BLK) {     // the partial sums would not fit the scratch
    set_error("mcmg_cgs2_noalloc: %d reduction blocks exceed the scratch's %d", nblk,
              NOALLOC_MAX_BLK);
    return MCMG_ERR_ARG;
  }
  double* part = base;
  double2* d1 = (double2*)(base + NOALLOC_PART);
  double2* d2 = d1 + NOALLOC_MAX_K;
  double* dsc = base + NOALLOC_DOUBLES - 8;
  const float2* V = (const float2*)V_dev;
  float2* w = (float2*)w_dev;
  dim3 grid((unsigned)nblk, (unsigned)((k + KV - 1) / KV));
  for (int pass = 0; pass < 2; ++pass) {
    double2* dd = pass == 0 ? d1 : d2;
    k_multidot<float2><<<grid, RED_T, 0, st>>>(V, nn, k, k, w, nn, part);
    MCMG_CHECK_LAUNCH("multidot");
    k_reduce_parts<<<k, RED_T, 0, st>>>(part, nblk, k, dd, nullptr);
    MCMG_CHECK_LAUNCH("reduce_parts");
    MCMG_TRY(launch_update(V, nn, k, dd, w, nn, part, nblk, st));
  }
  k_reduce_scalar<<<1, RED_T, 0, st>>>(part, nblk, dsc, nullptr);
  MCMG_CHECK_LAUNCH("reduce_scalar");
  k_sum_coeffs<<<(k + 127) / 128, 128, 0, st>>>(d1, d2, k, part);   // part is free again
  MCMG_CHECK_LAUNCH("sum_coeffs");
  double nrm2 = 0.0;
  MCMG_CUDA(cudaMemcpyAsync(h_host, part, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, st));
  MCMG_CUDA(cudaMemcpyAsync(&nrm2, dsc, sizeof(double), cudaMemcpyDeviceToHost, st));
  MCMG_CUDA(cudaStreamSynchronize(st));
  *norm_host = std::sqrt(nrm2);
  return MCMG_OK;
}
