// The background Green operator of the Born-series variant (Appendix, Born
// series and the discrete Green operator): G = (-Delta_h - k0^2)^{-1} in the
// h^2-scaled system, diagonalised by the discrete Fourier transform with the
// symbol of the discrete five-/seven-point Laplacian (Eq. discrete_symbol at
// xi_a h = 2 pi m / N_a, periodic modes):
//
//   G x = IDFT( DFT(x) / (sum_a 4 sin^2(pi m_a / N_a) - q0) ).
//
// The multi-dimensional DFT is separable: one batched one-dimensional
// transform per axis, written here as an in-place radix-2 decimation-in-time
// FFT in FP64 for power-of-two axis lengths.  A CTA loads W lines of one axis
// into shared memory at bit-reversed positions, runs the log2(N) butterfly
// stages there (twiddles exp(-+2 pi i k / N) tabulated on the host in double
// precision) and writes the lines back in natural order.  For the strided
// axes the W lines are consecutive along x, so every load and store of a
// line element is a coalesced run of W values.  The symbol and the 1/N
// normalisation are one kernel between the forward and the inverse pass.
// q0 = (k0 h)^2: Re q0 halfway between the extremes of Re q, Im q0 =
// -max |q - Re q0| (the convergent-Born-series choice with the sponge's
// damping sign), so the background symbol never vanishes.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mcmg_internal.cuh"

namespace mcmg {

namespace {

constexpr int FFT_THREADS = 256;
constexpr int FFT_MAX_N = 4096;          // longest axis (shared memory: N W 16 B <= 64 KB)

// lines per CTA for an axis of length n
int fft_lines(int n) { return std::max(1, std::min(16, 4096 / n)); }

// One batched radix-2 FFT pass over axis `axis` of the field x (in place).
// tw: n / 2 twiddles exp(-2 pi i k / n); inverse uses their conjugates.
// Lines of the axis are the points with that coordinate 0; CTA b takes the W
// lines that are consecutive along the fastest other axis.
__global__ void __launch_bounds__(FFT_THREADS) k_fft_axis(double2* __restrict__ x,
                                                         const double2* __restrict__ tw, int nx,
                                                         int ny, int nz, int axis, int logn, int W,
                                                         int inverse) {
  extern __shared__ double2 sbuf[];      // [n][W]
  const int n = 1 << logn;
  const long long nxy = (long long)nx * ny;
  // first line of this CTA and the strides
  long long base0, lstride, estride;     // line w at base0 + w lstride, element i at + i estride
  const int b = blockIdx.x;
  if (axis == 0) {                       // lines (y, z): W consecutive y
    const int per = ny / W;
    const int yb = (b % per) * W, z = b / per;
    base0 = ((long long)z * ny + yb) * nx;
    lstride = nx;
    estride = 1;
  } else if (axis == 1) {                // lines (x, z): W consecutive x
    const int per = nx / W;
    const int xb = (b % per) * W, z = b / per;
    base0 = (long long)z * nxy + xb;
    lstride = 1;
    estride = nx;
  } else {                               // lines (x, y): W consecutive x
    const int per = nx / W;
    const int xb = (b % per) * W, y = b / per;
    base0 = (long long)y * nx + xb;
    lstride = 1;
    estride = nxy;
  }
  const int total = n * W;
  // load: element i of line w -> sbuf[bitrev(i)][w]; for the strided axes
  // consecutive threads take consecutive w (a coalesced run along x)
  for (int t = threadIdx.x; t < total; t += FFT_THREADS) {
    int i, w;
    if (axis == 0) { w = t / n; i = t - w * n; }
    else { i = t / W; w = t - i * W; }
    const int j = (int)(__brev((unsigned)i) >> (32 - logn));
    sbuf[j * W + w] = x[base0 + w * lstride + i * estride];
  }
  __syncthreads();
  // butterfly stages: half-size m = 1, 2, 4, ..., n / 2
  for (int s = 0; s < logn; ++s) {
    const int m = 1 << s;
    for (int t = threadIdx.x; t < (n / 2) * W; t += FFT_THREADS) {
      const int w = t % W, bf = t / W;
      const int j = bf & (m - 1);
      const int i0 = ((bf >> s) << (s + 1)) + j, i1 = i0 + m;
      double2 c = tw[j << (logn - 1 - s)];  // exp(-2 pi i j / (2m))
      if (inverse) c.y = -c.y;
      const double2 u = sbuf[i0 * W + w], v = sbuf[i1 * W + w];
      const double2 vc = make_double2(v.x * c.x - v.y * c.y, v.x * c.y + v.y * c.x);
      sbuf[i0 * W + w] = make_double2(u.x + vc.x, u.y + vc.y);
      sbuf[i1 * W + w] = make_double2(u.x - vc.x, u.y - vc.y);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < total; t += FFT_THREADS) {
    int i, w;
    if (axis == 0) { w = t / n; i = t - w * n; }
    else { i = t / W; w = t - i * W; }
    x[base0 + w * lstride + i * estride] = sbuf[i * W + w];
  }
}

// x[p] *= inv_n / (sx[x] + sy[y] + sz[z] - q0)
__global__ void k_green_scale(double2* __restrict__ x, const double* __restrict__ sx,
                              const double* __restrict__ sy, const double* __restrict__ sz,
                              int nx, int ny, long long n, double q0r, double q0i, double inv_n) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const long long rest = p / nx;
  const int ix = (int)(p - rest * nx);
  const int iy = (int)(rest % ny);
  const int iz = (int)(rest / ny);
  const double mu = sx[ix] + sy[iy] + (sz ? sz[iz] : 0.0);
  const double dr = mu - q0r, di = -q0i;            // mu - q0
  const double s = inv_n / (dr * dr + di * di);      // inv_n / |mu - q0|^2
  const double2 v = x[p];
  // v * conj(mu - q0) * s
  x[p] = make_double2((v.x * dr + v.y * di) * s, (v.y * dr - v.x * di) * s);
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// every axis of the field once, forward or inverse
mcmg_status fft_all_axes(mcmg_handle_s* h, double2* x, bool inverse, cudaStream_t st) {
  const Grid& g = h->g0;
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < g.d; ++a) {
    const int n = dims[a];
    if (n == 1) continue;
    // W lines per CTA, consecutive along y for the x axis, along x otherwise
    const int other = a == 0 ? g.ny : g.nx;
    const int W = std::min(fft_lines(n), other);
    const long long lines = g.nodes() / n;
    const unsigned blocks = (unsigned)(lines / W);
    const size_t smem = sizeof(double2) * (size_t)n * W;
    k_fft_axis<<<blocks, FFT_THREADS, smem, st>>>(x, h->born_tw[a], g.nx, g.ny, g.nz, a,
                                                  ilog2(n), W, inverse ? 1 : 0);
    MCMG_CHECK_LAUNCH("fft_axis");
  }
  return MCMG_OK;
}

}  // namespace

mcmg_status born_prepare(mcmg_handle_s* h) {
  if (h->born_ready) return MCMG_OK;
  const Grid& g = h->g0;
  const long long n = g.nodes();
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < g.d; ++a)
    if (!pow2(dims[a]) || dims[a] > FFT_MAX_N) {
      set_error("the Born-series variant needs power-of-two axes of at most %d cells (axis %d "
                "has %d)", FFT_MAX_N, a, dims[a]);
      return MCMG_ERR_SHAPE;
    }
  // q0 from q (setup-time data, read back once)
  std::vector<double2> q((size_t)n);
  MCMG_CUDA(cudaMemcpy(q.data(), h->q64, sizeof(double2) * n, cudaMemcpyDeviceToHost));
  double lo = q[0].x, hi = q[0].x;
  for (const double2& v : q) { lo = std::min(lo, v.x); hi = std::max(hi, v.x); }
  const double mid = 0.5 * (lo + hi);
  double eps = 0.0;
  for (const double2& v : q) eps = std::max(eps, std::hypot(v.x - mid, v.y));
  h->born_q0r = mid;
  h->born_q0i = -eps;
  // per-axis symbols 4 sin^2(pi m / N) and twiddles exp(-2 pi i k / N)
  for (int a = 0; a < g.d; ++a) {
    const int N = dims[a];
    std::vector<double> s(N);
    for (int m = 0; m < N; ++m) {
      const double t = std::sin(M_PI * m / N);
      s[m] = 4.0 * t * t;
    }
    std::vector<double2> tw(std::max(1, N / 2));
    for (int k = 0; k < N / 2; ++k)
      tw[k] = make_double2(std::cos(2.0 * M_PI * k / N), -std::sin(2.0 * M_PI * k / N));
    MCMG_TRY(dev_alloc(h, h->arena, (void**)&h->born_sym[a], sizeof(double) * N));
    MCMG_TRY(dev_alloc(h, h->arena, (void**)&h->born_tw[a], sizeof(double2) * tw.size()));
    // ordered on the handle's stream and waited below: a synchronous copy
    // from pageable memory may still be in flight when it returns
    MCMG_CUDA(cudaMemcpyAsync(h->born_sym[a], s.data(), sizeof(double) * N,
                              cudaMemcpyHostToDevice, h->stream));
    MCMG_CUDA(cudaMemcpyAsync(h->born_tw[a], tw.data(), sizeof(double2) * tw.size(),
                              cudaMemcpyHostToDevice, h->stream));
  }
  MCMG_CUDA(cudaStreamSynchronize(h->stream));
  // the largest pass asks for 64 KB of shared memory
  MCMG_CUDA(cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 64 * 1024));
  h->born_ready = true;
  return MCMG_OK;
}

mcmg_status born_apply_G(mcmg_handle_s* h, double2* x, cudaStream_t st) {
  const Grid& g = h->g0;
  const long long n = g.nodes();
  MCMG_TRY(fft_all_axes(h, x, false, st));
  k_green_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      x, h->born_sym[0], h->born_sym[1], g.d == 3 ? h->born_sym[2] : nullptr, g.nx, g.ny, n,
      h->born_q0r, h->born_q0i, 1.0 / (double)n);
  MCMG_CHECK_LAUNCH("green_scale");
  return fft_all_axes(h, x, true, st);
}

void born_release(mcmg_handle_s* h) { h->born_ready = false; }

}  // namespace mcmg

mcmg_status mcmg_apply_G(mcmg_handle h, void* x_dev, void* stream) {
  using namespace mcmg;
  if (!h || !x_dev) {
    set_error("NULL argument");
    return MCMG_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(h->mu);
  MCMG_CUDA(cudaSetDevice(h->device));
  MCMG_TRY(born_prepare(h));
  return born_apply_G(h, (double2*)x_dev, (cudaStream_t)stream);
}
