// The background Green operator of the Born-series variant (Appendix, Born
// series and the discrete Green operator): G = (-Delta_h - k0^2)^{-1} in the
// h^2-scaled system, applied by FFT with the symbol of the discrete
// five-/seven-point Laplacian (Eq. discrete_symbol at xi_a h = 2 pi m / N_a,
// periodic modes):  G x = IFFT( FFT(x) / (sum_a 4 sin^2(pi m_a / N_a) - q0) ).
// The transforms are cuFFT double-complex plans (a library FFT used as a
// diagonalisation); the symbol and the 1/N normalisation are one kernel.
// q0 = (k0 h)^2: Re q0 halfway between the extremes of Re q, Im q0 =
// -max |q - Re q0| (the convergent-Born-series choice with the sponge's
// damping sign), so the background symbol never vanishes.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mcmg_internal.cuh"

namespace mcmg {

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

static mcmg_status fft_fail(cufftResult r, const char* what) {
  set_error("%s failed (cuFFT status %d)", what, (int)r);
  return MCMG_ERR_CUDA;
}

mcmg_status born_prepare(mcmg_handle_s* h) {
  if (h->born_ready) return MCMG_OK;
  const Grid& g = h->g0;
  const long long n = g.nodes();
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
  // per-axis symbols 4 sin^2(pi m / N)
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < g.d; ++a) {
    std::vector<double> s(dims[a]);
    for (int m = 0; m < dims[a]; ++m) {
      const double t = std::sin(M_PI * m / dims[a]);
      s[m] = 4.0 * t * t;
    }
    MCMG_TRY(dev_alloc(h, h->arena, (void**)&h->born_sym[a], sizeof(double) * dims[a]));
    MCMG_CUDA(cudaMemcpy(h->born_sym[a], s.data(), sizeof(double) * dims[a], cudaMemcpyHostToDevice));
  }
  cufftHandle plan;
  cufftResult r = g.d == 3 ? cufftPlan3d(&plan, g.nz, g.ny, g.nx, CUFFT_Z2Z)
                           : cufftPlan2d(&plan, g.ny, g.nx, CUFFT_Z2Z);
  if (r != CUFFT_SUCCESS) return fft_fail(r, "cufftPlan");
  h->born_plan = (int)plan;
  h->born_ready = true;
  return MCMG_OK;
}

mcmg_status born_apply_G(mcmg_handle_s* h, double2* x, cudaStream_t st) {
  const Grid& g = h->g0;
  const long long n = g.nodes();
  cufftHandle plan = (cufftHandle)h->born_plan;
  cufftResult r = cufftSetStream(plan, st);
  if (r != CUFFT_SUCCESS) return fft_fail(r, "cufftSetStream");
  r = cufftExecZ2Z(plan, (cufftDoubleComplex*)x, (cufftDoubleComplex*)x, CUFFT_FORWARD);
  if (r != CUFFT_SUCCESS) return fft_fail(r, "cufftExecZ2Z forward");
  k_green_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      x, h->born_sym[0], h->born_sym[1], g.d == 3 ? h->born_sym[2] : nullptr, g.nx, g.ny, n,
      h->born_q0r, h->born_q0i, 1.0 / (double)n);
  MCMG_CHECK_LAUNCH("green_scale");
  r = cufftExecZ2Z(plan, (cufftDoubleComplex*)x, (cufftDoubleComplex*)x, CUFFT_INVERSE);
  if (r != CUFFT_SUCCESS) return fft_fail(r, "cufftExecZ2Z inverse");
  return MCMG_OK;
}

void born_release(mcmg_handle_s* h) {
  if (h->born_ready) cufftDestroy((cufftHandle)h->born_plan);
  h->born_ready = false;
}

}  // namespace mcmg
