// Setup phase (Algorithm 1, Eq. phys_feature): the nonlinear setup networks
// that turn the medium into the cached per-level features a_l, s_l.  Run once
// per medium; not on the per-iteration path.
//
//   m      = ((kh)^2, (kh)^2 gamma)                 two real channels
//   a_1    = GELU(conv3(f_lift; m))                 2 C_1 real channels
//   s_l    = GELU(conv3(f_s^l; a_l))
//   a_{l+1}= GELU(conv3_stride2(f_a^l; a_l))
// Real channel pairs (2c, 2c+1) become complex channel c.  Channel 0 holds the
// classical shifted-Laplacian coefficient instead when feat_sl != 0:
//   a = -beta q_l,  s = 1 / (2 d 4^(-l) + a),  q_{l+1} = full weighting of q_l.
#include "mcmg_internal.cuh"

namespace mcmg {

__global__ void k_setup_input(const double2* __restrict__ q, float* __restrict__ m,
                              long long N) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double2 v = q[n];
  m[2 * n] = (float)v.x;        // (kh)^2
  m[2 * n + 1] = (float)(-v.y); // (kh)^2 gamma
}

mcmg_status launch_setup_input(const double2* q64, float* m, const Grid& g, cudaStream_t st) {
  long long N = g.nodes();
  k_setup_input<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(q64, m, N);
  MCMG_CHECK_LAUNCH("setup_input");
  return MCMG_OK;
}

__device__ __forceinline__ float gelu_exact(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

// out[J][co] = GELU(b[co] + sum_{o, ci} w[co][ci][o] in[stride * J + o][ci]),
// zero padding.  One thread per (output node, output channel).
__global__ void k_conv3_gelu(const float* __restrict__ in, int cin, float* __restrict__ out,
                             int cout, const float* __restrict__ w, const float* __restrict__ b,
                             Grid gi, Grid go, int stride) {
  long long N = go.nodes() * cout;
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= N) return;
  int co = (int)(id % cout);
  long long J = id / cout;
  int jx = (int)(J % go.nx);
  long long rest = J / go.nx;
  int jy = (int)(rest % go.ny);
  int jz = (int)(rest / go.ny);
  int T3 = gi.d == 3 ? 27 : 9;
  float acc = b[co];
  for (int o = 0; o < T3; ++o) {
    int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = gi.d == 3 ? o / 9 - 1 : 0;
    int fx = stride * jx + ox, fy = stride * jy + oy, fz = gi.d == 3 ? stride * jz + oz : 0;
    if (fx < 0 || fx >= gi.nx || fy < 0 || fy >= gi.ny || fz < 0 || fz >= gi.nz) continue;
    const float* src = in + (((long long)fz * gi.ny + fy) * gi.nx + fx) * cin;
    const float* wr = w + (long long)co * cin * T3 + o;
    for (int ci = 0; ci < cin; ++ci) acc = fmaf(wr[ci * T3], src[ci], acc);
  }
  out[id] = gelu_exact(acc);
}

mcmg_status launch_conv3_gelu(const float* in, int cin, float* out, int cout, const float* w,
                              const float* b, const Grid& gin, int stride, cudaStream_t st) {
  Grid go = stride == 2 ? gin.coarse() : gin;
  long long N = go.nodes() * cout;
  k_conv3_gelu<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(in, cin, out, cout, w, b, gin, go,
                                                             stride);
  MCMG_CHECK_LAUNCH("conv3_gelu");
  return MCMG_OK;
}

// qc[J] = sum_o fw(o) qf[2J + o], fw = (1,2,1)/4 per axis, zero outside.
__global__ void k_fw_restrict_q(const double2* __restrict__ qf, double2* __restrict__ qc, Grid gf,
                                Grid gc) {
  long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= gc.nodes()) return;
  int jx = (int)(J % gc.nx);
  long long rest = J / gc.nx;
  int jy = (int)(rest % gc.ny);
  int jz = (int)(rest / gc.ny);
  const double w1[3] = {0.25, 0.5, 0.25};
  double2 acc = make_double2(0.0, 0.0);
  int zlo = gf.d == 3 ? -1 : 0, zhi = gf.d == 3 ? 1 : 0;
  for (int oz = zlo; oz <= zhi; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        int fx = 2 * jx + ox, fy = 2 * jy + oy, fz = gf.d == 3 ? 2 * jz + oz : 0;
        if (fx < 0 || fx >= gf.nx || fy < 0 || fy >= gf.ny || fz < 0 || fz >= gf.nz) continue;
        double wt = w1[ox + 1] * w1[oy + 1] * (gf.d == 3 ? w1[oz + 1] : 1.0);
        double2 v = qf[((long long)fz * gf.ny + fy) * gf.nx + fx];
        acc.x += wt * v.x;
        acc.y += wt * v.y;
      }
  qc[J] = acc;
}

mcmg_status launch_fw_restrict_q(const double2* qf, double2* qc, const Grid& gf, cudaStream_t st) {
  Grid gc = gf.coarse();
  k_fw_restrict_q<<<(unsigned)((gc.nodes() + 255) / 256), 256, 0, st>>>(qf, qc, gf, gc);
  MCMG_CHECK_LAUNCH("fw_restrict_q");
  return MCMG_OK;
}

__global__ void k_assemble_features(const float* __restrict__ net_a, const float* __restrict__ net_s,
                                    const double2* __restrict__ ql, float2* __restrict__ a,
                                    float2* __restrict__ s, int C, long long N, double lap_diag,
                                    double feat_sl, double feat_eps, double br, double bi) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= N * C) return;
  int c = (int)(id % C);
  long long n = id / C;
  if (c == 0 && feat_sl != 0.0) {
    double2 q = ql[n];
    // a = -beta q
    double ar = -(br * q.x - bi * q.y), ai = -(br * q.y + bi * q.x);
    // s = 1 / (lap_diag + a)
    double dr = lap_diag + ar, di = ai;
    double den = dr * dr + di * di;
    double sr = dr / den, si = -di / den;
    a[id] = make_float2((float)(feat_sl * ar), (float)(feat_sl * ai));
    s[id] = make_float2((float)(feat_sl * sr), (float)(feat_sl * si));
  } else {
    const float* pa = net_a + n * 2 * C + 2 * c;
    const float* ps = net_s + n * 2 * C + 2 * c;
    a[id] = make_float2((float)(feat_eps * pa[0]), (float)(feat_eps * pa[1]));
    s[id] = make_float2((float)(feat_eps * ps[0]), (float)(feat_eps * ps[1]));
  }
}

mcmg_status launch_assemble_features(const float* net_a, const float* net_s, const double2* ql,
                                     float2* a, float2* s, int C, const Grid& g, int level,
                                     double feat_sl, double feat_eps, double beta_re,
                                     double beta_im, cudaStream_t st) {
  long long N = g.nodes();
  double lap_diag = 2.0 * g.d * ldexp(1.0, -2 * level);   // 2d * 4^(-l)
  k_assemble_features<<<(unsigned)((N * C + 255) / 256), 256, 0, st>>>(
      net_a, net_s, ql, a, s, C, N, lap_diag, feat_sl, feat_eps, beta_re, beta_im);
  MCMG_CHECK_LAUNCH("assemble_features");
  return MCMG_OK;
}

}  // namespace mcmg
