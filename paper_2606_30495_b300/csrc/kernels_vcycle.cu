// V-cycle kernels of Algorithm 2 (Section 3.2), FP32 channel mixing on the
// CUDA cores.  Fields are complex64, channels-last ([node][C]); mixing matrices
// are stored transposed (M^T[ci][co]) so a warp's output channels read
// consecutive weights.
//
// Fused smoothing step on level l (one launch per step):
//   t = r - A_l(e),   A_l(e) = W_l * e + a_l (.) (K_A e)     (stencil + K_A)
//   z = s_l (.) (K_S t)
//   e' = e + W^(i) z
// A block owns NB consecutive nodes and all C channels; thread (co, g) owns
// output channel co of TN nodes, so each weight load feeds TN complex FMAs.
// t and z go through shared memory because K_S and W^(i) mix all channels of
// a node.
#include "mcmg_internal.cuh"

namespace mcmg {

// Thread (co, g) of a 256-thread block owns output channel co of TN nodes;
// G = 256 / C node groups, NB = G * TN nodes per block.  TN is chosen per
// launch: large for big grids (weight reuse), small for coarse grids (enough
// blocks to cover the SMs).
template <int C, int TN_>
struct Tile {
  static constexpr int G = 256 / C;      // node groups
  static constexpr int TN = TN_;         // nodes per thread
  static constexpr int NB = G * TN;      // nodes per block
};

// Largest nodes-per-thread (of 8, 2, 1) that still gives at least two blocks
// per SM, so coarse levels are not left with a handful of blocks.
static int pick_tn(long long nodes, int C, int nrhs) {
  const long long want = 2 * 148;
  const int G = 256 / C;
  for (int tn : {8, 2}) {
    long long blocks = (nodes + (long long)G * tn - 1) / ((long long)G * tn) * nrhs;
    if (blocks >= want) return tn;
  }
  return 1;
}

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
};

__device__ __forceinline__ void node_xyz(long long n, int nx, int ny, int& x, int& y, int& z) {
  x = (int)(n % nx);
  long long rest = n / nx;
  y = (int)(rest % ny);
  z = (int)(rest / ny);
}

template <int C, int D, int MODE, int TN>
__global__ void __launch_bounds__(256) k_smooth(SmoothParams p) {
  using T = Tile<C, TN>;
  extern __shared__ float2 sm[];
  const int co = threadIdx.x % C;
  const int g = threadIdx.x / C;
  const long long N = p.nodes;
  const size_t off = (size_t)blockIdx.y * (size_t)N * C;
  const float2* __restrict__ r = p.r + off;
  const float2* __restrict__ ein = p.e_in ? p.e_in + off : nullptr;
  float2* __restrict__ eout = p.e_out + off;
  const long long n0 = (long long)blockIdx.x * T::NB;

  long long nn[T::TN];
  long long nc[T::TN];  // clamped (always a valid node)
#pragma unroll
  for (int k = 0; k < T::TN; ++k) {
    nn[k] = n0 + g + (long long)T::G * k;
    nc[k] = nn[k] < N ? nn[k] : N - 1;
  }

  float2 t[T::TN];
  if (ein) {
    float2 acc[T::TN], acca[T::TN];
    int cx[T::TN], cy[T::TN], cz[T::TN];
#pragma unroll
    for (int k = 0; k < T::TN; ++k) {
      node_xyz(nc[k], p.nx, p.ny, cx[k], cy[k], cz[k]);
      acc[k] = make_float2(0.f, 0.f);
      acca[k] = make_float2(0.f, 0.f);
    }
    // centre tap and K_A share the loads of e at the node itself
    for (int ci = 0; ci < C; ++ci) {
      const float2 w0 = __ldg(p.Wt + ci * C + co);
      const float2 wa = __ldg(p.KAt + ci * C + co);
#pragma unroll
      for (int k = 0; k < T::TN; ++k) {
        const float2 v = __ldg(ein + nc[k] * C + ci);
        cfma(acc[k], w0, v);
        cfma(acca[k], wa, v);
      }
    }
    const long long sxy = (long long)p.nx * p.ny;
#pragma unroll
    for (int tap = 1; tap <= 2 * D; ++tap) {
      const int axis = (tap - 1) >> 1;
      const int sgn = (tap & 1) ? -1 : 1;
      long long nb[T::TN];
      bool ok[T::TN];
#pragma unroll
      for (int k = 0; k < T::TN; ++k) {
        int c = axis == 0 ? cx[k] : (axis == 1 ? cy[k] : cz[k]);
        int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
        long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : sxy);
        ok[k] = (c + sgn >= 0) && (c + sgn < ext);
        nb[k] = ok[k] ? nc[k] + sgn * stride : nc[k];
      }
      const float2* wt = p.Wt + (size_t)tap * C * C;
      for (int ci = 0; ci < C; ++ci) {
        const float2 w = __ldg(wt + ci * C + co);
#pragma unroll
        for (int k = 0; k < T::TN; ++k) {
          const float2 v = __ldg(ein + nb[k] * C + ci);
          if (ok[k]) cfma(acc[k], w, v);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < T::TN; ++k) {
      const float2 rv = r[nc[k] * C + co];
      const float2 av = p.a[nc[k] * C + co];
      t[k] = csub(csub(rv, acc[k]), cmul(av, acca[k]));
    }
  } else {
#pragma unroll
    for (int k = 0; k < T::TN; ++k) t[k] = r[nc[k] * C + co];
  }

  if (MODE == 1) {  // residual only
#pragma unroll
    for (int k = 0; k < T::TN; ++k)
      if (nn[k] < N) eout[nn[k] * C + co] = t[k];
    return;
  }

  float2* sm_t = sm;
  float2* sm_z = sm + T::NB * C;
#pragma unroll
  for (int k = 0; k < T::TN; ++k) sm_t[(g + T::G * k) * C + co] = t[k];
  __syncthreads();

  // z = s (.) (K_S t)
  float2 z[T::TN];
#pragma unroll
  for (int k = 0; k < T::TN; ++k) z[k] = make_float2(0.f, 0.f);
  for (int ci = 0; ci < C; ++ci) {
    const float2 w = __ldg(p.KSt + ci * C + co);
#pragma unroll
    for (int k = 0; k < T::TN; ++k) cfma(z[k], w, sm_t[(g + T::G * k) * C + ci]);
  }
#pragma unroll
  for (int k = 0; k < T::TN; ++k) {
    z[k] = cmul(p.s[nc[k] * C + co], z[k]);
    sm_z[(g + T::G * k) * C + co] = z[k];
  }
  __syncthreads();

  // e' = e + W^(i) z
  float2 u[T::TN];
#pragma unroll
  for (int k = 0; k < T::TN; ++k) u[k] = make_float2(0.f, 0.f);
  for (int ci = 0; ci < C; ++ci) {
    const float2 w = __ldg(p.Wst + ci * C + co);
#pragma unroll
    for (int k = 0; k < T::TN; ++k) cfma(u[k], w, sm_z[(g + T::G * k) * C + ci]);
  }
#pragma unroll
  for (int k = 0; k < T::TN; ++k) {
    if (nn[k] < N) {
      float2 v = u[k];
      if (ein) v = cadd(v, ein[nn[k] * C + co]);
      eout[nn[k] * C + co] = v;
    }
  }
}

template <int C, int D, int TN>
static mcmg_status smooth_tn(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  using T = Tile<C, TN>;
  dim3 grid((unsigned)((p.nodes + T::NB - 1) / T::NB), (unsigned)nrhs);
  size_t smem = mode == 0 ? 2 * (size_t)T::NB * C * sizeof(float2) : 0;
  if (mode == 0)
    k_smooth<C, D, 0, TN><<<grid, 256, smem, st>>>(p);
  else
    k_smooth<C, D, 1, TN><<<grid, 256, smem, st>>>(p);
  MCMG_CHECK_LAUNCH("smooth");
  return MCMG_OK;
}

template <int C, int D>
static mcmg_status smooth_c(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  switch (pick_tn(p.nodes, C, nrhs)) {
    case 8: return smooth_tn<C, D, 8>(p, mode, nrhs, st);
    case 2: return smooth_tn<C, D, 2>(p, mode, nrhs, st);
    default: return smooth_tn<C, D, 1>(p, mode, nrhs, st);
  }
}

template <int D>
static mcmg_status smooth_d(const SmoothParams& p, int C, int mode, int nrhs, cudaStream_t st) {
  switch (C) {
    case 1: return smooth_c<1, D>(p, mode, nrhs, st);
    case 2: return smooth_c<2, D>(p, mode, nrhs, st);
    case 4: return smooth_c<4, D>(p, mode, nrhs, st);
    case 8: return smooth_c<8, D>(p, mode, nrhs, st);
    case 16: return smooth_c<16, D>(p, mode, nrhs, st);
    case 32: return smooth_c<32, D>(p, mode, nrhs, st);
    case 64: return smooth_c<64, D>(p, mode, nrhs, st);
  }
  set_error("unsupported channel count %d", C);
  return MCMG_ERR_SHAPE;
}

mcmg_status launch_smooth(const Level& L, int step, const float2* r, const float2* e_in,
                          float2* e_out, int mode, int nrhs, cudaStream_t st) {
  if (mode == 0 && L.use_tc)
    return launch_smooth_tc(L, L.tcw, step, r, e_in, e_out, nrhs, L.err, st);
  SmoothParams p;
  p.r = r;
  p.e_in = e_in;
  p.e_out = e_out;
  p.a = L.a;
  p.s = L.s;
  p.Wt = L.Wt;
  p.KAt = L.KAt;
  p.KSt = L.KSt;
  p.Wst = L.Wsmt + (size_t)(mode == 0 ? step : 0) * L.C * L.C;
  p.nx = L.g.nx;
  p.ny = L.g.ny;
  p.nz = L.g.nz;
  p.nodes = L.g.nodes();
  return L.g.d == 3 ? smooth_d<3>(p, L.C, mode, nrhs, st) : smooth_d<2>(p, L.C, mode, nrhs, st);
}

// ---------------------------------------------------------------------------
// Restriction: rc[J][co] = sum_{o in {-1,0,1}^d} sum_ci R[o][co][ci] t[2J+o][ci]
// (multi-channel strided convolution, stride 2, zero padding).  Thread (co, g)
// owns output channel co of TN coarse nodes.
// ---------------------------------------------------------------------------
struct TransferParams {
  const float2* src;
  float2* dst;
  const float2* Wt;    // [T3][cin][CO]
  int cin;
  int fx, fy, fz;      // fine grid
  int cx, cy, cz;      // coarse grid
  long long src_nodes, dst_nodes;
};

template <int CO, int D, int TN>
__global__ void __launch_bounds__(256) k_restrict(TransferParams p) {
  using T = Tile<CO, TN>;
  const int co = threadIdx.x % CO;
  const int g = threadIdx.x / CO;
  const long long NC = p.dst_nodes;
  const float2* __restrict__ t = p.src + (size_t)blockIdx.y * p.src_nodes * p.cin;
  float2* __restrict__ rc = p.dst + (size_t)blockIdx.y * NC * CO;
  const long long n0 = (long long)blockIdx.x * T::NB;
  long long nn[T::TN];
  int jx[T::TN], jy[T::TN], jz[T::TN];
  float2 acc[T::TN];
#pragma unroll
  for (int k = 0; k < T::TN; ++k) {
    nn[k] = n0 + g + (long long)T::G * k;
    long long c = nn[k] < NC ? nn[k] : NC - 1;
    node_xyz(c, p.cx, p.cy, jx[k], jy[k], jz[k]);
    acc[k] = make_float2(0.f, 0.f);
  }
  constexpr int T3 = D == 3 ? 27 : 9;
  for (int o = 0; o < T3; ++o) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = D == 3 ? o / 9 - 1 : 0;
    long long fi[T::TN];
    bool ok[T::TN];
#pragma unroll
    for (int k = 0; k < T::TN; ++k) {
      int x = 2 * jx[k] + ox, y = 2 * jy[k] + oy, z = D == 3 ? 2 * jz[k] + oz : 0;
      ok[k] = x >= 0 && x < p.fx && y >= 0 && y < p.fy && z >= 0 && z < p.fz;
      fi[k] = ok[k] ? ((long long)z * p.fy + y) * p.fx + x : 0;
    }
    const float2* w = p.Wt + (size_t)o * p.cin * CO;
    for (int ci = 0; ci < p.cin; ++ci) {
      const float2 wv = __ldg(w + ci * CO + co);
#pragma unroll
      for (int k = 0; k < T::TN; ++k) {
        const float2 v = __ldg(t + fi[k] * p.cin + ci);
        if (ok[k]) cfma(acc[k], wv, v);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < T::TN; ++k)
    if (nn[k] < NC) rc[nn[k] * CO + co] = acc[k];
}

// Prolongation-add: e[p][co] += sum over (J, o) with 2J + o = p of
// sum_ci P[o][co][ci] ec[J][ci]  (transposed strided convolution).  Per axis
// an even fine index has one source (J = p/2, o = 0) and an odd one two
// (J = (p-1)/2, o = +1 and J = (p+1)/2, o = -1), so each node visits the 2^d
// combinations of its candidates rather than all 3^d taps.
template <int CO, int D, int TN>
__global__ void __launch_bounds__(256) k_prolong_add(TransferParams p) {
  using T = Tile<CO, TN>;
  const int co = threadIdx.x % CO;
  const int g = threadIdx.x / CO;
  const long long NF = p.dst_nodes;
  const float2* __restrict__ ec = p.src + (size_t)blockIdx.y * p.src_nodes * p.cin;
  float2* __restrict__ e = p.dst + (size_t)blockIdx.y * NF * CO;
  const long long n0 = (long long)blockIdx.x * T::NB;
  long long nn[T::TN];
  int px[T::TN], py[T::TN], pz[T::TN];
  float2 acc[T::TN];
#pragma unroll
  for (int k = 0; k < T::TN; ++k) {
    nn[k] = n0 + g + (long long)T::G * k;
    long long c = nn[k] < NF ? nn[k] : NF - 1;
    node_xyz(c, p.fx, p.fy, px[k], py[k], pz[k]);
    acc[k] = make_float2(0.f, 0.f);
  }
  constexpr int NCOMB = D == 3 ? 8 : 4;
  for (int cb = 0; cb < NCOMB; ++cb) {
    const int bx = cb & 1, by = (cb >> 1) & 1, bz = (cb >> 2) & 1;
#pragma unroll
    for (int k = 0; k < T::TN; ++k) {
      // candidate along each axis: b = 0 -> o = 0 (even) or o = +1 (odd);
      // b = 1 -> o = -1 (odd only)
      int oxs = (px[k] & 1) ? (bx ? -1 : 1) : 0;
      int oys = (py[k] & 1) ? (by ? -1 : 1) : 0;
      int ozs = D == 3 ? ((pz[k] & 1) ? (bz ? -1 : 1) : 0) : 0;
      bool valid = !((bx && !(px[k] & 1)) || (by && !(py[k] & 1)) || (D == 3 && bz && !(pz[k] & 1)));
      int X = (px[k] - oxs) >> 1, Y = (py[k] - oys) >> 1, Z = D == 3 ? (pz[k] - ozs) >> 1 : 0;
      valid = valid && X >= 0 && X < p.cx && Y >= 0 && Y < p.cy && Z >= 0 && Z < p.cz;
      if (__syncthreads_or(valid) == 0) continue;
      const int o = D == 3 ? ((ozs + 1) * 3 + (oys + 1)) * 3 + (oxs + 1) : (oys + 1) * 3 + (oxs + 1);
      const float2* w = p.Wt + (size_t)o * p.cin * CO;
      const float2* src = ec + (valid ? (((long long)Z * p.cy + Y) * p.cx + X) * p.cin : 0);
      float2 a = make_float2(0.f, 0.f);
      for (int ci = 0; ci < p.cin; ++ci) {
        const float2 wv = __ldg(w + ci * CO + co);
        const float2 v = __ldg(src + ci);
        cfma(a, wv, v);
      }
      if (valid) acc[k] = cadd(acc[k], a);
    }
  }
#pragma unroll
  for (int k = 0; k < T::TN; ++k)
    if (nn[k] < NF) e[nn[k] * CO + co] = cadd(e[nn[k] * CO + co], acc[k]);
}

template <int CO, int D, int TN>
static mcmg_status transfer_tn(const TransferParams& p, bool restrict_, int nrhs, cudaStream_t st) {
  using T = Tile<CO, TN>;
  dim3 grid((unsigned)((p.dst_nodes + T::NB - 1) / T::NB), (unsigned)nrhs);
  if (restrict_)
    k_restrict<CO, D, TN><<<grid, 256, 0, st>>>(p);
  else
    k_prolong_add<CO, D, TN><<<grid, 256, 0, st>>>(p);
  MCMG_CHECK_LAUNCH(restrict_ ? "restrict" : "prolong_add");
  return MCMG_OK;
}

template <int CO, int D>
static mcmg_status transfer_c(const TransferParams& p, bool restrict_, int nrhs, cudaStream_t st) {
  switch (pick_tn(p.dst_nodes, CO, nrhs)) {
    case 8: return transfer_tn<CO, D, 8>(p, restrict_, nrhs, st);
    case 2: return transfer_tn<CO, D, 2>(p, restrict_, nrhs, st);
    default: return transfer_tn<CO, D, 1>(p, restrict_, nrhs, st);
  }
}

template <int D>
static mcmg_status transfer_d(const TransferParams& p, int CO, bool r, int nrhs, cudaStream_t st) {
  switch (CO) {
    case 1: return transfer_c<1, D>(p, r, nrhs, st);
    case 2: return transfer_c<2, D>(p, r, nrhs, st);
    case 4: return transfer_c<4, D>(p, r, nrhs, st);
    case 8: return transfer_c<8, D>(p, r, nrhs, st);
    case 16: return transfer_c<16, D>(p, r, nrhs, st);
    case 32: return transfer_c<32, D>(p, r, nrhs, st);
    case 64: return transfer_c<64, D>(p, r, nrhs, st);
  }
  set_error("unsupported channel count %d", CO);
  return MCMG_ERR_SHAPE;
}

mcmg_status launch_restrict(const Level& L, const float2* t, float2* rc, int nrhs,
                            cudaStream_t st) {
  Grid gc = L.g.coarse();
  TransferParams p;
  p.src = t;
  p.dst = rc;
  p.Wt = L.Rt;
  p.cin = L.C;
  p.fx = L.g.nx; p.fy = L.g.ny; p.fz = L.g.nz;
  p.cx = gc.nx; p.cy = gc.ny; p.cz = gc.nz;
  p.src_nodes = L.g.nodes();
  p.dst_nodes = gc.nodes();
  return L.g.d == 3 ? transfer_d<3>(p, L.Cn, true, nrhs, st)
                    : transfer_d<2>(p, L.Cn, true, nrhs, st);
}

mcmg_status launch_prolong_add(const Level& L, const float2* ec, float2* e, int nrhs,
                               cudaStream_t st) {
  Grid gc = L.g.coarse();
  TransferParams p;
  p.src = ec;
  p.dst = e;
  p.Wt = L.Pt;
  p.cin = L.Cn;
  p.fx = L.g.nx; p.fy = L.g.ny; p.fz = L.g.nz;
  p.cx = gc.nx; p.cy = gc.ny; p.cz = gc.nz;
  p.src_nodes = gc.nodes();
  p.dst_nodes = L.g.nodes();
  return L.g.d == 3 ? transfer_d<3>(p, L.C, false, nrhs, st)
                    : transfer_d<2>(p, L.C, false, nrhs, st);
}

// ---------------------------------------------------------------------------
// Lift r_1[p][c] = g_lift[c] r[p];  project e[p] = sum_c g_proj[c] e_1[p][c].
// ---------------------------------------------------------------------------
__global__ void k_lift(const float2* __restrict__ r, const float2* __restrict__ lift,
                       float2* __restrict__ r1, int C, long long N) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= N * C) return;
  size_t off = (size_t)blockIdx.y * N;
  r1[off * C + id] = cmul(lift[id % C], r[off + id / C]);
}

__global__ void k_project(const float2* __restrict__ e1, const float2* __restrict__ proj,
                          float2* __restrict__ e, int C, long long N) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  size_t off = (size_t)blockIdx.y * N;
  const float2* src = e1 + (off + n) * C;
  float2 acc = make_float2(0.f, 0.f);
  for (int c = 0; c < C; ++c) cfma(acc, proj[c], src[c]);
  e[off + n] = acc;
}

mcmg_status launch_lift(const float2* r, const float2* lift, float2* r1, int C, long long nodes,
                        int nrhs, cudaStream_t st) {
  dim3 grid((unsigned)((nodes * C + 255) / 256), (unsigned)nrhs);
  k_lift<<<grid, 256, 0, st>>>(r, lift, r1, C, nodes);
  MCMG_CHECK_LAUNCH("lift");
  return MCMG_OK;
}

mcmg_status launch_project(const float2* e1, const float2* proj, float2* e, int C,
                           long long nodes, int nrhs, cudaStream_t st) {
  dim3 grid((unsigned)((nodes + 255) / 256), (unsigned)nrhs);
  k_project<<<grid, 256, 0, st>>>(e1, proj, e, C, nodes);
  MCMG_CHECK_LAUNCH("project");
  return MCMG_OK;
}

}  // namespace mcmg
