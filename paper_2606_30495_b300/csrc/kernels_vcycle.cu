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
#include "vcycle_kernels.cuh"

namespace mcmg {

// Thread shapes.  Thread (cg, g) of a 256-thread block owns the CO
// consecutive output channels cg*CO .. cg*CO + CO - 1 of TN nodes
// n0 + g + G*k (k < TN), with CG = C / CO channel groups and G = 256 / CG
// node groups; a block covers NB = G * TN consecutive nodes.  Each weight load
// (CO complex values, one 32-byte vector load for CO = 4) feeds CO * TN
// complex FMAs.  The shape is chosen per level and mode by the autotuner at
// setup (autotune_smooth); pick_shape is the fallback heuristic.
struct Shape {
  int kind;    // 0: k_smooth (Tile), 1: k_smooth_ks (KsTile), 2: k_smooth_rt (RtTile),
               // 3: k_smooth_rtb (RtTile, matrices staged by bulk copies),
               // 4: k_smooth_tpn (co = output channels per lane)
  int tn, co;  // nodes and output channels per thread
  int kq;      // input channels per K-group (k_smooth_rt)
};
static constexpr Shape kShapes[] = {{0, 8, 1, 0}, {0, 2, 1, 0}, {0, 1, 1, 0}, {0, 2, 4, 0},
                                    {0, 1, 4, 0}, {1, 1, 1, 0}, {2, 8, 4, 4}, {2, 4, 4, 4},
                                    {2, 8, 4, 2}, {2, 4, 4, 2}, {2, 8, 4, 8}, {2, 4, 4, 8},
                                    {3, 8, 4, 4}, {3, 4, 4, 4}, {3, 4, 4, 8},
                                    {4, 1, 8, 0}, {4, 1, 4, 0}, {4, 1, 2, 0}};
static constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
static constexpr int kTunePasses = 3, kTuneReps = 10;   // autotuner timing

static bool shape_ok(int s, int C, int D) {
  const Shape& k = kShapes[s];
  if (k.kind == 4) return (C == 4 || C == 8 || C == 16 || C == 32) && k.co <= C && C / k.co <= 16;
  if (k.kind == 1) return C >= 8;
  if (k.kind == 2 || k.kind == 3) {
    if (k.kind == 3 && C < 8) return false;
    const size_t b = rt_smem(C, D, k.tn, k.co, k.kq, k.kind == 3);
    return b > 0 && b <= kMaxSmem;
  }
  return k.co <= C;
}

// Largest nodes-per-thread (8, 2 or 1, one channel per thread) that still
// gives at least two blocks per SM.
static int pick_shape(long long nodes, int C, int nrhs) {
  const long long want = 2 * 148;
  const int G = 256 / C;
  for (int s = 0; s < 2; ++s) {
    const int tn = kShapes[s].tn;
    long long blocks = (nodes + (long long)G * tn - 1) / ((long long)G * tn) * nrhs;
    if (blocks >= want) return s;
  }
  return 2;
}

// Largest nodes-per-thread (8, 2 or 1) for the transfer kernels.
static int pick_tn(long long nodes, int C, int nrhs) {
  return kShapes[pick_shape(nodes, C, nrhs)].tn;
}

template <int C, int D, int MODE, int TN, int CO>
__global__ void __launch_bounds__(256) k_smooth(SmoothParams p) {
  pdl_launch_dependents();
  pdl_wait();
  using T = Tile<C, TN, CO>;
  extern __shared__ float2 sm[];
  const int cg = threadIdx.x % T::CG;
  const int g = threadIdx.x / T::CG;
  const int co0 = cg * CO;
  const long long N = p.nodes;
  const size_t off = (size_t)blockIdx.y * (size_t)N * C;
  const float2* __restrict__ r = p.r + off;
  const float2* __restrict__ ein = p.e_in ? p.e_in + off : nullptr;
  float2* __restrict__ eout = p.e_out + off;
  const long long n0 = (long long)blockIdx.x * T::NB;

  long long nn[TN];
  long long nc[TN];  // clamped (always a valid node)
#pragma unroll
  for (int k = 0; k < TN; ++k) {
    nn[k] = n0 + g + (long long)T::G * k;
    nc[k] = nn[k] < N ? nn[k] : N - 1;
  }

  float2 t[TN][CO];
  if (ein) {
    float2 acc[TN][CO], acca[TN][CO];
    int cx[TN], cy[TN], cz[TN];
#pragma unroll
    for (int k = 0; k < TN; ++k) {
      node_xyz(nc[k], p.nx, p.ny, cx[k], cy[k], cz[k]);
#pragma unroll
      for (int c = 0; c < CO; ++c) {
        acc[k][c] = make_float2(0.f, 0.f);
        acca[k][c] = make_float2(0.f, 0.f);
      }
    }
    // centre tap and K_A share the loads of e at the node itself
    for (int ci = 0; ci < C; ++ci) {
      float2 w0[CO], wa[CO];
      ldc<CO>(p.Wt + ci * C + co0, w0);
      ldc<CO>(p.KAt + ci * C + co0, wa);
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        const float2 v = __ldg(ein + nc[k] * C + ci);
#pragma unroll
        for (int c = 0; c < CO; ++c) {
          cfma(acc[k][c], w0[c], v);
          cfma(acca[k][c], wa[c], v);
        }
      }
    }
    const long long sxy = (long long)p.nx * p.ny;
#pragma unroll
    for (int tap = 1; tap <= 2 * D; ++tap) {
      const int axis = (tap - 1) >> 1;
      const int sgn = (tap & 1) ? -1 : 1;
      long long nb[TN];
      bool ok[TN];
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        int c = axis == 0 ? cx[k] : (axis == 1 ? cy[k] : cz[k]);
        int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
        long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : sxy);
        ok[k] = (c + sgn >= 0) && (c + sgn < ext);
        nb[k] = ok[k] ? nc[k] + sgn * stride : nc[k];
      }
      const float2* wt = p.Wt + (size_t)tap * C * C;
      for (int ci = 0; ci < C; ++ci) {
        float2 w[CO];
        ldc<CO>(wt + ci * C + co0, w);
#pragma unroll
        for (int k = 0; k < TN; ++k) {
          const float2 v = __ldg(ein + nb[k] * C + ci);
          if (ok[k]) {
#pragma unroll
            for (int c = 0; c < CO; ++c) cfma(acc[k][c], w[c], v);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < TN; ++k) {
      float2 rv[CO], av[CO];
      ldc<CO>(r + nc[k] * C + co0, rv);
      ldc<CO>(p.a + nc[k] * C + co0, av);
#pragma unroll
      for (int c = 0; c < CO; ++c) t[k][c] = csub(csub(rv[c], acc[k][c]), cmul(av[c], acca[k][c]));
    }
  } else {
#pragma unroll
    for (int k = 0; k < TN; ++k) ldc<CO>(r + nc[k] * C + co0, t[k]);
  }

  if (MODE == 1) {  // residual only
#pragma unroll
    for (int k = 0; k < TN; ++k)
      if (nn[k] < N) stc<CO>(eout + nn[k] * C + co0, t[k]);
    return;
  }

  float2* sm_t = sm;
  float2* sm_z = sm + T::NB * C;
#pragma unroll
  for (int k = 0; k < TN; ++k)
#pragma unroll
    for (int c = 0; c < CO; ++c) sm_t[(g + T::G * k) * C + co0 + c] = t[k][c];
  __syncthreads();

  // z = s (.) (K_S t)
  float2 z[TN][CO];
#pragma unroll
  for (int k = 0; k < TN; ++k)
#pragma unroll
    for (int c = 0; c < CO; ++c) z[k][c] = make_float2(0.f, 0.f);
  for (int ci = 0; ci < C; ++ci) {
    float2 w[CO];
    ldc<CO>(p.KSt + ci * C + co0, w);
#pragma unroll
    for (int k = 0; k < TN; ++k) {
      const float2 v = sm_t[(g + T::G * k) * C + ci];
#pragma unroll
      for (int c = 0; c < CO; ++c) cfma(z[k][c], w[c], v);
    }
  }
#pragma unroll
  for (int k = 0; k < TN; ++k) {
    float2 sv[CO];
    ldc<CO>(p.s + nc[k] * C + co0, sv);
#pragma unroll
    for (int c = 0; c < CO; ++c) {
      z[k][c] = cmul(sv[c], z[k][c]);
      sm_z[(g + T::G * k) * C + co0 + c] = z[k][c];
    }
  }
  __syncthreads();

  // e' = e + W^(i) z
  float2 u[TN][CO];
#pragma unroll
  for (int k = 0; k < TN; ++k)
#pragma unroll
    for (int c = 0; c < CO; ++c) u[k][c] = make_float2(0.f, 0.f);
  for (int ci = 0; ci < C; ++ci) {
    float2 w[CO];
    ldc<CO>(p.Wst + ci * C + co0, w);
#pragma unroll
    for (int k = 0; k < TN; ++k) {
      const float2 v = sm_z[(g + T::G * k) * C + ci];
#pragma unroll
      for (int c = 0; c < CO; ++c) cfma(u[k][c], w[c], v);
    }
  }
#pragma unroll
  for (int k = 0; k < TN; ++k) {
    if (nn[k] < N) {
      if (ein) {
        float2 ev[CO];
        ldc<CO>(ein + nn[k] * C + co0, ev);
#pragma unroll
        for (int c = 0; c < CO; ++c) u[k][c] = cadd(u[k][c], ev[c]);
      }
      stc<CO>(eout + nn[k] * C + co0, u[k]);
    }
  }
}

template <int C, int D, int TN, int CO>
static mcmg_status smooth_shape(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  if constexpr (CO > C) {
    set_error("thread shape wider than the channel count");
    return MCMG_ERR_SHAPE;
  } else {
    using T = Tile<C, TN, CO>;
    dim3 grid((unsigned)((p.nodes + T::NB - 1) / T::NB), (unsigned)nrhs);
    size_t smem = mode == 0 ? 2 * (size_t)T::NB * C * sizeof(float2) : 0;
    if (mode == 0)
      MCMG_LAUNCH_PDL((k_smooth<C, D, 0, TN, CO>), grid, dim3(256), smem, st, p);
    else
      MCMG_LAUNCH_PDL((k_smooth<C, D, 1, TN, CO>), grid, dim3(256), smem, st, p);
    MCMG_CHECK_LAUNCH("smooth");
    return MCMG_OK;
  }
}


// K-split shape for coarse levels (few nodes, many channels): four lanes share
// one (node, output channel) pair and each sums a quarter of the input
// channels; two warp shuffles combine the partial sums.  A warp holds 8
// output channels x 4 quarters of one node, a 256-thread block NB = 64 / C * 8
// nodes' worth of C / 8 warps each.  Four times the threads of the one-output
// shape, so the latency of the weight and field loads is hidden by other warps.
template <int C>
struct KsTile {
  static constexpr int WPN = C / 8;          // warps per node
  static constexpr int NB = 8 / WPN;         // nodes per block
  static constexpr int KQ = C / 4;           // input channels per quarter
};

__device__ __forceinline__ float2 quad_sum(float2 v) {
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 8);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 8);
  v.x += __shfl_xor_sync(0xffffffffu, v.x, 16);
  v.y += __shfl_xor_sync(0xffffffffu, v.y, 16);
  return v;
}

template <int C, int D, int MODE>
__global__ void __launch_bounds__(256) k_smooth_ks(SmoothParams p) {
  pdl_launch_dependents();
  pdl_wait();
  using T = KsTile<C>;
  __shared__ float2 sm_t[T::NB * C];
  __shared__ float2 sm_z[T::NB * C];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = warp / T::WPN;                       // node within the block
  const int co = (warp % T::WPN) * 8 + (lane & 7);    // output channel
  const int q = lane >> 3;                            // input-channel quarter
  const int ci0 = q * T::KQ;
  const long long N = p.nodes;
  const size_t off = (size_t)blockIdx.y * (size_t)N * C;
  const float2* __restrict__ r = p.r + off;
  const float2* __restrict__ ein = p.e_in ? p.e_in + off : nullptr;
  float2* __restrict__ eout = p.e_out + off;
  const long long n = (long long)blockIdx.x * T::NB + nl;
  const long long nc = n < N ? n : N - 1;

  float2 t;
  if (ein) {
    float2 acc = make_float2(0.f, 0.f), acca = make_float2(0.f, 0.f);
    int cx, cy, cz;
    node_xyz(nc, p.nx, p.ny, cx, cy, cz);
    for (int ci = ci0; ci < ci0 + T::KQ; ++ci) {
      const float2 v = __ldg(ein + nc * C + ci);
      cfma(acc, __ldg(p.Wt + ci * C + co), v);
      cfma(acca, __ldg(p.KAt + ci * C + co), v);
    }
    const long long sxy = (long long)p.nx * p.ny;
#pragma unroll
    for (int tap = 1; tap <= 2 * D; ++tap) {
      const int axis = (tap - 1) >> 1;
      const int sgn = (tap & 1) ? -1 : 1;
      const int c = axis == 0 ? cx : (axis == 1 ? cy : cz);
      const int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
      const long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : sxy);
      if (c + sgn < 0 || c + sgn >= ext) continue;
      const float2* e_nb = ein + (nc + sgn * stride) * C;
      const float2* wt = p.Wt + (size_t)tap * C * C;
      for (int ci = ci0; ci < ci0 + T::KQ; ++ci) cfma(acc, __ldg(wt + ci * C + co), __ldg(e_nb + ci));
    }
    acc = quad_sum(acc);
    acca = quad_sum(acca);
    t = csub(csub(__ldg(r + nc * C + co), acc), cmul(__ldg(p.a + nc * C + co), acca));
  } else {
    t = __ldg(r + nc * C + co);
  }
  if (MODE == 1) {
    if (q == 0 && n < N) eout[n * C + co] = t;
    return;
  }
  if (q == 0) sm_t[nl * C + co] = t;
  __syncthreads();
  float2 z = make_float2(0.f, 0.f);
  for (int ci = ci0; ci < ci0 + T::KQ; ++ci) cfma(z, __ldg(p.KSt + ci * C + co), sm_t[nl * C + ci]);
  z = cmul(__ldg(p.s + nc * C + co), quad_sum(z));
  if (q == 0) sm_z[nl * C + co] = z;
  __syncthreads();
  float2 u = make_float2(0.f, 0.f);
  for (int ci = ci0; ci < ci0 + T::KQ; ++ci) cfma(u, __ldg(p.Wst + ci * C + co), sm_z[nl * C + ci]);
  u = quad_sum(u);
  if (q == 0 && n < N) eout[n * C + co] = ein ? cadd(u, ein[n * C + co]) : u;
}

template <int C, int D>
static mcmg_status smooth_ks(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  if constexpr (C < 8) {
    set_error("the K-split shape needs at least 8 channels");
    return MCMG_ERR_SHAPE;
  } else {
    using T = KsTile<C>;
    dim3 grid((unsigned)((p.nodes + T::NB - 1) / T::NB), (unsigned)nrhs);
    if (mode == 0)
      MCMG_LAUNCH_PDL((k_smooth_ks<C, D, 0>), grid, dim3(256), 0, st, p);
    else
      MCMG_LAUNCH_PDL((k_smooth_ks<C, D, 1>), grid, dim3(256), 0, st, p);
    MCMG_CHECK_LAUNCH("smooth_ks");
    return MCMG_OK;
  }
}

// Thread-per-node smoothing step for few channels (C = 4 .. 32).  G = C / CT
// adjacent lanes share a node, each owning CT output channels; a block covers
// 256 / G nodes.  Every mixing matrix of the step sits in shared memory and is
// read as a broadcast (all nodes' lanes read the same weights); each lane loads
// the C values of every tap of its node with 16-byte loads (a warp reads
// whole rows of consecutive nodes); t and z stay in registers and reach a
// node's G lanes through warp shuffles.  No block barrier after the weights
// are staged, no shared-memory traffic for the fields.
template <int C, int D, int MODE, int CT>
__global__ void __launch_bounds__(256) k_smooth_tpn(SmoothParams p) {
  pdl_launch_dependents();
  constexpr int G = C / CT, NPB = 256 / G, NT = 2 * D + 1, MSZ = C * C, NM = NT + 3;
  extern __shared__ float4 wsm4[];
  float2* Wsm = reinterpret_cast<float2*>(wsm4);   // [NM][C][C]: taps, K_A, K_S, W^(i)
  for (int i = threadIdx.x; i < NM * MSZ / 2; i += 256) {   // setup-time data
    const int m = (2 * i) / MSZ, o = (2 * i) % MSZ;
    const float2* src = m < NT ? p.Wt + (size_t)m * MSZ
                               : (m == NT ? p.KAt : (m == NT + 1 ? p.KSt : p.Wst));
    wsm4[i] = __ldg(reinterpret_cast<const float4*>(src + o));
  }
  __syncthreads();
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int g = threadIdx.x % G;
  const int base = lane - g;                        // first lane of this node
  const long long N = p.nodes;
  const long long n = (long long)blockIdx.x * NPB + threadIdx.x / G;
  const bool live = n < N;
  const long long nc = live ? n : N - 1;            // every lane joins the shuffles
  const size_t off = (size_t)blockIdx.y * (size_t)N * C;
  const float2* __restrict__ r = p.r + off;
  const float2* __restrict__ ein = p.e_in ? p.e_in + off : nullptr;
  float2* __restrict__ eout = p.e_out + off;
  const int c0 = g * CT;

  auto load_vec = [&](const float2* q, float2* x, int cnt) {   // cnt complex, 16-byte loads
    const float4* q4 = reinterpret_cast<const float4*>(q);
    for (int i = 0; i < cnt / 2; ++i) {
      const float4 v = __ldg(q4 + i);
      x[2 * i] = make_float2(v.x, v.y);
      x[2 * i + 1] = make_float2(v.z, v.w);
    }
  };
  // acc[co] += sum_ci M[c0 + co][ci] x[ci], M^T[ci][.] in shared memory
  auto mix = [&](const float2* Mt, const float2 (&x)[C], float2 (&acc)[CT]) {
#pragma unroll
    for (int ci = 0; ci < C; ++ci) {
      const float4* w4 = reinterpret_cast<const float4*>(Mt + ci * C + c0);
#pragma unroll
      for (int h = 0; h < CT / 2; ++h) {
        const float4 w = w4[h];
        cfma(acc[2 * h], make_float2(w.x, w.y), x[ci]);
        cfma(acc[2 * h + 1], make_float2(w.z, w.w), x[ci]);
      }
    }
  };
  // all C values of a node from its G lanes' CT each
  auto gather = [&](const float2 (&v)[CT], float2 (&all)[C]) {
#pragma unroll
    for (int q = 0; q < G; ++q)
#pragma unroll
      for (int co = 0; co < CT; ++co) {
        if constexpr (G == 1) {
          all[co] = v[co];
        } else {
          all[q * CT + co] = make_float2(__shfl_sync(0xffffffffu, v[co].x, base + q),
                                         __shfl_sync(0xffffffffu, v[co].y, base + q));
        }
      }
  };

  float2 t[CT];
  if (ein) {
    float2 acc[CT], accA[CT];
#pragma unroll
    for (int co = 0; co < CT; ++co) acc[co] = accA[co] = make_float2(0.f, 0.f);
    const int ni = (int)nc, rest = ni / p.nx;
    const int cx = ni - rest * p.nx, cy = rest % p.ny, cz = rest / p.ny;
    const long long sxy = (long long)p.nx * p.ny;
#pragma unroll
    for (int tap = 0; tap < NT; ++tap) {
      long long nb = nc;
      bool ok = true;
      if (tap > 0) {
        const int axis = (tap - 1) >> 1;
        const int sgn = (tap & 1) ? -1 : 1;
        const int c = axis == 0 ? cx : (axis == 1 ? cy : cz);
        const int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
        const long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : sxy);
        ok = c + sgn >= 0 && c + sgn < ext;
        nb = ok ? nc + sgn * stride : nc;
      }
      float2 x[C];
      load_vec(ein + nb * C, x, C);
      if (!ok)
#pragma unroll
        for (int ci = 0; ci < C; ++ci) x[ci] = make_float2(0.f, 0.f);
      mix(Wsm + tap * MSZ, x, acc);
      if (tap == 0) mix(Wsm + NT * MSZ, x, accA);
    }
    float2 rv[CT], av[CT];
    load_vec(r + nc * C + c0, rv, CT);
    load_vec(p.a + nc * C + c0, av, CT);
#pragma unroll
    for (int co = 0; co < CT; ++co) t[co] = csub(csub(rv[co], acc[co]), cmul(av[co], accA[co]));
    if (MODE == 1) {
      if (live) {
        float4* o4 = reinterpret_cast<float4*>(eout + n * C + c0);
#pragma unroll
        for (int h = 0; h < CT / 2; ++h)
          o4[h] = make_float4(t[2 * h].x, t[2 * h].y, t[2 * h + 1].x, t[2 * h + 1].y);
      }
      return;
    }
  } else {
    load_vec(r + nc * C + c0, t, CT);
  }
  // z = s (.) (K_S t)
  float2 all[C], z[CT], sv[CT];
  gather(t, all);
#pragma unroll
  for (int co = 0; co < CT; ++co) z[co] = make_float2(0.f, 0.f);
  mix(Wsm + (NT + 1) * MSZ, all, z);
  load_vec(p.s + nc * C + c0, sv, CT);
#pragma unroll
  for (int co = 0; co < CT; ++co) z[co] = cmul(sv[co], z[co]);
  // e' = e + W^(i) z
  gather(z, all);
  float2 u[CT];
#pragma unroll
  for (int co = 0; co < CT; ++co) u[co] = make_float2(0.f, 0.f);
  mix(Wsm + (NT + 2) * MSZ, all, u);
  if (live) {
    if (ein) {
      float2 ev[CT];
      load_vec(ein + n * C + c0, ev, CT);
#pragma unroll
      for (int co = 0; co < CT; ++co) u[co] = cadd(u[co], ev[co]);
    }
    float4* o4 = reinterpret_cast<float4*>(eout + n * C + c0);
#pragma unroll
    for (int h = 0; h < CT / 2; ++h)
      o4[h] = make_float4(u[2 * h].x, u[2 * h].y, u[2 * h + 1].x, u[2 * h + 1].y);
  }
}

template <int C, int CT>
constexpr bool tpn_valid() {
  return (C == 4 || C == 8 || C == 16 || C == 32) && (CT == 2 || CT == 4 || CT == 8) && CT <= C &&
         C / CT <= 16;
}

template <int C, int D, int CT>
static mcmg_status smooth_tpn(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  if constexpr (!tpn_valid<C, CT>()) {
    set_error("thread-per-node shape does not fit %d channels", C);
    return MCMG_ERR_SHAPE;
  } else {
    constexpr int NPB = 256 / (C / CT);
    constexpr size_t smem = (size_t)(2 * D + 4) * C * C * sizeof(float2);
    dim3 grid((unsigned)((p.nodes + NPB - 1) / NPB), (unsigned)nrhs);
    if (mode == 0) {
      if (smem > 48 * 1024)
        MCMG_CUDA(cudaFuncSetAttribute(k_smooth_tpn<C, D, 0, CT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL((k_smooth_tpn<C, D, 0, CT>), grid, dim3(256), smem, st, p);
    } else {
      if (smem > 48 * 1024)
        MCMG_CUDA(cudaFuncSetAttribute(k_smooth_tpn<C, D, 1, CT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL((k_smooth_tpn<C, D, 1, CT>), grid, dim3(256), smem, st, p);
    }
    MCMG_CHECK_LAUNCH("smooth_tpn");
    return MCMG_OK;
  }
}

template <int C, int D>
static mcmg_status smooth_c(const SmoothParams& p, int mode, int shape, int nrhs, cudaStream_t st) {
  switch (shape) {
    case 0: return smooth_shape<C, D, 8, 1>(p, mode, nrhs, st);
    case 1: return smooth_shape<C, D, 2, 1>(p, mode, nrhs, st);
    case 2: return smooth_shape<C, D, 1, 1>(p, mode, nrhs, st);
    case 3: return smooth_shape<C, D, 2, 4>(p, mode, nrhs, st);
    case 4: return smooth_shape<C, D, 1, 4>(p, mode, nrhs, st);
    case 5: return smooth_ks<C, D>(p, mode, nrhs, st);
    case 15: return smooth_tpn<C, D, 8>(p, mode, nrhs, st);
    case 16: return smooth_tpn<C, D, 4>(p, mode, nrhs, st);
    case 17: return smooth_tpn<C, D, 2>(p, mode, nrhs, st);
    default:
      return smooth_rt_launch(p, C, D, mode, kShapes[shape].tn, kShapes[shape].co,
                              kShapes[shape].kq, kShapes[shape].kind == 3, nrhs, st);
  }
}

template <int D>
static mcmg_status smooth_d(const SmoothParams& p, int C, int mode, int shape, int nrhs,
                            cudaStream_t st) {
  switch (C) {
    case 1: return smooth_c<1, D>(p, mode, shape, nrhs, st);
    case 2: return smooth_c<2, D>(p, mode, shape, nrhs, st);
    case 4: return smooth_c<4, D>(p, mode, shape, nrhs, st);
    case 8: return smooth_c<8, D>(p, mode, shape, nrhs, st);
    case 16: return smooth_c<16, D>(p, mode, shape, nrhs, st);
    case 32: return smooth_c<32, D>(p, mode, shape, nrhs, st);
    case 64: return smooth_c<64, D>(p, mode, shape, nrhs, st);
  }
  set_error("unsupported channel count %d", C);
  return MCMG_ERR_SHAPE;
}

static SmoothParams smooth_params(const Level& L, int step, const float2* r, const float2* e_in,
                                  float2* e_out, int mode) {
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
  p.err = L.err;
  return p;
}

static mcmg_status smooth_run(const Level& L, const SmoothParams& p, int mode, int shape, int nrhs,
                              cudaStream_t st) {
  return L.g.d == 3 ? smooth_d<3>(p, L.C, mode, shape, nrhs, st)
                    : smooth_d<2>(p, L.C, mode, shape, nrhs, st);
}

mcmg_status launch_smooth(const Level& L, int step, const float2* r, const float2* e_in,
                          float2* e_out, int mode, int nrhs, cudaStream_t st) {
  if (L.use_ts && (mode == 0 || e_in))
    return launch_smooth_ts(L, step, r, e_in, e_out, mode, nrhs, st);
  const SmoothParams p = smooth_params(L, step, r, e_in, e_out, mode);
  int shape = L.shape[mode];
  if (shape < 0 || !shape_ok(shape, L.C, L.g.d)) shape = pick_shape(p.nodes, L.C, nrhs);
  return smooth_run(L, p, mode, shape, nrhs, st);
}

// Autotuner: time every valid thread shape of the CUDA-core smoothing kernel
// on this level (the step with e and the residual mode) with CUDA events on
// scratch fields, and keep the fastest in L.shape[mode].  Three passes of ten
// launches over the shapes, keeping each shape's best time, so a clock still
// ramping up or a noisy pass does not decide.  Run once per medium at setup, before any
// V-cycle graph is captured.
mcmg_status autotune_smooth(Level& L, float2* r, float2* e, float2* out, cudaStream_t st) {
  cudaEvent_t e0, e1;
  MCMG_CUDA(cudaEventCreate(&e0));
  MCMG_CUDA(cudaEventCreate(&e1));
  mcmg_status status = MCMG_OK;
  for (int mode = 0; mode < 2 && status == MCMG_OK; ++mode) {
    if (L.use_ts) continue;
    const SmoothParams p = smooth_params(L, 0, r, e, out, mode);
    float best_ms[kNumShapes];
    for (int s = 0; s < kNumShapes; ++s) best_ms[s] = 1e30f;
    for (int pass = 0; pass < kTunePasses && status == MCMG_OK; ++pass) {
      for (int s = 0; s < kNumShapes; ++s) {
        if (!shape_ok(s, L.C, L.g.d)) continue;
        for (int rep = 0; rep < 2; ++rep)
          if ((status = smooth_run(L, p, mode, s, 1, st)) != MCMG_OK) break;
        if (status != MCMG_OK) break;
        cudaEventRecord(e0, st);
        const int reps = kTuneReps;
        for (int rep = 0; rep < reps; ++rep)
          if ((status = smooth_run(L, p, mode, s, 1, st)) != MCMG_OK) break;
        if (status != MCMG_OK) break;
        cudaEventRecord(e1, st);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) { status = cuda_fail(ce, "autotune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms[s]) best_ms[s] = ms;
      }
    }
    int best_s = -1;
    for (int s = 0; s < kNumShapes; ++s)
      if (best_ms[s] < 1e29f && (best_s < 0 || best_ms[s] < best_ms[best_s])) best_s = s;
    L.shape[mode] = best_s;
    L.tuned[mode] = best_s;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

// ---------------------------------------------------------------------------
// Restriction: rc[J][co] = sum_{o in {-1,0,1}^d} sum_ci R[o][co][ci] t[2J+o][ci]
// (multi-channel strided convolution, stride 2, zero padding).  Thread (co, g)
// owns output channel co of TN coarse nodes.
// ---------------------------------------------------------------------------
template <int CO, int D, int TN>
__global__ void __launch_bounds__(256) k_restrict(TransferParams p) {
  pdl_launch_dependents();
  pdl_wait();
  using T = Tile<CO, TN, 1>;
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

// Prolongation-add, coarse-node form: the transposed strided convolution
// x[2J + o] += P[o] e_c[J] is regrouped by coarse node.  For tap o, write
// b_a = (o_a != 0) and c_a = (o_a == -1) per axis; then fine node 2J + b(o)
// receives P[o] e_c[J + c(o)].  A thread owning coarse node J therefore
// computes its 2^d fine nodes 2J + {0,1}^d (the grid is even, so all exist)
// with every tap used exactly once and no divergent control flow; e_c outside
// the coarse grid is zero.
template <int CO, int D, int TN>
__global__ void __launch_bounds__(256) k_prolong_add(TransferParams p) {
  pdl_launch_dependents();
  pdl_wait();
  using T = Tile<CO, TN, 1>;
  constexpr int NB2 = D == 3 ? 8 : 4;
  constexpr int T3 = D == 3 ? 27 : 9;
  const int co = threadIdx.x % CO;
  const int g = threadIdx.x / CO;
  const long long NC = p.src_nodes;
  const float2* __restrict__ ec = p.src + (size_t)blockIdx.y * NC * p.cin;
  float2* __restrict__ e = p.dst + (size_t)blockIdx.y * p.dst_nodes * CO;
  const long long n0 = (long long)blockIdx.x * T::NB;
  long long nn[TN];
  int jx[TN], jy[TN], jz[TN];
  float2 acc[TN][NB2];
#pragma unroll
  for (int k = 0; k < TN; ++k) {
    nn[k] = n0 + g + (long long)T::G * k;
    const long long c = nn[k] < NC ? nn[k] : NC - 1;
    node_xyz(c, p.cx, p.cy, jx[k], jy[k], jz[k]);
#pragma unroll
    for (int b = 0; b < NB2; ++b) acc[k][b] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int o = 0; o < T3; ++o) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = D == 3 ? o / 9 - 1 : 0;
    const int b = (ox != 0) | ((oy != 0) << 1) | ((oz != 0) << 2);
    const int cx = ox == -1, cy = oy == -1, cz = oz == -1;
    long long src[TN];
    bool ok[TN];
#pragma unroll
    for (int k = 0; k < TN; ++k) {
      const int X = jx[k] + cx, Y = jy[k] + cy, Z = jz[k] + cz;
      ok[k] = X < p.cx && Y < p.cy && (D == 3 ? Z < p.cz : true);
      src[k] = ok[k] ? (((long long)Z * p.cy + Y) * p.cx + X) * p.cin : 0;
    }
    const float2* w = p.Wt + (size_t)o * p.cin * CO;
    for (int ci = 0; ci < p.cin; ++ci) {
      const float2 wv = __ldg(w + ci * CO + co);
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        const float2 v = __ldg(ec + src[k] + ci);
        if (ok[k]) cfma(acc[k][b], wv, v);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < TN; ++k) {
    if (nn[k] >= NC) continue;
#pragma unroll
    for (int b = 0; b < NB2; ++b) {
      const long long fx = 2 * jx[k] + (b & 1), fy = 2 * jy[k] + ((b >> 1) & 1),
                      fz = D == 3 ? 2 * jz[k] + ((b >> 2) & 1) : 0;
      const long long fi = ((fz * p.fy + fy) * p.fx + fx) * CO + co;
      e[fi] = cadd(e[fi], acc[k][b]);
    }
  }
}

// Register-tiled transfers.  Same scheme as k_smooth_rt: thread
// (kg, ng, cg) holds a TN x CV output tile and sums the KQ input channels
// kg*KQ .. +KQ-1 over every tap; the block stages the source values its
// nodes read ([offset][node][CI], zero outside the grid) and adds the KS
// partial tiles through shared memory.  A weight load feeds TN nodes.
// Transfer shapes: 0 is the one-channel-per-thread kernel above.
struct TShape {
  int tn, cv, kq;
};
// kq < 0: thread per coarse node (k_restrict_tpn / k_prolong_tpn), cv channels per lane
static constexpr TShape kTShapes[] = {{0, 0, 0}, {1, 4, 4}, {2, 4, 4}, {1, 4, 8}, {2, 4, 8},
                                     {1, 4, 2}, {1, 2, -1}, {1, 4, -1}, {1, 8, -1}};
static constexpr int kNumTShapes = sizeof(kTShapes) / sizeof(kTShapes[0]);
// The shape after the table: the tensor-core transfer (kernels_xts.cu), on
// tensor-core levels whose input side has at least 16 channels (restriction: 8).
static constexpr int kXtsShape = kNumTShapes;
// and, prolongation only, the block form of it (all parity classes at once)
static constexpr int kXtsBlockShape = kNumTShapes + 1;
// and, restriction from 8 channels only, the line-staged form
static constexpr int kXtsLineShape = kNumTShapes + 2;
static constexpr int kNumXShapes = kNumTShapes + 3;

// Register-tiled transfers are built for channel pairs (fine, coarse) with
// the coarse count equal to or twice the fine one; other pairs use shape 0.
static bool xt_pair(int Cf, int Cc) {
  return (Cf == 4 || Cf == 8 || Cf == 16 || Cf == 32 || Cf == 64) && (Cc == Cf || Cc == 2 * Cf) &&
         Cc <= 64;
}

// Shared memory of a register-tiled transfer (0: shape cannot run).
static size_t xt_smem(bool restrict_, int CI, int CO, int D, int tn, int cv, int kq) {
  if (kq < 0) {   // thread per coarse node: the weights only
    const int G = cv > 0 && CO % cv == 0 ? CO / cv : 0;
    const int NP = D == 3 ? 8 : 4;
    if (G < 1 || 32 % G || CI > 32 || CI % 2 || cv % 2 || (!restrict_ && NP * cv > 32)) return 0;
    return (size_t)(D == 3 ? 27 : 9) * CI * CO * sizeof(float2);
  }
  if (cv > CO || CO % cv || kq > CI || CI % kq || CI % 2) return 0;
  const int cg = CO / cv, ks = CI / kq;
  if (cg * ks > 256 || 256 % (cg * ks)) return 0;
  const size_t nb = (size_t)(256 / (cg * ks)) * tn;
  const size_t T3 = D == 3 ? 27 : 9, NP = D == 3 ? 8 : 4;
  const size_t f2 = restrict_ ? T3 * nb * CI + ks * nb * CO : NP * nb * CI + ks * nb * NP * CO;
  return f2 * sizeof(float2);
}

template <int CO, int D, int TN>
static mcmg_status transfer_tn(const TransferParams& p, bool restrict_, int nrhs, cudaStream_t st) {
  using T = Tile<CO, TN, 1>;
  // restriction: one thread per coarse output; prolongation: per coarse source
  const long long units = restrict_ ? p.dst_nodes : p.src_nodes;
  dim3 grid((unsigned)((units + T::NB - 1) / T::NB), (unsigned)nrhs);
  if (restrict_)
    MCMG_LAUNCH_PDL((k_restrict<CO, D, TN>), grid, dim3(256), 0, st, p);
  else
    MCMG_LAUNCH_PDL((k_prolong_add<CO, D, TN>), grid, dim3(256), 0, st, p);
  MCMG_CHECK_LAUNCH(restrict_ ? "restrict" : "prolong_add");
  return MCMG_OK;
}

template <int CO, int D>
static mcmg_status transfer_c(const TransferParams& p, bool restrict_, int nrhs, cudaStream_t st) {
  switch (pick_tn(restrict_ ? p.dst_nodes : p.src_nodes, CO, nrhs)) {
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

static TransferParams transfer_params(const Level& L, bool restrict_, const float2* src,
                                      float2* dst) {
  Grid gc = L.g.coarse();
  TransferParams p;
  p.src = src;
  p.dst = dst;
  p.Wt = restrict_ ? L.Rt : L.Pt;
  p.cin = restrict_ ? L.C : L.Cn;
  p.fx = L.g.nx; p.fy = L.g.ny; p.fz = L.g.nz;
  p.cx = gc.nx; p.cy = gc.ny; p.cz = gc.nz;
  p.src_nodes = restrict_ ? L.g.nodes() : gc.nodes();
  p.dst_nodes = restrict_ ? gc.nodes() : L.g.nodes();
  return p;
}

static bool xshape_ok(int s, const Level& L, bool restrict_) {
  if (s == 0) return true;
  if (s == kXtsShape) return xts_supported(L, restrict_);
  if (s == kXtsBlockShape) return !restrict_ && xts_block_supported(L);
  if (s == kXtsLineShape) return restrict_ && xts_lines_supported(L);
  if (!xt_pair(L.C, L.Cn)) return false;
  const TShape& k = kTShapes[s];
  const int CI = restrict_ ? L.C : L.Cn, CO = restrict_ ? L.Cn : L.C;
  const size_t b = xt_smem(restrict_, CI, CO, L.g.d, k.tn, k.cv, k.kq);
  return b > 0 && b <= kMaxSmem;
}

static mcmg_status transfer_run(const Level& L, const TransferParams& p, bool restrict_, int shape,
                                int nrhs, cudaStream_t st) {
  if (shape == kXtsShape) return launch_transfer_ts(L, restrict_, p.src, p.dst, nrhs, st);
  if (shape == kXtsBlockShape) return launch_prolong_block_ts(L, p.src, p.dst, nrhs, st);
  if (shape == kXtsLineShape) return launch_restrict_lines_ts(L, p.src, p.dst, nrhs, st);
  if (shape > 0)
    return transfer_rt_launch(p, L.C, L.Cn, L.g.d, restrict_, kTShapes[shape].tn,
                              kTShapes[shape].cv, kTShapes[shape].kq, nrhs, st);
  const int CO = restrict_ ? L.Cn : L.C;
  return L.g.d == 3 ? transfer_d<3>(p, CO, restrict_, nrhs, st)
                    : transfer_d<2>(p, CO, restrict_, nrhs, st);
}

mcmg_status launch_restrict(const Level& L, const float2* t, float2* rc, int nrhs,
                            cudaStream_t st) {
  int shape = L.shape[2];
  if (shape < 0 || !xshape_ok(shape, L, true)) shape = 0;
  return transfer_run(L, transfer_params(L, true, t, rc), true, shape, nrhs, st);
}

mcmg_status launch_prolong_add(const Level& L, const float2* ec, float2* e, int nrhs,
                               cudaStream_t st) {
  int shape = L.shape[3];
  if (shape < 0 || !xshape_ok(shape, L, false)) shape = 0;
  return transfer_run(L, transfer_params(L, false, ec, e), false, shape, nrhs, st);
}

// Autotuner for the transfers of level L (L.shape[2] restriction, [3]
// prolongation): timed passes over the valid shapes, as for smoothing.
// fine, coarse: scratch fields of at least nodes_l * C_l and
// nodes_{l+1} * C_{l+1} elements.
mcmg_status autotune_transfer(Level& L, float2* fine, float2* coarse, cudaStream_t st) {
  cudaEvent_t e0, e1;
  MCMG_CUDA(cudaEventCreate(&e0));
  MCMG_CUDA(cudaEventCreate(&e1));
  mcmg_status status = MCMG_OK;
  for (int op = 2; op < 4 && status == MCMG_OK; ++op) {
    const bool r = op == 2;
    const TransferParams p = transfer_params(L, r, r ? fine : coarse, r ? coarse : fine);
    float best_ms[kNumXShapes];
    for (int s = 0; s < kNumXShapes; ++s) best_ms[s] = 1e30f;
    for (int pass = 0; pass < kTunePasses && status == MCMG_OK; ++pass) {
      for (int s = 0; s < kNumXShapes; ++s) {
        if (!xshape_ok(s, L, r)) continue;
        // thread-per-node transfers time well alone but slowed the whole
        // V-cycle on grids with small coarse levels (measured on 256^2;
        // faster on 1024^2): candidates only from 2^16 coarse nodes on
        if (s < kNumTShapes && kTShapes[s].kq < 0 && L.g.coarse().nodes() < (1 << 16)) continue;
        for (int rep = 0; rep < 2; ++rep)
          if ((status = transfer_run(L, p, r, s, 1, st)) != MCMG_OK) break;
        if (status != MCMG_OK) break;
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < kTuneReps; ++rep)
          if ((status = transfer_run(L, p, r, s, 1, st)) != MCMG_OK) break;
        if (status != MCMG_OK) break;
        cudaEventRecord(e1, st);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) { status = cuda_fail(ce, "autotune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms[s]) best_ms[s] = ms;
      }
    }
    int best_s = 0;
    for (int s = 0; s < kNumXShapes; ++s)
      if (best_ms[s] < best_ms[best_s]) best_s = s;
    L.shape[op] = best_s;
    L.tuned[op] = best_s;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

int kernel_shape_count(int op) { return op < 2 ? kNumShapes : kNumXShapes; }
bool kernel_shape_valid(const Level& L, int op, int shape) {
  if (shape < 0 || shape >= kernel_shape_count(op)) return false;
  return op < 2 ? shape_ok(shape, L.C, L.g.d) : xshape_ok(shape, L, op == 2);
}

// ---------------------------------------------------------------------------
// Lift r_1[p][c] = g_lift[c] r[p];  project e[p] = sum_c g_proj[c] e_1[p][c].
// ---------------------------------------------------------------------------
__global__ void k_lift(const float2* __restrict__ r, const float2* __restrict__ lift,
                       float2* __restrict__ r1, int C, long long N) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= N * C) return;
  size_t off = (size_t)blockIdx.y * N;
  r1[off * C + id] = cmul_rn(lift[id % C], r[off + id / C]);
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

// Batched forms: field k of the batch reads srcs[k] / writes dsts[k].
__global__ void k_lift_gather(const float2* const* __restrict__ srcs, const float2* __restrict__ lift,
                              float2* __restrict__ r1, int C, long long N) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= N * C) return;
  const float2* r = srcs[blockIdx.y];
  r1[(size_t)blockIdx.y * N * C + id] = cmul_rn(lift[id % C], r[id / C]);
}

__global__ void k_project_scatter(const float2* __restrict__ e1, const float2* __restrict__ proj,
                                  float2* const* __restrict__ dsts, int C, long long N) {
  long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const float2* src = e1 + ((size_t)blockIdx.y * N + n) * C;
  float2 acc = make_float2(0.f, 0.f);
  for (int c = 0; c < C; ++c) cfma(acc, proj[c], src[c]);
  dsts[blockIdx.y][n] = acc;
}

mcmg_status launch_lift_gather(const float2* const* srcs, const float2* lift, float2* r1, int C,
                               long long nodes, int count, cudaStream_t st) {
  dim3 grid((unsigned)((nodes * C + 255) / 256), (unsigned)count);
  k_lift_gather<<<grid, 256, 0, st>>>(srcs, lift, r1, C, nodes);
  MCMG_CHECK_LAUNCH("lift_gather");
  return MCMG_OK;
}

mcmg_status launch_project_scatter(const float2* e1, const float2* proj, float2* const* dsts, int C,
                                   long long nodes, int count, cudaStream_t st) {
  dim3 grid((unsigned)((nodes + 255) / 256), (unsigned)count);
  k_project_scatter<<<grid, 256, 0, st>>>(e1, proj, dsts, C, nodes);
  MCMG_CHECK_LAUNCH("project_scatter");
  return MCMG_OK;
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
