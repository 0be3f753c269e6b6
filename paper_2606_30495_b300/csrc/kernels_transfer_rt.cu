// Register-tiled restriction and prolongation (the inter-grid transfers of
// Section 3.2 / Algorithm 2): kernels, launch, dispatch over channel pairs.
#include "vcycle_kernels.cuh"

namespace mcmg {

// rc[J][co] = sum_o sum_ci R[o][co][ci] t[2J + o][ci]   (CI fine, CO coarse channels)
template <int CI, int CO, int D, int TN, int CV, int KQ>
__global__ void __launch_bounds__(256) k_restrict_rt(TransferParams p) {
  pdl_launch_dependents();
  pdl_wait();
  using T = XTile<CI, CO, TN, CV, KQ>;
  constexpr int NB = T::NB, KS = T::KS, T3 = D == 3 ? 27 : 9, CI2 = CI / 2;
  extern __shared__ float4 sm4[];
  float2* E = reinterpret_cast<float2*>(sm4);   // [T3][NB][CI]
  float2* red = E + T3 * NB * CI;               // [KS][NB][CO]
  const int tid = threadIdx.x;
  const int cg = tid % T::CG;
  const int ng = (tid / T::CG) % T::NG;
  const int kg = tid / (T::CG * T::NG);
  const int co0 = cg * CV, j0 = ng * TN, ci0 = kg * KQ;
  const long long NC = p.dst_nodes;
  const float2* __restrict__ t = p.src + (size_t)blockIdx.y * p.src_nodes * CI;
  float2* __restrict__ rc = p.dst + (size_t)blockIdx.y * NC * CO;
  const long long n0 = (long long)blockIdx.x * NB;
  for (int idx = tid; idx < T3 * NB * CI2; idx += 256) {
    const int c2 = idx % CI2;
    const int j = (idx / CI2) % NB;
    const int o = idx / (CI2 * NB);
    const long long n = n0 + j;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < NC) {
      int jx, jy, jz;
      node_xyz32((int)n, p.cx, p.cy, jx, jy, jz);
      const int x = 2 * jx + o % 3 - 1, y = 2 * jy + (o / 3) % 3 - 1;
      const int z = D == 3 ? 2 * jz + o / 9 - 1 : 0;
      if (x >= 0 && x < p.fx && y >= 0 && y < p.fy && z >= 0 && z < p.fz)
        v = __ldg(reinterpret_cast<const float4*>(t + (((long long)z * p.fy + y) * p.fx + x) * CI) + c2);
    }
    sm4[(o * NB + j) * CI2 + c2] = v;
  }
  __syncthreads();
  float2 acc[TN][CV];
#pragma unroll
  for (int k = 0; k < TN; ++k)
#pragma unroll
    for (int c = 0; c < CV; ++c) acc[k][c] = make_float2(0.f, 0.f);
#pragma unroll 3
  for (int o = 0; o < T3; ++o) {
    const float2* __restrict__ wt = p.Wt + (size_t)o * CI * CO;
    const float2* X = E + o * NB * CI;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
      float2 w[CV];
      ldc<CV>(wt + (ci0 + i) * CO + co0, w);
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        const float2 v = X[(j0 + k) * CI + ci0 + i];
#pragma unroll
        for (int c = 0; c < CV; ++c) cfma(acc[k][c], w[c], v);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < TN; ++k) stc<CV>(red + (kg * NB + j0 + k) * CO + co0, acc[k]);
  __syncthreads();
  for (int idx = tid; idx < NB * CO; idx += 256) {
    const long long n = n0 + idx / CO;
    if (n < NC) {
      float2 v = red[idx];
#pragma unroll
      for (int q = 1; q < KS; ++q) v = cadd(v, red[q * NB * CO + idx]);
      rc[n0 * CO + idx] = v;
    }
  }
}

// e[2J + b] += sum over taps o with b(o) = b of P[o] e_c[J + c(o)]
// (coarse-node form of the transposed convolution, as k_prolong_add; CI
// coarse, CO fine channels).  The block stages e_c at J + {0,1}^d.
template <int CI, int CO, int D, int TN, int CV, int KQ>
__global__ void __launch_bounds__(256) k_prolong_rt(TransferParams p) {
  pdl_launch_dependents();
  pdl_wait();
  using T = XTile<CI, CO, TN, CV, KQ>;
  constexpr int NB = T::NB, KS = T::KS, T3 = D == 3 ? 27 : 9, NP = D == 3 ? 8 : 4;
  constexpr int CI2 = CI / 2;
  extern __shared__ float4 sm4[];
  float2* E = reinterpret_cast<float2*>(sm4);   // [NP][NB][CI]
  float2* red = E + NP * NB * CI;               // [KS][NB][NP][CO]
  const int tid = threadIdx.x;
  const int cg = tid % T::CG;
  const int ng = (tid / T::CG) % T::NG;
  const int kg = tid / (T::CG * T::NG);
  const int co0 = cg * CV, j0 = ng * TN, ci0 = kg * KQ;
  const long long NC = p.src_nodes;
  const float2* __restrict__ ec = p.src + (size_t)blockIdx.y * NC * CI;
  float2* __restrict__ e = p.dst + (size_t)blockIdx.y * p.dst_nodes * CO;
  const long long n0 = (long long)blockIdx.x * NB;
  for (int idx = tid; idx < NP * NB * CI2; idx += 256) {
    const int c2 = idx % CI2;
    const int j = (idx / CI2) % NB;
    const int c = idx / (CI2 * NB);
    const long long n = n0 + j;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (n < NC) {
      int jx, jy, jz;
      node_xyz32((int)n, p.cx, p.cy, jx, jy, jz);
      const int X = jx + (c & 1), Y = jy + ((c >> 1) & 1), Z = jz + ((c >> 2) & 1);
      if (X < p.cx && Y < p.cy && (D == 3 ? Z < p.cz : true))
        v = __ldg(reinterpret_cast<const float4*>(ec + (((long long)(D == 3 ? Z : 0) * p.cy + Y) * p.cx + X) * CI) + c2);
    }
    sm4[(c * NB + j) * CI2 + c2] = v;
  }
  __syncthreads();
  float2 acc[NP][TN][CV];
#pragma unroll
  for (int b = 0; b < NP; ++b)
#pragma unroll
    for (int k = 0; k < TN; ++k)
#pragma unroll
      for (int c = 0; c < CV; ++c) acc[b][k][c] = make_float2(0.f, 0.f);
#pragma unroll
  for (int o = 0; o < T3; ++o) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = D == 3 ? o / 9 - 1 : 0;
    const int b = (ox != 0) | ((oy != 0) << 1) | ((oz != 0) << 2);
    const int c = (ox == -1) | ((oy == -1) << 1) | ((oz == -1) << 2);
    const float2* __restrict__ wt = p.Wt + (size_t)o * CI * CO;
    const float2* X = E + c * NB * CI;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
      float2 w[CV];
      ldc<CV>(wt + (ci0 + i) * CO + co0, w);
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        const float2 v = X[(j0 + k) * CI + ci0 + i];
#pragma unroll
        for (int cc = 0; cc < CV; ++cc) cfma(acc[b][k][cc], w[cc], v);
      }
    }
  }
#pragma unroll
  for (int b = 0; b < NP; ++b)
#pragma unroll
    for (int k = 0; k < TN; ++k) stc<CV>(red + ((kg * NB + j0 + k) * NP + b) * CO + co0, acc[b][k]);
  __syncthreads();
  for (int idx = tid; idx < NB * NP * CO; idx += 256) {
    const int co = idx % CO;
    const int b = (idx / CO) % NP;
    const long long n = n0 + idx / (CO * NP);
    if (n < NC) {
      float2 v = red[idx];
#pragma unroll
      for (int q = 1; q < KS; ++q) v = cadd(v, red[q * NB * NP * CO + idx]);
      int jx, jy, jz;
      node_xyz32((int)n, p.cx, p.cy, jx, jy, jz);
      const long long fx = 2 * jx + (b & 1), fy = 2 * jy + ((b >> 1) & 1),
                      fz = D == 3 ? 2 * jz + ((b >> 2) & 1) : 0;
      const long long fi = ((fz * p.fy + fy) * p.fx + fx) * CO + co;
      e[fi] = cadd(e[fi], v);
    }
  }
}

template <int CI, int CO, int D, int TN, int CV, int KQ>
static mcmg_status transfer_rt(const TransferParams& p, bool restrict_, int nrhs, cudaStream_t st) {
  using T = XTile<CI, CO, TN, CV, KQ>;
  constexpr int T3 = D == 3 ? 27 : 9, NP = D == 3 ? 8 : 4;
  constexpr size_t smem_r = (size_t)(T3 * T::NB * CI + T::KS * T::NB * CO) * sizeof(float2);
  constexpr size_t smem_p = (size_t)(NP * T::NB * CI + T::KS * T::NB * NP * CO) * sizeof(float2);
  if constexpr (!T::valid) {
    set_error("register-tiled transfer shape does not fit %d -> %d channels", CI, CO);
    return MCMG_ERR_SHAPE;
  } else {
    if ((restrict_ ? smem_r : smem_p) > kMaxSmem) {
      set_error("register-tiled transfer shape needs too much shared memory");
      return MCMG_ERR_SHAPE;
    }
    const long long units = restrict_ ? p.dst_nodes : p.src_nodes;
    dim3 grid((unsigned)((units + T::NB - 1) / T::NB), (unsigned)nrhs);
    if (restrict_) {
      auto k = k_restrict_rt<CI, CO, D, TN, CV, KQ>;
      if (smem_r > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem_r, st, p);
    } else {
      auto k = k_prolong_rt<CI, CO, D, TN, CV, KQ>;
      if (smem_p > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem_p, st, p);
    }
    MCMG_CHECK_LAUNCH(restrict_ ? "restrict_rt" : "prolong_rt");
    return MCMG_OK;
  }
}

// Thread per coarse node (few channels).  G = CO / CT adjacent lanes share a
// coarse node J, each owning CT output channels; the transfer weights sit in
// shared memory ([tap][CI][CO], read as broadcasts: every node's lanes read
// the same weights) and each lane reads a source node's CI values with
// 16-byte loads.  No block barrier after the weights are staged.
template <int CI, int CO, int D, int CT, bool RESTRICT>
constexpr bool tpnx_valid() {
  constexpr int G = CT > 0 && CO % CT == 0 ? CO / CT : 0;
  return G >= 1 && 32 % G == 0 && CI <= 32 && CI % 2 == 0 && CT % 2 == 0 &&
         (RESTRICT || (D == 3 ? 8 : 4) * CT <= 32);
}

// rc[J][co] = sum_o sum_ci R[o][co][ci] t[2J + o][ci]   (CI fine, CO coarse)
template <int CI, int CO, int D, int CT>
__global__ void __launch_bounds__(256) k_restrict_tpn(TransferParams p) {
  pdl_launch_dependents();
  constexpr int G = CO / CT, NPB = 256 / G, T3 = D == 3 ? 27 : 9, MSZ = CI * CO;
  extern __shared__ float4 xw4[];
  const float2* Wsm = reinterpret_cast<const float2*>(xw4);   // [T3][CI][CO]
  for (int i = threadIdx.x; i < T3 * MSZ / 2; i += 256)
    xw4[i] = __ldg(reinterpret_cast<const float4*>(p.Wt) + i);
  __syncthreads();
  pdl_wait();
  const int c0 = (threadIdx.x % G) * CT;
  const long long NC = p.dst_nodes;
  const long long J = (long long)blockIdx.x * NPB + threadIdx.x / G;
  if (J >= NC) return;
  const float2* __restrict__ t = p.src + (size_t)blockIdx.y * p.src_nodes * CI;
  float2* __restrict__ rc = p.dst + (size_t)blockIdx.y * NC * CO;
  int jx, jy, jz;
  node_xyz32((int)J, p.cx, p.cy, jx, jy, jz);
  float2 acc[CT];
#pragma unroll
  for (int c = 0; c < CT; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll 3
  for (int o = 0; o < T3; ++o) {
    const int x = 2 * jx + o % 3 - 1, y = 2 * jy + (o / 3) % 3 - 1;
    const int z = D == 3 ? 2 * jz + o / 9 - 1 : 0;
    if (x < 0 || x >= p.fx || y < 0 || y >= p.fy || z < 0 || z >= p.fz) continue;
    const float4* src4 =
        reinterpret_cast<const float4*>(t + (((long long)z * p.fy + y) * p.fx + x) * CI);
    float2 xv[CI];
#pragma unroll
    for (int h = 0; h < CI / 2; ++h) {
      const float4 v = __ldg(src4 + h);
      xv[2 * h] = make_float2(v.x, v.y);
      xv[2 * h + 1] = make_float2(v.z, v.w);
    }
    const float2* Mt = Wsm + o * MSZ;
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) {
      const float4* w4 = reinterpret_cast<const float4*>(Mt + ci * CO + c0);
#pragma unroll
      for (int h = 0; h < CT / 2; ++h) {
        const float4 w = w4[h];
        cfma(acc[2 * h], make_float2(w.x, w.y), xv[ci]);
        cfma(acc[2 * h + 1], make_float2(w.z, w.w), xv[ci]);
      }
    }
  }
  float4* o4 = reinterpret_cast<float4*>(rc + J * CO + c0);
#pragma unroll
  for (int h = 0; h < CT / 2; ++h)
    o4[h] = make_float4(acc[2 * h].x, acc[2 * h].y, acc[2 * h + 1].x, acc[2 * h + 1].y);
}

// e[2J + b] += sum over taps o with b(o) = b of P[o] e_c[J + c(o)] (coarse-node
// form, as k_prolong_rt; CI coarse, CO fine channels): a lane accumulates its
// CT channels of all 2^d fine nodes of J, reading each of the 2^d coarse
// neighbours once.
template <int CI, int CO, int D, int CT>
__global__ void __launch_bounds__(256) k_prolong_tpn(TransferParams p) {
  pdl_launch_dependents();
  constexpr int G = CO / CT, NPB = 256 / G, T3 = D == 3 ? 27 : 9, NP = D == 3 ? 8 : 4;
  constexpr int MSZ = CI * CO;
  extern __shared__ float4 xw4[];
  const float2* Wsm = reinterpret_cast<const float2*>(xw4);   // [T3][CI][CO]
  for (int i = threadIdx.x; i < T3 * MSZ / 2; i += 256)
    xw4[i] = __ldg(reinterpret_cast<const float4*>(p.Wt) + i);
  __syncthreads();
  pdl_wait();
  const int c0 = (threadIdx.x % G) * CT;
  const long long NC = p.src_nodes;
  const long long J = (long long)blockIdx.x * NPB + threadIdx.x / G;
  if (J >= NC) return;
  const float2* __restrict__ ec = p.src + (size_t)blockIdx.y * NC * CI;
  float2* __restrict__ e = p.dst + (size_t)blockIdx.y * p.dst_nodes * CO;
  int jx, jy, jz;
  node_xyz32((int)J, p.cx, p.cy, jx, jy, jz);
  float2 acc[NP][CT];
#pragma unroll
  for (int b = 0; b < NP; ++b)
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[b][c] = make_float2(0.f, 0.f);
#pragma unroll
  for (int cs = 0; cs < NP; ++cs) {          // coarse neighbour J + {0,1}^d
    const int X = jx + (cs & 1), Y = jy + ((cs >> 1) & 1), Z = jz + ((cs >> 2) & 1);
    if (X >= p.cx || Y >= p.cy || (D == 3 && Z >= p.cz)) continue;
    const float4* src4 = reinterpret_cast<const float4*>(
        ec + (((long long)(D == 3 ? Z : 0) * p.cy + Y) * p.cx + X) * CI);
    float2 xv[CI];
#pragma unroll
    for (int h = 0; h < CI / 2; ++h) {
      const float4 v = __ldg(src4 + h);
      xv[2 * h] = make_float2(v.x, v.y);
      xv[2 * h + 1] = make_float2(v.z, v.w);
    }
#pragma unroll
    for (int o = 0; o < T3; ++o) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = D == 3 ? o / 9 - 1 : 0;
      const int c = (ox == -1) | ((oy == -1) << 1) | ((oz == -1) << 2);
      if (c != cs) continue;                  // taps reading this neighbour
      const int b = (ox != 0) | ((oy != 0) << 1) | ((oz != 0) << 2);
      const float2* Mt = Wsm + o * MSZ;
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) {
        const float4* w4 = reinterpret_cast<const float4*>(Mt + ci * CO + c0);
#pragma unroll
        for (int h = 0; h < CT / 2; ++h) {
          const float4 w = w4[h];
          cfma(acc[b][2 * h], make_float2(w.x, w.y), xv[ci]);
          cfma(acc[b][2 * h + 1], make_float2(w.z, w.w), xv[ci]);
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < NP; ++b) {
    const long long fx = 2 * jx + (b & 1), fy = 2 * jy + ((b >> 1) & 1),
                    fz = D == 3 ? 2 * jz + ((b >> 2) & 1) : 0;
    float4* o4 = reinterpret_cast<float4*>(e + ((fz * p.fy + fy) * p.fx + fx) * CO + c0);
#pragma unroll
    for (int h = 0; h < CT / 2; ++h) {
      const float4 v = o4[h];
      o4[h] = make_float4(v.x + acc[b][2 * h].x, v.y + acc[b][2 * h].y,
                          v.z + acc[b][2 * h + 1].x, v.w + acc[b][2 * h + 1].y);
    }
  }
}

template <int CI, int CO, int D, int CT>
static mcmg_status transfer_tpn(const TransferParams& p, bool restrict_, int nrhs,
                                cudaStream_t st) {
  constexpr bool okr = tpnx_valid<CI, CO, D, CT, true>();
  constexpr bool okp = tpnx_valid<CI, CO, D, CT, false>();
  constexpr size_t smem = (size_t)(D == 3 ? 27 : 9) * CI * CO * sizeof(float2);
  if (smem > kMaxSmem || (restrict_ ? !okr : !okp)) {
    set_error("thread-per-node transfer shape does not fit %d -> %d channels", CI, CO);
    return MCMG_ERR_SHAPE;
  }
  constexpr int NPB = CT > 0 && CO % CT == 0 ? 256 / (CO / CT) : 1;
  const long long units = restrict_ ? p.dst_nodes : p.src_nodes;
  dim3 grid((unsigned)((units + NPB - 1) / NPB), (unsigned)nrhs);
  if constexpr (okr && smem <= kMaxSmem) {
    if (restrict_) {
      auto k = k_restrict_tpn<CI, CO, D, CT>;
      if (smem > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem, st, p);
    }
  }
  if constexpr (okp && smem <= kMaxSmem) {
    if (!restrict_) {
      auto k = k_prolong_tpn<CI, CO, D, CT>;
      if (smem > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem, st, p);
    }
  }
  MCMG_CHECK_LAUNCH(restrict_ ? "restrict_tpn" : "prolong_tpn");
  return MCMG_OK;
}

template <int CI, int CO, int D>
static mcmg_status transfer_rt_shape(const TransferParams& p, bool r, int tn, int cv, int kq,
                                     int nrhs, cudaStream_t st) {
  if (kq < 0) {   // thread per coarse node, cv output channels per lane
    if (cv == 2) return transfer_tpn<CI, CO, D, 2>(p, r, nrhs, st);
    if (cv == 4) return transfer_tpn<CI, CO, D, 4>(p, r, nrhs, st);
    if (cv == 8) return transfer_tpn<CI, CO, D, 8>(p, r, nrhs, st);
  }
  if (cv == 4) {
    if (tn == 1 && kq == 4) return transfer_rt<CI, CO, D, 1, 4, 4>(p, r, nrhs, st);
    if (tn == 2 && kq == 4) return transfer_rt<CI, CO, D, 2, 4, 4>(p, r, nrhs, st);
    if (tn == 1 && kq == 8) return transfer_rt<CI, CO, D, 1, 4, 8>(p, r, nrhs, st);
    if (tn == 2 && kq == 8) return transfer_rt<CI, CO, D, 2, 4, 8>(p, r, nrhs, st);
    if (tn == 1 && kq == 2) return transfer_rt<CI, CO, D, 1, 4, 2>(p, r, nrhs, st);
  }
  set_error("register-tiled transfer shape (%d, %d, %d) is not built", tn, cv, kq);
  return MCMG_ERR_SHAPE;
}

template <int D>
static mcmg_status transfer_rt_d(const TransferParams& p, int Cf, int Cc, bool r, int tn, int cv,
                                 int kq, int nrhs, cudaStream_t st) {
#define MCMG_XT_PAIR(F, Cq)                                                                 \
  if (Cf == F && Cc == Cq)                                                                  \
    return r ? transfer_rt_shape<F, Cq, D>(p, true, tn, cv, kq, nrhs, st)                        \
             : transfer_rt_shape<Cq, F, D>(p, false, tn, cv, kq, nrhs, st);
  MCMG_XT_PAIR(4, 4) MCMG_XT_PAIR(4, 8) MCMG_XT_PAIR(8, 8) MCMG_XT_PAIR(8, 16)
  MCMG_XT_PAIR(16, 16) MCMG_XT_PAIR(16, 32) MCMG_XT_PAIR(32, 32) MCMG_XT_PAIR(32, 64)
  MCMG_XT_PAIR(64, 64)
#undef MCMG_XT_PAIR
  set_error("no register-tiled transfer for %d -> %d channels", Cf, Cc);
  return MCMG_ERR_SHAPE;
}

mcmg_status transfer_rt_launch(const TransferParams& p, int Cf, int Cc, int D, bool restrict_,
                               int tn, int cv, int kq, int nrhs, cudaStream_t st) {
  return D == 3 ? transfer_rt_d<3>(p, Cf, Cc, restrict_, tn, cv, kq, nrhs, st)
                : transfer_rt_d<2>(p, Cf, Cc, restrict_, tn, cv, kq, nrhs, st);
}

}  // namespace mcmg
