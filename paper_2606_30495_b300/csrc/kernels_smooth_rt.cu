// Register-tiled, K-split FP32 smoothing step (Section 3.2) for coarse and
// mid levels: the kernel, its launch, and the dispatch over channel counts
// and thread shapes.
#include "vcycle_kernels.cuh"

namespace mcmg {

// Register-tiled, K-split smoothing step.  Thread (kg, ng, cg) of a
// 256-thread block holds the TN x CO output tile (block nodes ng*TN .. +TN-1,
// channels cg*CO .. +CO-1) and sums only the KQ input channels
// kg*KQ .. +KQ-1 of each mixing matrix; the KS partial tiles are added through
// shared memory.  A weight load (CO values) feeds TN nodes and a field value
// (a shared-memory broadcast) feeds CO channels, so few nodes per block still
// give every thread a dense contraction: the shape for coarse levels, where
// one block per handful of nodes is all the parallelism there is.
// The block first stages, per stencil tap, the neighbour values of its NB
// nodes ([tap][node][C], zero outside the grid: Dirichlet closure).  The
// thread's KQ x CO slice of the next mixing matrix is loaded into registers
// while the current one is applied (K_A, the 2D+1 taps, K_S, W^(i) in turn),
// so weight latency overlaps arithmetic across the phase barriers.  K_A
// partials go to their own buffer so a_l (.) is applied once, in the sum.
// Two blocks per SM (at most 128 registers a thread) while the accumulator
// tile and the two weight slices take at most 96 registers.
template <int TN, int CO, int KQ>
__host__ __device__ constexpr int rt_min_blocks() { return 2 * TN * CO + 4 * KQ * CO <= 96 ? 2 : 1; }

template <int C, int D, int MODE, int TN, int CO, int KQ>
__global__ void __launch_bounds__(256, rt_min_blocks<TN, CO, KQ>())
k_smooth_rt(SmoothParams p) {
  using T = RtTile<C, TN, CO, KQ>;
  constexpr int NB = T::NB, KS = T::KS, NT = 2 * D + 1, C2 = C / 2;
  extern __shared__ float4 sm4[];
  float2* E = reinterpret_cast<float2*>(sm4);   // [NT][NB][C]
  float2* red = E + NT * NB * C;                // [KS][NB][C]  taps / K_S / W^(i)
  float2* redA = red + KS * NB * C;             // [KS][NB][C]  K_A
  float2* Ts = E;                               // [NB][C], after the taps are used
  float2* Zs = E + NB * C;                      // [NB][C]
  const int tid = threadIdx.x;
  const int cg = tid % T::CG;
  const int ng = (tid / T::CG) % T::NG;
  const int kg = tid / (T::CG * T::NG);
  const int co0 = cg * CO, j0 = ng * TN, ci0 = kg * KQ;
  const long long N = p.nodes;
  const size_t off = (size_t)blockIdx.y * (size_t)N * C;
  const float2* __restrict__ r = p.r + off;
  const float2* __restrict__ ein = p.e_in ? p.e_in + off : nullptr;
  float2* __restrict__ eout = p.e_out + off;
  const long long n0 = (long long)blockIdx.x * NB;

  if (MODE == 1 && !ein) {  // residual of e = 0
    for (int idx = tid; idx < NB * C; idx += 256) {
      const long long n = n0 + idx / C;
      if (n < N) eout[n0 * C + idx] = r[n0 * C + idx];
    }
    return;
  }

  float2 w[2][KQ][CO];      // this thread's slice of the current and next matrix
  auto load_w = [&](const float2* __restrict__ Mt, float2 (&dst)[KQ][CO]) {
#pragma unroll
    for (int i = 0; i < KQ; ++i) ldc<CO>(Mt + (ci0 + i) * C + co0, dst[i]);
  };
  float2 acc[TN][CO];
  auto zero = [&]() {
#pragma unroll
    for (int k = 0; k < TN; ++k)
#pragma unroll
      for (int c = 0; c < CO; ++c) acc[k][c] = make_float2(0.f, 0.f);
  };
  // acc += (slice of M^T) applied to X[node][ci]
  auto contract = [&](const float2 (&wm)[KQ][CO], const float2* X) {
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        const float2 v = X[(j0 + k) * C + ci0 + i];
#pragma unroll
        for (int c = 0; c < CO; ++c) cfma(acc[k][c], wm[i][c], v);
      }
    }
  };
  auto store_partial = [&](float2* dst) {
#pragma unroll
    for (int k = 0; k < TN; ++k) stc<CO>(dst + (kg * NB + j0 + k) * C + co0, acc[k]);
  };
  auto reduced = [&](const float2* src, int idx) {
    float2 v = src[idx];
#pragma unroll
    for (int q = 1; q < KS; ++q) v = cadd(v, src[q * NB * C + idx]);
    return v;
  };

  if (ein) {
    load_w(p.KAt, w[0]);
    load_w(p.Wt, w[1]);
    const long long sxy = (long long)p.nx * p.ny;
    for (int idx = tid; idx < NT * NB * C2; idx += 256) {
      const int c2 = idx % C2;
      const int j = (idx / C2) % NB;
      const int tap = idx / (C2 * NB);
      const long long n = n0 + j;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n < N) {
        long long nb = n;
        bool ok = true;
        if (tap > 0) {
          int x, y, z;
          node_xyz(n, p.nx, p.ny, x, y, z);
          const int axis = (tap - 1) >> 1;
          const int sgn = (tap & 1) ? -1 : 1;
          const int c = axis == 0 ? x : (axis == 1 ? y : z);
          const int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
          const long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : sxy);
          ok = c + sgn >= 0 && c + sgn < ext;
          nb = n + sgn * stride;
        }
        if (ok) v = __ldg(reinterpret_cast<const float4*>(ein + nb * C) + c2);
      }
      sm4[(tap * NB + j) * C2 + c2] = v;
    }
    __syncthreads();

    // t = r - (W_l * e + a (.) (K_A e))
    zero();
    contract(w[0], E);
    store_partial(redA);
    zero();
#pragma unroll
    for (int tap = 0; tap < NT; ++tap) {
      // W_tap sits in w[(tap + 1) & 1]; the next matrix goes to the other buffer
      if (tap + 1 < NT)
        load_w(p.Wt + (size_t)(tap + 1) * C * C, w[tap & 1]);
      else if (MODE == 0)
        load_w(p.KSt, w[tap & 1]);
      contract(w[(tap + 1) & 1], E + tap * NB * C);
    }
    store_partial(red);
    __syncthreads();
    for (int idx = tid; idx < NB * C; idx += 256) {
      const long long n = n0 + idx / C;
      float2 t = make_float2(0.f, 0.f);
      if (n < N) {
        const float2 rv = __ldg(r + n0 * C + idx);
        const float2 av = __ldg(p.a + n0 * C + idx);
        t = csub(csub(rv, reduced(red, idx)), cmul(av, reduced(redA, idx)));
      }
      if (MODE == 1) {
        if (n < N) eout[n0 * C + idx] = t;
      } else {
        Ts[idx] = t;
      }
    }
    if (MODE == 1) return;
    __syncthreads();
  } else {
    load_w(p.KSt, w[0]);
    for (int idx = tid; idx < NB * C2; idx += 256) {
      const long long n = n0 + idx / C2;
      sm4[idx] = n < N ? __ldg(reinterpret_cast<const float4*>(r + n0 * C) + idx)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
  }
  // K_S is in w[0] on both paths ((2D+1) taps leave it in w[(NT-1) & 1] = w[0])
  static_assert(((NT - 1) & 1) == 0, "tap count is odd");

  // z = s (.) (K_S t)
  load_w(p.Wst, w[1]);
  zero();
  contract(w[0], Ts);
  store_partial(red);
  __syncthreads();
  for (int idx = tid; idx < NB * C; idx += 256) {
    const long long n = n0 + idx / C;
    Zs[idx] = n < N ? cmul(__ldg(p.s + n0 * C + idx), reduced(red, idx)) : make_float2(0.f, 0.f);
  }
  __syncthreads();

  // e' = e + W^(i) z
  zero();
  contract(w[1], Zs);
  store_partial(red);
  __syncthreads();
  for (int idx = tid; idx < NB * C; idx += 256) {
    const long long n = n0 + idx / C;
    if (n < N) {
      const float2 u = reduced(red, idx);
      eout[n0 * C + idx] = ein ? cadd(u, ein[n0 * C + idx]) : u;
    }
  }
}

template <int C, int D, int TN, int CO, int KQ>
static mcmg_status smooth_rt(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  using T = RtTile<C, TN, CO, KQ>;
  constexpr size_t smem =
      (size_t)(2 * D + 1 + 2 * (T::valid ? T::KS : 0)) * T::NB * C * sizeof(float2);
  if constexpr (!T::valid || C < 2 || smem > kMaxSmem) {
    set_error("register-tiled shape does not fit %d channels", C);
    return MCMG_ERR_SHAPE;
  } else {
    dim3 grid((unsigned)((p.nodes + T::NB - 1) / T::NB), (unsigned)nrhs);
    if (mode == 0) {
      auto k = k_smooth_rt<C, D, 0, TN, CO, KQ>;
      if (smem > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<grid, 256, smem, st>>>(p);
    } else {
      auto k = k_smooth_rt<C, D, 1, TN, CO, KQ>;
      if (smem > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k<<<grid, 256, smem, st>>>(p);
    }
    MCMG_CHECK_LAUNCH("smooth_rt");
    return MCMG_OK;
  }
}

template <int C, int D>
static mcmg_status smooth_rt_c(const SmoothParams& p, int mode, int tn, int co, int kq, int nrhs,
                               cudaStream_t st) {
  if (co == 4) {
    if (tn == 8 && kq == 4) return smooth_rt<C, D, 8, 4, 4>(p, mode, nrhs, st);
    if (tn == 4 && kq == 4) return smooth_rt<C, D, 4, 4, 4>(p, mode, nrhs, st);
    if (tn == 8 && kq == 2) return smooth_rt<C, D, 8, 4, 2>(p, mode, nrhs, st);
    if (tn == 4 && kq == 2) return smooth_rt<C, D, 4, 4, 2>(p, mode, nrhs, st);
    if (tn == 8 && kq == 8) return smooth_rt<C, D, 8, 4, 8>(p, mode, nrhs, st);
    if (tn == 4 && kq == 8) return smooth_rt<C, D, 4, 4, 8>(p, mode, nrhs, st);
  }
  set_error("register-tiled smoothing shape (%d, %d, %d) is not built", tn, co, kq);
  return MCMG_ERR_SHAPE;
}

template <int D>
static mcmg_status smooth_rt_d(const SmoothParams& p, int C, int mode, int tn, int co, int kq,
                               int nrhs, cudaStream_t st) {
  switch (C) {
    case 4: return smooth_rt_c<4, D>(p, mode, tn, co, kq, nrhs, st);
    case 8: return smooth_rt_c<8, D>(p, mode, tn, co, kq, nrhs, st);
    case 16: return smooth_rt_c<16, D>(p, mode, tn, co, kq, nrhs, st);
    case 32: return smooth_rt_c<32, D>(p, mode, tn, co, kq, nrhs, st);
    case 64: return smooth_rt_c<64, D>(p, mode, tn, co, kq, nrhs, st);
  }
  set_error("register-tiled smoothing needs 4 to 64 channels, got %d", C);
  return MCMG_ERR_SHAPE;
}

mcmg_status smooth_rt_launch(const SmoothParams& p, int C, int D, int mode, int tn, int co, int kq,
                             int nrhs, cudaStream_t st) {
  return D == 3 ? smooth_rt_d<3>(p, C, mode, tn, co, kq, nrhs, st)
                : smooth_rt_d<2>(p, C, mode, tn, co, kq, nrhs, st);
}

}  // namespace mcmg
