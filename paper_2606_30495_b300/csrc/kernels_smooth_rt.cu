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
// nodes ([tap][node][C], zero outside the grid: Dirichlet closure).  K_A
// partials go to their own buffer so a_l (.) is applied once, in the sum.
// Two blocks per SM (at most 128 registers a thread) while the accumulator
// tile and one weight slice take at most 96 registers.
template <int TN, int CO, int KQ>
__host__ __device__ constexpr int rt_min_blocks() { return 2 * TN * CO + 2 * KQ * CO <= 96 ? 2 : 1; }

template <int C, int D, int MODE, int TN, int CO, int KQ>
__global__ void __launch_bounds__(256, rt_min_blocks<TN, CO, KQ>())
k_smooth_rt(SmoothParams p) {
  pdl_launch_dependents();
  using T = RtTile<C, TN, CO, KQ>;
  // node rows of the staged fields are C + 1 apart, so a warp's node groups
  // fall on different banks
  constexpr int NB = T::NB, KS = T::KS, NT = 2 * D + 1, C2 = C / 2, CP = C + 1;
  constexpr int ESZ = (NT * NB * CP + 1) & ~1;
  extern __shared__ float4 sm4[];
  float2* E = reinterpret_cast<float2*>(sm4);   // [NT][NB][CP]
  float2* red = E + ESZ;                        // [KS][NB][C]  taps / K_S / W^(i)
  float2* redA = red + KS * NB * C;             // [KS][NB][C]  K_A
  float2* Ts = E;                               // [NB][CP], after the taps are used
  float2* Zs = E + NB * CP;                     // [NB][CP]
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
  // this thread's outputs in the sums below are idx = tid + 256 q (node
  // n0 + idx / C, channel idx % C); their r, a, s and e values are loaded
  // now so that no dependent global load sits between the phases
  // (when there are at most two per thread; otherwise they are loaded where used)
  constexpr int RQ = (NB * C + 255) / 256;
  constexpr bool PF = RQ <= 2;
  constexpr int RP = PF ? RQ : 1;
  float2 rq[RP], aq[RP], sq[RP], eq[RP];
  if constexpr (PF) {   // features: setup-time data, read before the wait
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      const int idx = tid + 256 * q;
      const bool in = idx < NB * C && n0 + idx / C < N;
      const size_t g = in ? (size_t)(n0 * C + idx) : 0;
      aq[q] = in && ein ? __ldg(p.a + g) : make_float2(0.f, 0.f);
      sq[q] = in && MODE == 0 ? __ldg(p.s + g) : make_float2(0.f, 0.f);
    }
  }
  pdl_wait();
  if constexpr (PF) {
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      const int idx = tid + 256 * q;
      const bool in = idx < NB * C && n0 + idx / C < N;
      const size_t g = in ? (size_t)(n0 * C + idx) : 0;
      rq[q] = in ? __ldg(r + g) : make_float2(0.f, 0.f);
      eq[q] = in && ein && MODE == 0 ? __ldg(ein + g) : make_float2(0.f, 0.f);
    }
  }
  // value of output q (idx = tid + 256 q, a node inside the grid)
  auto pre = [&](const float2 (&arr)[RP], const float2* src, int q) -> float2 {
    if constexpr (PF) return arr[q];
    else return __ldg(src + n0 * C + tid + 256 * q);
  };

  if (MODE == 1 && !ein) {  // residual of e = 0
    for (int idx = tid; idx < NB * C; idx += 256) {
      const long long n = n0 + idx / C;
      if (n < N) eout[n0 * C + idx] = r[n0 * C + idx];
    }
    return;
  }

  float2 acc[TN][CO];
  auto zero = [&]() {
#pragma unroll
    for (int k = 0; k < TN; ++k)
#pragma unroll
      for (int c = 0; c < CO; ++c) acc[k][c] = make_float2(0.f, 0.f);
  };
  // acc += (this thread's slice of M^T) applied to X[node][ci]
  auto contract = [&](const float2* __restrict__ Mt, const float2* X) {
    float2 w[KQ][CO];
#pragma unroll
    for (int i = 0; i < KQ; ++i) ldc<CO>(Mt + (ci0 + i) * C + co0, w[i]);
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        const float2 v = X[(j0 + k) * CP + ci0 + i];
#pragma unroll
        for (int c = 0; c < CO; ++c) cfma(acc[k][c], w[i][c], v);
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
          // grids hold fewer than 2^31 nodes (checked at setup): 32-bit index math
          const int ni = (int)n, rest = ni / p.nx;
          const int axis = (tap - 1) >> 1;
          const int sgn = (tap & 1) ? -1 : 1;
          const int c = axis == 0 ? ni - rest * p.nx : (axis == 1 ? rest % p.ny : rest / p.ny);
          const int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
          const long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : sxy);
          ok = c + sgn >= 0 && c + sgn < ext;
          nb = n + sgn * stride;
        }
        if (ok) v = __ldg(reinterpret_cast<const float4*>(ein + nb * C) + c2);
      }
      E[(tap * NB + j) * CP + 2 * c2] = make_float2(v.x, v.y);
      E[(tap * NB + j) * CP + 2 * c2 + 1] = make_float2(v.z, v.w);
    }
  } else {
    for (int idx = tid; idx < NB * C2; idx += 256) {
      const long long n = n0 + idx / C2;
      const float4 v = n < N ? __ldg(reinterpret_cast<const float4*>(r + n0 * C) + idx)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
      Ts[(idx / C2) * CP + 2 * (idx % C2)] = make_float2(v.x, v.y);
      Ts[(idx / C2) * CP + 2 * (idx % C2) + 1] = make_float2(v.z, v.w);
    }
  }
  __syncthreads();

  // One contraction per round, the code emitted once (a fully unrolled round
  // sequence overflows the instruction cache): with e, K_A on the centre
  // values, then W_tap on each tap's values (t = r - W_l * e - a (.) K_A e);
  // then K_S on t (z = s (.) K_S t) and W^(i) on z (e' = e + W^(i) z).
  const int nA = ein ? NT + 1 : 0;
  const int nm = nA + (MODE == 0 ? 2 : 0);
  zero();
#pragma unroll 1
  for (int m = 0; m < nm; ++m) {
    const float2* Mt;
    const float2* X;
    if (m < nA) {
      Mt = m == 0 ? p.KAt : p.Wt + (size_t)(m - 1) * C * C;
      X = E + (m == 0 ? 0 : m - 1) * NB * CP;
    } else {
      Mt = m == nA ? p.KSt : p.Wst;
      X = m == nA ? Ts : Zs;
    }
    contract(Mt, X);
    if (m == 0 && nA > 0) {            // K_A partials apart
      store_partial(redA);
      zero();
    } else if (m == nA - 1) {          // t = r - sum - a (.) sum_A
      store_partial(red);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const int idx = tid + 256 * q;
        if (idx < NB * C) {
          const long long n = n0 + idx / C;
          float2 t = make_float2(0.f, 0.f);
          if (n < N)
            t = csub(csub(pre(rq, r, q), reduced(red, idx)), cmul(pre(aq, p.a, q), reduced(redA, idx)));
          if (MODE == 1) {
            if (n < N) eout[n0 * C + idx] = t;
          } else {
            Ts[(idx / C) * CP + idx % C] = t;
          }
        }
      }
      if (MODE == 1) return;
      __syncthreads();
      zero();
    } else if (m == nA) {              // z = s (.) (K_S t)
      store_partial(red);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const int idx = tid + 256 * q;
        if (idx < NB * C)
          Zs[(idx / C) * CP + idx % C] =
              n0 + idx / C < N ? cmul(pre(sq, p.s, q), reduced(red, idx)) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      zero();
    } else if (m == nA + 1) {          // e' = e + W^(i) z
      store_partial(red);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < RQ; ++q) {
        const int idx = tid + 256 * q;
        if (idx < NB * C && n0 + idx / C < N) {
          const float2 u = reduced(red, idx);
          eout[n0 * C + idx] = ein ? cadd(u, pre(eq, ein, q)) : u;
        }
      }
    }
  }
}

template <int C, int D, int TN, int CO, int KQ>
static mcmg_status smooth_rt(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  using T = RtTile<C, TN, CO, KQ>;
  constexpr size_t smem = (size_t)((((2 * D + 1) * T::NB * (C + 1) + 1) & ~1) +
                                   2 * (T::valid ? T::KS : 0) * T::NB * C) * sizeof(float2);
  if constexpr (!T::valid || C < 2 || smem > kMaxSmem) {
    set_error("register-tiled shape does not fit %d channels", C);
    return MCMG_ERR_SHAPE;
  } else {
    dim3 grid((unsigned)((p.nodes + T::NB - 1) / T::NB), (unsigned)nrhs);
    if (mode == 0) {
      auto k = k_smooth_rt<C, D, 0, TN, CO, KQ>;
      if (smem > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem, st, p);
    } else {
      auto k = k_smooth_rt<C, D, 1, TN, CO, KQ>;
      if (smem > 48 * 1024) MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem, st, p);
    }
    MCMG_CHECK_LAUNCH("smooth_rt");
    return MCMG_OK;
  }
}

// ---------------------------------------------------------------------------
// Bulk-copy variant.  The same tiles and phases as k_smooth_rt, but each
// mixing matrix (C x C complex, C^2 * 8 bytes) is brought into shared memory
// by one bulk asynchronous copy (cp.async.bulk, completion counted on an
// mbarrier), double-buffered: while the block applies matrix i, the copy of
// matrix i + 1 is in flight.  The weight stream then costs no load
// instructions or registers, and its latency hides behind the arithmetic.
// Every wait on a copy is bounded (about a second); on timeout the block
// records code 2 in the error word, waits (bounded) for its copies still in
// flight and returns.
// ---------------------------------------------------------------------------
namespace bulk {

constexpr unsigned SPIN_LIMIT = 1u << 20;   // try_waits of at most ~1 us each

__device__ __forceinline__ uint32_t smem_u32(const void* q) {
  return (uint32_t)__cvta_generic_to_shared(q);
}

__device__ __forceinline__ void bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
}

// One bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing a transaction on `bar`.
__device__ __forceinline__ void copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for the phase of `bar` with parity `parity`.
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity, const int* err) {
  const uint32_t a = smem_u32(bar);
  for (unsigned it = 0; it < SPIN_LIMIT; ++it) {
    if ((it & 255) == 255 && err && *(const volatile int*)err) return false;
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
  }
  return false;
}

}  // namespace bulk

template <int C, int D, int MODE, int TN, int CO, int KQ>
__global__ void __launch_bounds__(256, rt_min_blocks<TN, CO, KQ>())
k_smooth_rtb(SmoothParams p) {
  pdl_launch_dependents();
  using T = RtTile<C, TN, CO, KQ>;
  constexpr int NB = T::NB, KS = T::KS, NT = 2 * D + 1, C2 = C / 2, MSZ = C * C, CP = C + 1;
  constexpr int ESZ = (NT * NB * CP + 1) & ~1;   // node rows C + 1 apart (banks)
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ int s_fail;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);            // [2]
  float2* Wb = reinterpret_cast<float2*>(smraw + 128);           // [2][C][C]
  float2* E = Wb + 2 * MSZ;                                      // [NT][NB][CP]
  float2* red = E + ESZ;                                         // [KS][NB][C]
  float2* redA = red + KS * NB * C;                              // [KS][NB][C]
  float2* Ts = E;
  float2* Zs = E + NB * CP;
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
  // this thread's outputs in the sums below are idx = tid + 256 q (node
  // n0 + idx / C, channel idx % C); their r, a, s and e values are loaded
  // now so that no dependent global load sits between the phases
  // (when there are at most two per thread; otherwise they are loaded where used)
  constexpr int RQ = (NB * C + 255) / 256;
  constexpr bool PF = RQ <= 2;
  constexpr int RP = PF ? RQ : 1;
  float2 rq[RP], aq[RP], sq[RP], eq[RP];
  if constexpr (PF) {   // features: setup-time data, read before the wait
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      const int idx = tid + 256 * q;
      const bool in = idx < NB * C && n0 + idx / C < N;
      const size_t g = in ? (size_t)(n0 * C + idx) : 0;
      aq[q] = in && ein ? __ldg(p.a + g) : make_float2(0.f, 0.f);
      sq[q] = in && MODE == 0 ? __ldg(p.s + g) : make_float2(0.f, 0.f);
    }
  }
  // value of output q (idx = tid + 256 q, a node inside the grid)
  auto pre = [&](const float2 (&arr)[RP], const float2* src, int q) -> float2 {
    if constexpr (PF) return arr[q];
    else return __ldg(src + n0 * C + tid + 256 * q);
  };

  if (MODE == 1 && !ein) {  // residual of e = 0
    pdl_wait();
    for (int idx = tid; idx < NB * C; idx += 256) {
      const long long n = n0 + idx / C;
      if (n < N) eout[n0 * C + idx] = r[n0 * C + idx];
    }
    return;
  }

  // the matrices of this step in order: [K_A, W_0 .. W_2D] (with e), then
  // [K_S, W^(i)] (smoothing)
  const int nA = ein ? NT + 1 : 0;
  const int nm = nA + (MODE == 0 ? 2 : 0);
  auto mat = [&](int i) -> const float2* {
    if (i < nA) return i == 0 ? p.KAt : p.Wt + (size_t)(i - 1) * MSZ;
    return i == nA ? p.KSt : p.Wst;
  };
  int issued = 0;   // thread 0 only
  if (tid == 0) {
    s_fail = 0;
    bulk::bar_init(&bar[0]);
    bulk::bar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    for (; issued < 2 && issued < nm; ++issued)
      bulk::copy(Wb + (issued & 1) * MSZ, mat(issued), MSZ * sizeof(float2), &bar[issued & 1]);
  }
  pdl_wait();   // fields written by earlier kernels from here on
  if constexpr (PF) {
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      const int idx = tid + 256 * q;
      const bool in = idx < NB * C && n0 + idx / C < N;
      const size_t g = in ? (size_t)(n0 * C + idx) : 0;
      rq[q] = in ? __ldg(r + g) : make_float2(0.f, 0.f);
      eq[q] = in && ein && MODE == 0 ? __ldg(ein + g) : make_float2(0.f, 0.f);
    }
  }

  // Matrix i ready in Wb[i & 1] and visible to every thread; every thread has
  // finished with matrix i - 1, so its buffer takes matrix i + 1.
  auto acquire = [&](int i) -> bool {
    if (tid == 0 && !bulk::wait(&bar[i & 1], (i >> 1) & 1, p.err)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      if (tid == 0) {
        if (p.err) atomicOr(p.err, 2);
        for (int q = i; q < issued; ++q) bulk::wait(&bar[q & 1], (q >> 1) & 1, nullptr);
      }
      return false;
    }
    if (tid == 0 && i >= 1 && issued < nm) {
      bulk::copy(Wb + (issued & 1) * MSZ, mat(issued), MSZ * sizeof(float2), &bar[issued & 1]);
      ++issued;
    }
    return true;
  };

  float2 acc[TN][CO];
  auto zero = [&]() {
#pragma unroll
    for (int k = 0; k < TN; ++k)
#pragma unroll
      for (int c = 0; c < CO; ++c) acc[k][c] = make_float2(0.f, 0.f);
  };
  // acc += (slice of the matrix in Wb[b]) applied to X[node][ci]
  auto contract = [&](int b, const float2* X) {
    const float2* Mt = Wb + b * MSZ;
#pragma unroll
    for (int i = 0; i < KQ; ++i) {
      float2 w[CO];
      const float4* q4 = reinterpret_cast<const float4*>(Mt + (ci0 + i) * C + co0);
#pragma unroll
      for (int c = 0; c < CO / 2; ++c) {
        const float4 v4 = q4[c];
        w[2 * c] = make_float2(v4.x, v4.y);
        w[2 * c + 1] = make_float2(v4.z, v4.w);
      }
#pragma unroll
      for (int k = 0; k < TN; ++k) {
        const float2 v = X[(j0 + k) * CP + ci0 + i];
#pragma unroll
        for (int c = 0; c < CO; ++c) cfma(acc[k][c], w[c], v);
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

  int mi = 0;
  if (ein) {
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
          // grids hold fewer than 2^31 nodes (checked at setup): 32-bit index math
          const int ni = (int)n, rest = ni / p.nx;
          const int axis = (tap - 1) >> 1;
          const int sgn = (tap & 1) ? -1 : 1;
          const int c = axis == 0 ? ni - rest * p.nx : (axis == 1 ? rest % p.ny : rest / p.ny);
          const int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
          const long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : sxy);
          ok = c + sgn >= 0 && c + sgn < ext;
          nb = n + sgn * stride;
        }
        if (ok) v = __ldg(reinterpret_cast<const float4*>(ein + nb * C) + c2);
      }
      E[(tap * NB + j) * CP + 2 * c2] = make_float2(v.x, v.y);
      E[(tap * NB + j) * CP + 2 * c2 + 1] = make_float2(v.z, v.w);
    }
    // t = r - (W_l * e + a (.) (K_A e))
    if (!acquire(mi)) return;
    zero();
    contract(mi & 1, E);
    store_partial(redA);
    ++mi;
    zero();
#pragma unroll 1
    for (int tap = 0; tap < NT; ++tap, ++mi) {
      if (!acquire(mi)) return;
      contract(mi & 1, E + tap * NB * CP);
    }
    store_partial(red);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      const int idx = tid + 256 * q;
      if (idx < NB * C) {
        const long long n = n0 + idx / C;
        float2 t = make_float2(0.f, 0.f);
        if (n < N) t = csub(csub(pre(rq, r, q), reduced(red, idx)), cmul(pre(aq, p.a, q), reduced(redA, idx)));
        if (MODE == 1) {
          if (n < N) eout[n0 * C + idx] = t;
        } else {
          Ts[(idx / C) * CP + idx % C] = t;
        }
      }
    }
    if (MODE == 1) return;
  } else {
    for (int idx = tid; idx < NB * C2; idx += 256) {
      const long long n = n0 + idx / C2;
      const float4 v = n < N ? __ldg(reinterpret_cast<const float4*>(r + n0 * C) + idx)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
      Ts[(idx / C2) * CP + 2 * (idx % C2)] = make_float2(v.x, v.y);
      Ts[(idx / C2) * CP + 2 * (idx % C2) + 1] = make_float2(v.z, v.w);
    }
  }

  // z = s (.) (K_S t)
  if (!acquire(mi)) return;
  zero();
  contract(mi & 1, Ts);
  store_partial(red);
  ++mi;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < RQ; ++q) {
    const int idx = tid + 256 * q;
    if (idx < NB * C)
      Zs[(idx / C) * CP + idx % C] =
          n0 + idx / C < N ? cmul(pre(sq, p.s, q), reduced(red, idx)) : make_float2(0.f, 0.f);
  }

  // e' = e + W^(i) z
  if (!acquire(mi)) return;
  zero();
  contract(mi & 1, Zs);
  store_partial(red);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < RQ; ++q) {
    const int idx = tid + 256 * q;
    if (idx < NB * C && n0 + idx / C < N) {
      const float2 u = reduced(red, idx);
      eout[n0 * C + idx] = ein ? cadd(u, pre(eq, ein, q)) : u;
    }
  }
}

template <int C, int D, int TN, int CO, int KQ>
static mcmg_status smooth_rtb(const SmoothParams& p, int mode, int nrhs, cudaStream_t st) {
  using T = RtTile<C, TN, CO, KQ>;
  constexpr size_t smem = 128 + (size_t)2 * C * C * sizeof(float2) +
      (size_t)((((2 * D + 1) * T::NB * (C + 1) + 1) & ~1) + 2 * (T::valid ? T::KS : 0) * T::NB * C) *
          sizeof(float2);
  if constexpr (!T::valid || C < 8 || smem > kMaxSmem) {
    set_error("bulk register-tiled shape does not fit %d channels", C);
    return MCMG_ERR_SHAPE;
  } else {
    dim3 grid((unsigned)((p.nodes + T::NB - 1) / T::NB), (unsigned)nrhs);
    if (mode == 0) {
      auto k = k_smooth_rtb<C, D, 0, TN, CO, KQ>;
      MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem, st, p);
    } else {
      auto k = k_smooth_rtb<C, D, 1, TN, CO, KQ>;
      MCMG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      MCMG_LAUNCH_PDL(k, grid, dim3(256), smem, st, p);
    }
    MCMG_CHECK_LAUNCH("smooth_rtb");
    return MCMG_OK;
  }
}

size_t rt_smem(int C, int D, int tn, int co, int kq, bool bulk) {
  if (co > C || C % co || kq > C || C % kq) return 0;
  const int cg = C / co, ks = C / kq;
  if (cg * ks > 256 || 256 % (cg * ks)) return 0;
  const size_t nb = (size_t)(256 / (cg * ks)) * tn;
  const size_t esz = ((2 * D + 1) * nb * (C + 1) + 1) & ~(size_t)1;   // padded node rows
  return (esz + 2 * ks * nb * C) * sizeof(float2) +
         (bulk ? 128 + (size_t)2 * C * C * sizeof(float2) : 0);
}

template <int C, int D>
static mcmg_status smooth_rt_c(const SmoothParams& p, int mode, int tn, int co, int kq, bool bulk,
                               int nrhs, cudaStream_t st) {
  if (co == 4 && bulk) {
    if (tn == 8 && kq == 4) return smooth_rtb<C, D, 8, 4, 4>(p, mode, nrhs, st);
    if (tn == 4 && kq == 4) return smooth_rtb<C, D, 4, 4, 4>(p, mode, nrhs, st);
    if (tn == 4 && kq == 8) return smooth_rtb<C, D, 4, 4, 8>(p, mode, nrhs, st);
  } else if (co == 4) {
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
                               bool bulk, int nrhs, cudaStream_t st) {
  switch (C) {
    case 4: return smooth_rt_c<4, D>(p, mode, tn, co, kq, bulk, nrhs, st);
    case 8: return smooth_rt_c<8, D>(p, mode, tn, co, kq, bulk, nrhs, st);
    case 16: return smooth_rt_c<16, D>(p, mode, tn, co, kq, bulk, nrhs, st);
    case 32: return smooth_rt_c<32, D>(p, mode, tn, co, kq, bulk, nrhs, st);
    case 64: return smooth_rt_c<64, D>(p, mode, tn, co, kq, bulk, nrhs, st);
  }
  set_error("register-tiled smoothing needs 4 to 64 channels, got %d", C);
  return MCMG_ERR_SHAPE;
}

mcmg_status smooth_rt_launch(const SmoothParams& p, int C, int D, int mode, int tn, int co, int kq,
                             bool bulk, int nrhs, cudaStream_t st) {
  return D == 3 ? smooth_rt_d<3>(p, C, mode, tn, co, kq, bulk, nrhs, st)
                : smooth_rt_d<2>(p, C, mode, tn, co, kq, bulk, nrhs, st);
}

}  // namespace mcmg
