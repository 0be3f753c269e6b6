// Fused smoothing step with the channel mixing on the 5th-generation tensor
// cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// One CTA owns M = 128 consecutive nodes of a level and all C channels.  In
// real form a complex C x C matrix is the 2C x 2C block matrix
// [[Mr, -Mi], [Mi, Mr]] in interleaved (re, im) order, so every channel-mixing
// convolution of Section 3.2 becomes a dense GEMM with K = N = 2C:
//
//   X = sum_tap E_tap W~_tap^T      (neural PDE operator stencil, 2d+1 taps)
//   Y = E_0 K~_A^T                  (K_A applied to e)
//   t = r - X - a (.) Y             (FP32, complex product per channel)
//   Z = T K~_S^T,   z = s (.) Z
//   U = Z W~_i^T,   e' = e + U
//
// E_tap holds e at each node's neighbour along the tap (zero outside the
// grid).  A operands (E_tap, T, Z) and B operands (weights) live in shared
// memory in the no-swizzle K-major core-matrix layout: for every 8-element
// (16-byte) chunk of K, all rows are contiguous at a 16-byte stride, so an
// 8-row core matrix is 128 contiguous bytes (SBO = 128 B) and consecutive K
// chunks are one tile-height apart (LBO = rows * 16 B).  The tap loop is a
// two-stage pipeline: while the MMAs of tap j run, all threads gather tap j+1
// into the other buffer.  X, Y (then Z, U) occupy 2 * 2C TMEM columns.
//
// Every mbarrier wait is bounded: on timeout the CTA records an error code,
// waits (bounded) for its own MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "mcmg_internal.cuh"
#include "tcgen05.cuh"

namespace mcmg {

struct TcParams {
  const float2* r;
  const float2* e_in;     // null: e = 0 (first pre-smoothing step)
  float2* e_out;
  const float2* a;
  const float2* s;
  const uint4* Wtap;      // [T] tiles, each K2*K2 bf16 in the core-matrix layout
  const uint4* KA;
  const uint4* KS;
  const uint4* Wi;        // W^(i) of this step
  int nx, ny, nz;
  long long nodes;
  int* err;               // error word (mapped host memory), may be null
};

// MMAs of one GEMM: D[128 x K2] (+)= A[128 x K2] B[K2 x K2]^T, K in steps of 16.
template <int K2>
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, const uint8_t* A, const uint8_t* B,
                                           bool accumulate) {
  constexpr uint32_t idesc = tc::make_idesc(tc::M, K2);
  const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
  const uint32_t lbo_a = tc::M * 16, lbo_b = K2 * 16;
#pragma unroll
  for (int s = 0; s < K2 / 16; ++s) {
    const uint64_t ad = tc::make_desc(a0 + 2 * s * lbo_a, lbo_a, 128);
    const uint64_t bd = tc::make_desc(b0 + 2 * s * lbo_b, lbo_b, 128);
    tc::mma_bf16(d_tmem, ad, bd, idesc, (accumulate || s > 0) ? 1u : 0u);
  }
}

// Load the 16-byte chunk `ch` of row `row` of a tap's A tile (BF16 of the
// neighbour's e, zero outside the grid) into a register.
template <int K2>
__device__ __forceinline__ uint4 load_chunk(const float2* __restrict__ src, long long n0, int row,
                                            int ch, const TcParams& p, int tap) {
  const long long n = n0 + row;
  uint4 out = make_uint4(0, 0, 0, 0);
  if (n >= p.nodes) return out;
  long long nb = n;
  if (tap > 0) {
    const int axis = (tap - 1) >> 1;
    const int sgn = (tap & 1) ? -1 : 1;
    const int x = (int)(n % p.nx);
    const long long rest = n / p.nx;
    const int y = (int)(rest % p.ny);
    const int z = (int)(rest / p.ny);
    const int c = axis == 0 ? x : (axis == 1 ? y : z);
    const int ext = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
    const long long stride = axis == 0 ? 1 : (axis == 1 ? p.nx : (long long)p.nx * p.ny);
    if (c + sgn < 0 || c + sgn >= ext) return out;
    nb = n + sgn * stride;
  }
  const float4* q = reinterpret_cast<const float4*>(src + nb * (K2 / 2) + ch * 4);
  const float4 u = __ldg(q), v = __ldg(q + 1);
  out.x = tc::pack_bf16(u.x, u.y);
  out.y = tc::pack_bf16(u.z, u.w);
  out.z = tc::pack_bf16(v.x, v.y);
  out.w = tc::pack_bf16(v.z, v.w);
  return out;
}

__device__ __forceinline__ void store_chunk(uint8_t* tile, int row, int ch, uint4 v) {
  *reinterpret_cast<uint4*>(tile + (size_t)ch * tc::M * 16 + (size_t)row * 16) = v;
}

// Tiles staged through registers: every global load of a tile is issued
// before any of its shared-memory stores, so the loads of a thread overlap.
template <int K2>
struct Stage {
  static constexpr int T = tc::Threads<K2>::value;
  static constexpr int PER = tc::M * (K2 / 8) / T;              // A chunks / thread
  static constexpr int N16 = K2 * K2 * 2 / 16;                  // B uint4 per tile
  static constexpr int BPER = (N16 + T - 1) / T;                // B uint4 / thread
};

template <int K2>
__device__ __forceinline__ void load_a(uint4 (&v)[Stage<K2>::PER], const float2* __restrict__ src,
                                       long long n0, const TcParams& p, int tap) {
#pragma unroll
  for (int i = 0; i < Stage<K2>::PER; ++i) {
    const int idx = threadIdx.x + i * Stage<K2>::T;
    v[i] = load_chunk<K2>(src, n0, idx % tc::M, idx / tc::M, p, tap);
  }
}

template <int K2>
__device__ __forceinline__ void store_a(uint8_t* tile, const uint4 (&v)[Stage<K2>::PER]) {
#pragma unroll
  for (int i = 0; i < Stage<K2>::PER; ++i) {
    const int idx = threadIdx.x + i * Stage<K2>::T;
    store_chunk(tile, idx % tc::M, idx / tc::M, v[i]);
  }
}

template <int K2>
__device__ __forceinline__ void load_b(uint4 (&v)[Stage<K2>::BPER], const uint4* __restrict__ src) {
#pragma unroll
  for (int i = 0; i < Stage<K2>::BPER; ++i) {
    const int idx = threadIdx.x + i * Stage<K2>::T;
    v[i] = idx < Stage<K2>::N16 ? __ldg(src + idx) : make_uint4(0, 0, 0, 0);
  }
}

template <int K2>
__device__ __forceinline__ void store_b(uint8_t* tile, const uint4 (&v)[Stage<K2>::BPER]) {
#pragma unroll
  for (int i = 0; i < Stage<K2>::BPER; ++i) {
    const int idx = threadIdx.x + i * Stage<K2>::T;
    if (idx < Stage<K2>::N16) reinterpret_cast<uint4*>(tile)[idx] = v[i];
  }
}

// Epilogue thread mapping: warp w reads TMEM lanes 32 (w % 4) .. + 31 (one node
// per lane) and the column half w / 4.
template <int K2>
struct Epi {
  static constexpr int GROUPS = tc::Threads<K2>::value / 128;   // warps sharing a lane quarter
  static constexpr int HC = K2 / GROUPS;             // FP32 columns per thread
  static constexpr int STEP = HC < 16 ? HC : 16;     // columns per TMEM load
  static constexpr int NCH = HC / 2;                 // complex channels per thread
};

template <int K2>
__device__ __forceinline__ void tmem_cols(uint32_t taddr, float* v) {
  if (Epi<K2>::STEP == 16) tc::tmem_ld16(taddr, v);
  else tc::tmem_ld8(taddr, v);
}

template <int K2, int D>
__global__ void __launch_bounds__(tc::Threads<K2>::value, (K2 >= 64 ? 1 : 8)) k_smooth_tc(TcParams p) {
  constexpr int C = K2 / 2;
  constexpr int NT = 2 * D + 1;
  constexpr int NA = 2;                      // A tiles (double buffer)
  constexpr uint32_t TM_COLS = (2 * K2 < 32) ? 32 : 2 * K2;
  constexpr size_t A_BYTES = (size_t)tc::M * K2 * 2;
  constexpr size_t B_BYTES = (size_t)K2 * K2 * 2;
  constexpr int PER = Stage<K2>::PER;                // chunks per thread per tile (>= 1)
  static_assert(PER >= 1, "tile smaller than the block");
  using E = Epi<K2>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Abase = smem;
  uint8_t* Bbase = smem + NA * A_BYTES;
  auto Atile = [&](int i) { return Abase + (size_t)i * A_BYTES; };
  auto Btile = [&](int i) { return Bbase + (size_t)i * B_BYTES; };
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_base_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long N = p.nodes;
  const size_t off = (size_t)blockIdx.y * (size_t)N * C;
  const float2* r = p.r + off;
  const float2* ein = p.e_in ? p.e_in + off : nullptr;
  float2* eout = p.e_out + off;
  const long long n0 = (long long)blockIdx.x * tc::M;
  // epilogue mapping
  const int q4 = warp & 3, half = warp >> 2;
  const int erow = 32 * q4 + lane;
  const long long en = n0 + erow;
  const long long enc = en < N ? en : N - 1;
  const uint32_t lanebits = (uint32_t)(32 * q4) << 16;
  const int cbase = half * E::HC;                    // first FP32 column of this thread

  if (threadIdx.x == 0) {
    tc::bar_init(&bars[0], 1);
    tc::bar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base_sh)),
                 "r"(TM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t tX = tmem, tY = tmem + K2;          // later Z in tX, U in tY
  uint32_t phase[2] = {0, 0};
  bool ok = true;
  auto wait_bar = [&](int b) -> bool {
    const bool w = tc::bar_wait(&bars[b], phase[b], p.err);
    phase[b] ^= 1;
    return w;
  };

  // ---------------- phase 1: X = sum_tap E_tap W~_tap^T, Y = E_0 K~_A^T ----------------
  if (ein) {
    {
      // tap t's gather lives in register stage t & 1 from the iteration
      // before it is stored: the global loads of tap j+2 are issued before the
      // wait for the MMAs of tap j-1 and the stores of tap j+1
      uint4 av0[Stage<K2>::PER], av1[Stage<K2>::PER], bv[Stage<K2>::BPER], kv[Stage<K2>::BPER];
      load_a<K2>(av0, ein, n0, p, 0);
      load_a<K2>(av1, ein, n0, p, 1);
      load_b<K2>(bv, p.Wtap);
      load_b<K2>(kv, p.KA);
      store_a<K2>(Atile(0), av0);
      store_b<K2>(Btile(0), bv);
      store_b<K2>(Btile(2), kv);
      tc::fence_async_smem();
      __syncthreads();
      auto advance = [&](uint4 (&cur)[Stage<K2>::PER], uint4 (&nxt)[Stage<K2>::PER],
                         int j) -> bool {
        const int nb = (j + 1) & 1;
        if (j + 2 < NT) load_a<K2>(nxt, ein, n0, p, j + 2);
        load_b<K2>(bv, p.Wtap + (size_t)(j + 1) * (B_BYTES / 16));
        if (j >= 1 && !wait_bar(nb)) return false;   // buffers of tap j-1 free
        store_a<K2>(Atile(nb), cur);
        store_b<K2>(Btile(nb), bv);
        tc::fence_async_smem();
        __syncthreads();
        return true;
      };
      for (int j = 0; j < NT && ok; ++j) {
        const int b = j & 1;
        if (threadIdx.x == 0) {
          tc::fence_after();
          issue_gemm<K2>(tX, Atile(b), Btile(b), j > 0);
          if (j == 0) issue_gemm<K2>(tY, Atile(0), Btile(2), false);
          tc::mma_commit(&bars[b]);
        }
        if (j + 1 < NT) ok = (j & 1) ? advance(av0, av1, j) : advance(av1, av0, j);
      }
      // outstanding: the commits of taps NT-2 and NT-1
      if (ok) ok = wait_bar((NT - 2) & 1);
      if (ok) ok = wait_bar((NT - 1) & 1);
    }
    if (!ok) goto fail;
    tc::fence_after();
    // ---- epilogue 1: t = r - X - a (.) Y -> BF16 into A tile 0
    for (int c0 = cbase; c0 < cbase + E::HC; c0 += E::STEP) {
      float x[16], y[16];
      tmem_cols<K2>(tX + lanebits + c0, x);
      tmem_cols<K2>(tY + lanebits + c0, y);
      uint32_t pk[8];
#pragma unroll
      for (int k = 0; k < E::STEP / 2; ++k) {
        const int ch = c0 / 2 + k;
        const float2 rv = r[enc * C + ch];
        const float2 av = p.a[enc * C + ch];
        const float tr = rv.x - x[2 * k] - (av.x * y[2 * k] - av.y * y[2 * k + 1]);
        const float ti = rv.y - x[2 * k + 1] - (av.x * y[2 * k + 1] + av.y * y[2 * k]);
        pk[k] = (en < N) ? tc::pack_bf16(tr, ti) : 0u;
      }
#pragma unroll
      for (int k8 = 0; k8 < E::STEP / 8; ++k8)
        store_chunk(Atile(0), erow, (c0 + 8 * k8) / 8,
                    make_uint4(pk[4 * k8], pk[4 * k8 + 1], pk[4 * k8 + 2], pk[4 * k8 + 3]));
    }
  } else {
    // first pre-smoothing step: t = r
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = threadIdx.x + i * Stage<K2>::T;
      store_chunk(Atile(0), idx % tc::M, idx / tc::M, load_chunk<K2>(r, n0, idx % tc::M, idx / tc::M, p, 0));
    }
  }

  // ---------------- phase 2: Z = T K~_S^T, z = s (.) Z -> BF16 into A tile 1 ----------------
  {
    {
      uint4 bv[Stage<K2>::BPER];
      load_b<K2>(bv, p.KS);
      store_b<K2>(Btile(0), bv);
    }
    // operands of the epilogue, fetched while the MMA runs
    float2 sv[E::NCH <= 8 ? E::NCH : 1];
    if constexpr (E::NCH <= 8) {
#pragma unroll
      for (int k = 0; k < E::NCH; ++k) sv[k] = p.s[enc * C + cbase / 2 + k];
    }
    tc::fence_before();
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after();
      issue_gemm<K2>(tX, Atile(0), Btile(0), false);
      tc::mma_commit(&bars[0]);
    }
    if (!wait_bar(0)) { ok = false; goto fail; }
    tc::fence_after();
    for (int c0 = cbase; c0 < cbase + E::HC; c0 += E::STEP) {
      float zv[16];
      tmem_cols<K2>(tX + lanebits + c0, zv);
      uint32_t pk[8];
#pragma unroll
      for (int k = 0; k < E::STEP / 2; ++k) {
        float2 s2;
        if constexpr (E::NCH <= 8) s2 = sv[k];
        else s2 = p.s[enc * C + c0 / 2 + k];
        const float zr = s2.x * zv[2 * k] - s2.y * zv[2 * k + 1];
        const float zi = s2.x * zv[2 * k + 1] + s2.y * zv[2 * k];
        pk[k] = (en < N) ? tc::pack_bf16(zr, zi) : 0u;
      }
#pragma unroll
      for (int k8 = 0; k8 < E::STEP / 8; ++k8)
        store_chunk(Atile(1), erow, (c0 + 8 * k8) / 8,
                    make_uint4(pk[4 * k8], pk[4 * k8 + 1], pk[4 * k8 + 2], pk[4 * k8 + 3]));
    }
  }

  // ---------------- phase 3: U = Z W~_i^T, e' = e + U ----------------
  {
    {
      uint4 bv[Stage<K2>::BPER];
      load_b<K2>(bv, p.Wi);
      store_b<K2>(Btile(1), bv);
    }
    float2 ev[E::NCH <= 8 ? E::NCH : 1];
    if constexpr (E::NCH <= 8) {
#pragma unroll
      for (int k = 0; k < E::NCH; ++k)
        ev[k] = ein ? ein[enc * C + cbase / 2 + k] : make_float2(0.f, 0.f);
    }
    tc::fence_before();
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after();
      issue_gemm<K2>(tY, Atile(1), Btile(1), false);
      tc::mma_commit(&bars[1]);
    }
    if (!wait_bar(1)) { ok = false; goto fail; }
    tc::fence_after();
    for (int c0 = cbase; c0 < cbase + E::HC; c0 += E::STEP) {
      float u[16];
      tmem_cols<K2>(tY + lanebits + c0, u);
      if (en < N) {
#pragma unroll
        for (int k = 0; k < E::STEP / 2; ++k) {
          const int ch = c0 / 2 + k;
          float2 v = make_float2(u[2 * k], u[2 * k + 1]);
          if constexpr (E::NCH <= 8) v = cadd(v, ev[k]);
          else if (ein) v = cadd(v, ein[en * C + ch]);
          eout[en * C + ch] = v;
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(TM_COLS));
  }
  return;

fail:
  // a bounded wait ran out: record it, give the MMAs a last bounded chance to
  // finish, release tensor memory and leave.
  if (p.err) atomicOr(p.err, 1);
  tc::bar_wait(&bars[0], phase[0], nullptr);
  tc::bar_wait(&bars[1], phase[1], nullptr);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(TM_COLS));
  }
}

template <int K2, int D>
static size_t tc_smem_bytes() {
  const size_t need = 2 * (size_t)tc::M * K2 * 2 + 3 * (size_t)K2 * K2 * 2 + 1024;
  const size_t guard = (size_t)tc::M * K2 * 2 + 36 * 1024;
  return need > guard ? need : guard;
}

template <int K2, int D>
static mcmg_status tc_launch(const TcParams& p, int nrhs, cudaStream_t st) {
  const size_t smem = tc_smem_bytes<K2, D>();
  static bool attr_set = false;   // one attribute call per instantiation
  if (!attr_set) {
    MCMG_CUDA(cudaFuncSetAttribute(k_smooth_tc<K2, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    attr_set = true;
  }
  dim3 grid((unsigned)((p.nodes + tc::M - 1) / tc::M), (unsigned)nrhs);
  k_smooth_tc<K2, D><<<grid, tc::Threads<K2>::value, smem, st>>>(p);
  MCMG_CHECK_LAUNCH("smooth_tc");
  return MCMG_OK;
}

bool tc_supported(int C) { return C == 8 || C == 16 || C == 32 || C == 64; }

mcmg_status launch_smooth_tc(const Level& L, const TcWeights& W, int step, const float2* r,
                             const float2* e_in, float2* e_out, int nrhs, int* err,
                             cudaStream_t st) {
  TcParams p;
  p.r = r;
  p.e_in = e_in;
  p.e_out = e_out;
  p.a = L.a;
  p.s = L.s;
  const size_t tile16 = (size_t)(2 * L.C) * (2 * L.C) * 2 / 16;
  p.Wtap = W.tiles;
  p.KA = W.tiles + (size_t)(2 * L.g.d + 1) * tile16;
  p.KS = p.KA + tile16;
  p.Wi = p.KS + tile16 * (1 + step);
  p.nx = L.g.nx;
  p.ny = L.g.ny;
  p.nz = L.g.nz;
  p.nodes = L.g.nodes();
  p.err = err;
  const bool d3 = L.g.d == 3;
  switch (L.C) {
    case 8: return d3 ? tc_launch<16, 3>(p, nrhs, st) : tc_launch<16, 2>(p, nrhs, st);
    case 16: return d3 ? tc_launch<32, 3>(p, nrhs, st) : tc_launch<32, 2>(p, nrhs, st);
    case 32: return d3 ? tc_launch<64, 3>(p, nrhs, st) : tc_launch<64, 2>(p, nrhs, st);
    case 64: return d3 ? tc_launch<128, 3>(p, nrhs, st) : tc_launch<128, 2>(p, nrhs, st);
  }
  set_error("tensor-core smoothing needs C in {8, 16, 32, 64}, got %d", L.C);
  return MCMG_ERR_SHAPE;
}

// Host: a complex C x C matrix M[co][ci] (float2, row-major) -> its real
// 2C x 2C block form as BF16 in the core-matrix layout of a B operand
// (row n = output index, K = input index, chunk-major).
void pack_tc_tile(const float2* Mc, int C, uint16_t* out) {
  const int K2 = 2 * C;
  for (int n = 0; n < K2; ++n)
    for (int k = 0; k < K2; ++k) {
      const float2 m = Mc[(size_t)(n >> 1) * C + (k >> 1)];
      float v;
      if ((n & 1) == 0) v = (k & 1) == 0 ? m.x : -m.y;   // re out: Mr re_in - Mi im_in
      else v = (k & 1) == 0 ? m.y : m.x;                 // im out: Mi re_in + Mr im_in
      __nv_bfloat16 b = __float2bfloat16_rn(v);
      const size_t pos = ((size_t)(k >> 3) * K2 + n) * 8 + (k & 7);
      out[pos] = *reinterpret_cast<uint16_t*>(&b);
    }
}

}  // namespace mcmg
