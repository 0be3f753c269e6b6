// Smoothing step and residual of the McMg V-cycle (Section 3.2, Algorithm 2)
// with every channel-mixing convolution on the tcgen05 tensor cores, the A
// operands in tensor memory and persistent CTAs.
//
// In real form a complex C x C matrix is the 2C x 2C block matrix
// [[Mr, -Mi], [Mi, Mr]] in interleaved (re, im) order, so with K2 = 2C every
// mixing convolution is a GEMM over a tile of M = 128 nodes:
//
//   X = sum_tap E_tap W~_tap^T     (neural PDE operator stencil, 2d+1 taps)
//   Y = E_0 K~_A^T
//   t = r - X - a (.) Y            (FP32)          -- residual mode stops here
//   Z = T K~_S^T,  z = s (.) Z
//   U = Z W~_i^T,  e' = e + U
//
// Thread i of the 128 owns node n0 + i and TMEM lane i.  For each tap it
// gathers the neighbour's C complex values into registers (zero outside the
// grid), converts them to the operand type and writes them to one of two
// A slots in tensor memory with tcgen05.st; one thread then issues the MMAs
// that read A from tensor memory and B (the weights, copied to shared memory
// once per CTA) through shared-memory descriptors, accumulating in TMEM.
// While the MMAs of tap j run, the threads fill the other slot with tap j+1,
// and the loads of tap j+2 are already in flight.
//
// Operand precision:
//   BF16    one MMA per K step (BF16 A and B, FP32 accumulation).
//   TF32x3  FP32-accurate: each FP32 value x is split into hi = tf32(x) and
//           lo = tf32(x - hi) (round to nearest), likewise every weight, and
//           D += A_lo B_hi + A_hi B_lo + A_hi B_hi, dropping only A_lo B_lo:
//           about 2^-21 relative per product, the FP32 rounding order aside.
//
// CTAs are persistent: each allocates its TMEM columns and loads the weights
// once, then walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...  so at any
// time the CTAs of the grid work on a contiguous window of the level and the
// stencil neighbours of a tile are still in L2.  The launch keeps at most
// 512 / (TMEM columns per CTA) CTAs on one SM, so an allocation never waits.
//
// Every mbarrier wait is bounded (about a second); the block votes on the
// outcome at its next barrier, so all threads leave together: the CTA records
// an error code, waits (bounded) for its own MMAs, frees its TMEM and returns.
#include <algorithm>
#include <cstring>

#include "mcmg_internal.cuh"
#include "tcgen05.cuh"
#include "vcycle_kernels.cuh"

namespace mcmg {

namespace ts {

constexpr int M = 128;          // nodes per tile (MMA M), one thread per node
constexpr int THREADS = 128;
constexpr int SM_SMEM = 228 * 1024;   // shared memory of one SM
constexpr int BLOCK_RESERVED = 1024;  // per-block shared memory the system keeps

template <int K2, int P>  // P: 0 BF16, 1 TF32x3
struct Cfg {
  static constexpr int AW = P ? 2 * K2 : K2 / 2;     // TMEM columns of one A slot
  static constexpr int NEED = 2 * K2 + 2 * AW;        // X, Y, two A slots
  static constexpr int COLS = NEED <= 32 ? 32 : NEED <= 64 ? 64 : NEED <= 128 ? 128
                              : NEED <= 256 ? 256 : 512;
  static constexpr int PER_SM = 512 / COLS;           // CTAs per SM that TMEM holds
  static constexpr int HALF = P ? K2 * K2 * 4 : K2 * K2 * 2;  // one weight matrix
  static constexpr int MAT = P ? 2 * HALF : HALF;     // hi + lo, or BF16
  static constexpr int KSTEP = P ? 8 : 16;            // K of one MMA
};

}  // namespace ts

struct TsParams {
  const float2* r;
  const float2* e_in;     // null: e = 0 (first pre-smoothing step, step mode only)
  float2* out;            // e' (step mode) or t = r - A_l(e) (residual mode)
  const float2* a;
  const float2* s;
  const uint4* mats;      // [taps][K_A][K_S][W^(0) ...], ts::Cfg::MAT bytes each
  int wi;                 // matrix index of this step's W^(i)
  int nx, ny, nz;
  long long nodes;        // per field
  int tiles;              // per field
  int items;              // tiles * fields (or the descriptors' tiles in total)
  int* err;               // error word (mapped host memory), may be null
  // batched launch over fields of different grids and features: when set,
  // item i belongs to the last descriptor whose `first` <= i, and the fields
  // above (r, e_in, out, a, s, nx, ny, nz, nodes, tiles) are not used, except
  // that e_in is non-null exactly when every descriptor's e_in is
  const TsField* fields;
  int nfields;
  // Level 0 of a one-field V-cycle (k_smooth_ts only; null otherwise): the
  // lift and the projection of Algorithm 2 folded into the step.  r_cell
  // holds the address of the scalar residual r and the step reads
  // r_1 = lift (x) r[n] in place of p.r; z_cell holds the address of the
  // scalar output, and the step writes sum_c proj[c] e'[n][c] there in place
  // of e'.  The addresses sit in device cells so that a captured graph
  // follows the caller's buffers.
  const float2* const* r_cell;
  const float2* lift;
  float2* const* z_cell;
  const float2* proj;
};

namespace ts {

// The MMAs of D (+)= A B^T for one weight matrix: A in TMEM at a_slot, B in
// shared memory at b (no-swizzle K-major core matrices, LBO = K2 * 16 B
// between 16-byte K chunks, SBO = 128 B between 8-row groups).
template <int K2, int P>
__device__ __forceinline__ void gemm(uint32_t d, uint32_t a_slot, uint32_t b, bool accumulate) {
  // one descriptor per matrix, stepped along K by adding the byte offset >> 4
  // to its start-address field (the shared-memory addresses stay below 256 KB)
  constexpr uint32_t lbo = K2 * 16;
  constexpr uint64_t kstep = (2 * lbo) >> 4;
  if constexpr (P == 0) {
    constexpr uint32_t idesc = tc::make_idesc(M, K2);
    const uint64_t b0 = tc::make_desc(b, lbo, 128);
#pragma unroll
    for (int s = 0; s < K2 / 16; ++s)
      tc::mma_bf16_ts(d, a_slot + 8 * s, b0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
  } else {
    constexpr uint32_t idesc = tc::make_idesc_tf32(M, K2);
    const uint64_t bh0 = tc::make_desc(b, lbo, 128);
    const uint64_t bl0 = bh0 + (Cfg<K2, P>::HALF >> 4);
#pragma unroll
    for (int s = 0; s < K2 / 8; ++s) {
      const uint32_t ahi = a_slot + 8 * s, alo = a_slot + K2 + 8 * s;
      tc::mma_tf32_ts(d, alo, bh0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
      tc::mma_tf32_ts(d, ahi, bl0 + s * kstep, idesc, 1u);
      tc::mma_tf32_ts(d, ahi, bh0 + s * kstep, idesc, 1u);
    }
  }
}

// 16 FP32 values of this thread's row -> operand columns c0 .. c0+15 of an
// A slot (TF32 hi at c0, lo at K2 + c0; or 8 packed BF16 pairs at c0 / 2).
template <int K2, int P>
__device__ __forceinline__ void put16(uint32_t slot, int c0, const float* v) {
  if constexpr (P == 1) {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      hi[i] = tc::to_tf32(v[i]);
      lo[i] = tc::to_tf32(v[i] - __uint_as_float(hi[i]));
    }
    tc::tmem_st16(slot + c0, hi);
    tc::tmem_st16(slot + K2 + c0, lo);
  } else {
    uint32_t pk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) pk[i] = tc::pack_bf16(v[2 * i], v[2 * i + 1]);
    tc::tmem_st8(slot + c0 / 2, pk);
  }
}

// Row `n` of a [nodes][C] complex field as K2 floats (zeros when !ok).
template <int K2>
__device__ __forceinline__ void load_row(float (&v)[K2], const float2* __restrict__ src,
                                         long long n, bool ok) {
  const float4* q = reinterpret_cast<const float4*>(src + n * (K2 / 2));
#pragma unroll
  for (int i = 0; i < K2 / 4; ++i) {
    const float4 t = ok ? __ldg(q + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    v[4 * i] = t.x;
    v[4 * i + 1] = t.y;
    v[4 * i + 2] = t.z;
    v[4 * i + 3] = t.w;
  }
}

// 16 floats (8 complex channels) of row n starting at float c0.
__device__ __forceinline__ void load16(float* v, const float2* __restrict__ src, int C, long long n,
                                       int c0) {
  const float4* q = reinterpret_cast<const float4*>(src + n * C + c0 / 2);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 t = __ldg(q + i);
    v[4 * i] = t.x;
    v[4 * i + 1] = t.y;
    v[4 * i + 2] = t.z;
    v[4 * i + 3] = t.w;
  }
}

// One tile's field: its pointers (field offsets applied), grid and first node.
struct Tile {
  const float2* r;
  const float2* e_in;
  float2* out;
  const float2* a;
  const float2* s;
  long long nodes, n0;
  int nx, ny, nz;
};

__device__ __forceinline__ Tile tile_of(const TsParams& p, int item, int C) {
  Tile t;
  if (!p.fields) {
    const int field = item / p.tiles, tile = item - field * p.tiles;
    const size_t off = (size_t)field * (size_t)p.nodes * C;
    t.r = p.r + off;
    t.e_in = p.e_in ? p.e_in + off : nullptr;
    t.out = p.out + off;
    t.a = p.a;
    t.s = p.s;
    t.nodes = p.nodes;
    t.nx = p.nx;
    t.ny = p.ny;
    t.nz = p.nz;
    t.n0 = (long long)tile * M;
  } else {
    int lo = 0, hi = p.nfields - 1;       // the last descriptor with first <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.fields[mid].first <= item) lo = mid;
      else hi = mid - 1;
    }
    const TsField& d = p.fields[lo];
    t.r = d.r;
    t.e_in = d.e_in;
    t.out = d.out;
    t.a = d.a;
    t.s = d.s;
    t.nodes = d.nodes;
    t.nx = d.nx;
    t.ny = d.ny;
    t.nz = d.nz;
    t.n0 = (long long)(item - d.first) * M;
  }
  return t;
}

__device__ __forceinline__ void store16(float2* dst, int C, long long n, int c0, const float* v) {
  float4* q = reinterpret_cast<float4*>(dst + n * C + c0 / 2);
#pragma unroll
  for (int i = 0; i < 4; ++i) q[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// ---- the copy ring of the K2 <= 32 kernels --------------------------------
// A segment is 128 consecutive rows (nodes) of a [nodes][C] complex field,
// K2 floats each.  Every thread copies CPR = K2 / 4 chunks of 16 bytes with
// cp.async (consecutive threads read consecutive chunks: coalesced) into a
// ring buffer, 16-byte chunk c of row r stored at chunk position c ^ swz(r),
// so that thread r later reads its own row without bank conflicts; rows
// outside the field are zero-filled.  Each thread's copies arrive on the
// buffer's mbarrier (count 128) once they have landed.
template <int K2, int P>
struct Ring {
  static constexpr int CPR = K2 / 4;                     // 16-byte chunks per row
  static constexpr int ROWB = K2 * 4;                    // bytes per row
  static constexpr int SEG = M * ROWB;                   // bytes per segment
  static constexpr int R = K2 == 16 ? 4 : 2;             // ring depth (segments)
  static constexpr int WBYTES_MAX = 10 * Cfg<K2, P>::MAT;  // 3D step: 7 taps + K_A, K_S, W^(i)
  static constexpr int SMEM = WBYTES_MAX + R * SEG;
  static constexpr int BY_SMEM = SM_SMEM / (SMEM + 2 * BLOCK_RESERVED);
  static constexpr int PER_SM = Cfg<K2, P>::PER_SM < BY_SMEM ? Cfg<K2, P>::PER_SM : BY_SMEM;
};

template <int K2>
__device__ __forceinline__ int swz(int row) {
  return K2 == 16 ? (row >> 1) & 3 : row & 7;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(src_bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(tc::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Copy rows start .. start+127 of `base` ([nodes][K2/2] complex) into a ring
// buffer; rows outside [0, nodes) are zero-filled without a read.
template <int K2, int P>
__device__ __forceinline__ void copy_segment(uint32_t dst, const float2* base, long long start,
                                             long long nodes, int tid) {
  using RG = Ring<K2, P>;
#pragma unroll
  for (int m = 0; m < RG::CPR; ++m) {
    const int k = tid + m * THREADS;
    const int row = k / RG::CPR, c = k % RG::CPR;
    const long long sr = start + row;
    const bool v = sr >= 0 && sr < nodes;
    const float2* src = base + (v ? sr : 0) * (K2 / 2) + 2 * c;
    cp_async16(dst + row * RG::ROWB + 16 * (c ^ swz<K2>(row)), src, v ? 16u : 0u);
  }
}

// 16 floats of this thread's row (columns c0 .. c0+15) from a ring buffer.
template <int K2, int P>
__device__ __forceinline__ void ring_read16(const uint8_t* buf, int row, int c0, float* v) {
  using RG = Ring<K2, P>;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = c0 / 4 + i;
    const float4 t = *reinterpret_cast<const float4*>(buf + row * RG::ROWB + 16 * (c ^ swz<K2>(row)));
    v[4 * i] = t.x;
    v[4 * i + 1] = t.y;
    v[4 * i + 2] = t.z;
    v[4 * i + 3] = t.w;
  }
}

}  // namespace ts

template <int K2, int D, int P, int MODE>
__global__ void __launch_bounds__(ts::THREADS, ts::Cfg<K2, P>::PER_SM) k_smooth_ts(TsParams p) {
  using G = ts::Cfg<K2, P>;
  constexpr int C = K2 / 2;
  constexpr int NT = 2 * D + 1;
  constexpr int NM = MODE == 0 ? NT + 3 : NT + 1;     // matrices this kernel reads
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5;

  // weights -> shared memory: taps, K_A [, K_S, W^(i)]
  {
    constexpr int PER = G::MAT / 16;
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (int m = 0; m < NM; ++m) {
      const int gm = (MODE == 0 && m == NT + 2) ? p.wi : m;
      for (int i = tid; i < PER; i += ts::THREADS)
        dst[m * PER + i] = __ldg(p.mats + (size_t)gm * PER + i);
    }
  }
  if (tid == 0) {
    tc::bar_init(&bars[0], 1);
    tc::bar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)G::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t lane = (uint32_t)(32 * warp) << 16;
  const uint32_t tX = tmem, tY = tmem + K2;          // Z reuses X, U reuses Y
  const uint32_t slot0 = tmem + 2 * K2, slot1 = slot0 + G::AW;
  const uint32_t wbase = tc::smem_u32(smem);
  auto mat = [&](int m) { return wbase + (uint32_t)(m * G::MAT); };
  uint32_t phase[2] = {0, 0};
  bool ok = true;
  auto wait_bar = [&](int b) -> bool {
    const bool w = tc::bar_wait(&bars[b], phase[b], p.err);
    phase[b] ^= 1;
    return w;
  };

  for (int item = blockIdx.x; item < p.items; item += gridDim.x) {
    const ts::Tile tv = ts::tile_of(p, item, C);
    // r_1 row of node nn: read, or lifted from the scalar residual
    auto load_r = [&](float (&v)[K2], long long nn) {
      if (p.r_cell) {
        const float2 rs = (*p.r_cell)[nn];
#pragma unroll
        for (int c = 0; c < C; ++c) {       // as k_lift: bit for bit
          const float2 t = cmul_rn(__ldg(p.lift + c), rs);
          v[2 * c] = t.x;
          v[2 * c + 1] = t.y;
        }
      } else {
        ts::load_row<K2>(v, tv.r, nn, true);
      }
    };
    const float2* ein = tv.e_in;
    float2* out = tv.out;
    const long long n = tv.n0 + tid;
    const bool row_ok = n < tv.nodes;
    const long long nc = row_ok ? n : tv.nodes - 1;
    int x, y, z;
    node_xyz(nc, tv.nx, tv.ny, x, y, z);
    // neighbour of node n along tap j (centre, -x, +x, -y, +y, -z, +z)
    auto nbr = [&](int j, long long& nb) -> bool {
      if (j == 0) { nb = nc; return row_ok; }
      const int axis = (j - 1) >> 1;
      const int sgn = (j & 1) ? -1 : 1;
      const int c = axis == 0 ? x : (axis == 1 ? y : z);
      const int ext = axis == 0 ? tv.nx : (axis == 1 ? tv.ny : tv.nz);
      const long long stride = axis == 0 ? 1 : (axis == 1 ? tv.nx : (long long)tv.nx * tv.ny);
      nb = nc + sgn * stride;
      return row_ok && c + sgn >= 0 && c + sgn < ext;
    };

    // Two register rows: the stencil taps two ahead, and after the last two
    // taps the epilogue operands (r and a, then s and e) as soon as a row
    // frees up, so that their loads overlap the MMAs and the other epilogues.
    float va[K2], vb[K2];
    float(&rbuf)[K2] = ((NT - 2) & 1) ? vb : va;      // r, then s
    float(&abuf)[K2] = ((NT - 1) & 1) ? vb : va;      // a, then e
    if (ein) {
      // ---- phase 1: X = sum_tap E_tap W~_tap^T, Y = E_0 K~_A^T
      {
        long long nb;
        bool v = nbr(0, nb);
        ts::load_row<K2>(va, ein, nb, v);
        v = nbr(1, nb);
        ts::load_row<K2>(vb, ein, nb, v);
      }
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        float(&cur)[K2] = (j & 1) ? vb : va;
        const uint32_t slot = (j & 1) ? slot1 : slot0;
        if (j >= 2) ok = wait_bar(j & 1) && ok;        // MMAs of tap j-2 have read this slot
#pragma unroll
        for (int c0 = 0; c0 < K2; c0 += 16) ts::put16<K2, P>(slot + lane, c0, cur + c0);
        tc::tmem_st_wait();
        if (j + 2 < NT) {
          long long nb;
          const bool v = nbr(j + 2, nb);
          ts::load_row<K2>(cur, ein, nb, v);
        } else {
          if (j == NT - 2) load_r(cur, nc);                          // rbuf
          else ts::load_row<K2>(cur, tv.a, nc, true);                 // abuf
        }
        tc::fence_before();
        ok = __syncthreads_and(ok);
        if (!ok) goto fail;
        if (tid == 0) {
          tc::fence_after();
          ts::gemm<K2, P>(tX, slot, mat(j), j > 0);
          if (j == 0) ts::gemm<K2, P>(tY, slot, mat(NT), false);
          tc::mma_commit(&bars[j & 1]);
        }
      }
      ok = wait_bar((NT - 2) & 1) && ok;
      ok = wait_bar((NT - 1) & 1) && ok;
      tc::fence_after();
      // ---- epilogue 1: t = r - X - a (.) Y
#pragma unroll
      for (int c0 = 0; c0 < K2; c0 += 16) {
        float xv[16], yv[16], t[16];
        const float* rv = rbuf + c0;
        const float* av = abuf + c0;
        tc::tmem_ld16(tX + lane + c0, xv);
        tc::tmem_ld16(tY + lane + c0, yv);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          t[2 * k] = rv[2 * k] - xv[2 * k] - (av[2 * k] * yv[2 * k] - av[2 * k + 1] * yv[2 * k + 1]);
          t[2 * k + 1] =
              rv[2 * k + 1] - xv[2 * k + 1] - (av[2 * k] * yv[2 * k + 1] + av[2 * k + 1] * yv[2 * k]);
        }
        if constexpr (MODE == 1) {
          if (row_ok) ts::store16(out, C, n, c0, t);
        } else {
          if (!row_ok) {
#pragma unroll
            for (int k = 0; k < 16; ++k) t[k] = 0.f;
          }
          ts::put16<K2, P>(slot0 + lane, c0, t);
        }
      }
      if constexpr (MODE == 0) {
        ts::load_row<K2>(rbuf, tv.s, nc, true);     // s for epilogue 2
        ts::load_row<K2>(abuf, ein, nc, true);      // e for epilogue 3
      }
    } else {
      // first pre-smoothing step: t = r
      load_r(abuf, nc);
      ts::load_row<K2>(rbuf, tv.s, nc, true);
#pragma unroll
      for (int c0 = 0; c0 < K2; c0 += 16) {
        float rv[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) rv[k] = row_ok ? abuf[c0 + k] : 0.f;
        ts::put16<K2, P>(slot0 + lane, c0, rv);
      }
    }

    if constexpr (MODE == 0) {
      // ---- phase 2: Z = T K~_S^T; epilogue 2: z = s (.) Z
      tc::tmem_st_wait();
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) goto fail;
      if (tid == 0) {
        tc::fence_after();
        ts::gemm<K2, P>(tX, slot0, mat(NT + 1), false);
        tc::mma_commit(&bars[0]);
      }
      ok = wait_bar(0) && ok;
      tc::fence_after();
#pragma unroll
      for (int c0 = 0; c0 < K2; c0 += 16) {
        float zv[16], zz[16];
        const float* sv = rbuf + c0;
        tc::tmem_ld16(tX + lane + c0, zv);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          zz[2 * k] = sv[2 * k] * zv[2 * k] - sv[2 * k + 1] * zv[2 * k + 1];
          zz[2 * k + 1] = sv[2 * k] * zv[2 * k + 1] + sv[2 * k + 1] * zv[2 * k];
        }
        if (!row_ok) {
#pragma unroll
          for (int k = 0; k < 16; ++k) zz[k] = 0.f;
        }
        ts::put16<K2, P>(slot1 + lane, c0, zz);
      }
      // ---- phase 3: U = Z W~_i^T; epilogue 3: e' = e + U
      tc::tmem_st_wait();
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) goto fail;
      if (tid == 0) {
        tc::fence_after();
        ts::gemm<K2, P>(tY, slot1, mat(NT + 2), false);
        tc::mma_commit(&bars[1]);
      }
      ok = wait_bar(1) && ok;
      tc::fence_after();
      float2 zsum = make_float2(0.f, 0.f);          // projection (z_cell)
#pragma unroll
      for (int c0 = 0; c0 < K2; c0 += 16) {
        float uv[16];
        tc::tmem_ld16(tY + lane + c0, uv);
        if (ein) {
#pragma unroll
          for (int k = 0; k < 16; ++k) uv[k] += abuf[c0 + k];
        }
        if (p.z_cell) {                     // as k_project: channels in order
#pragma unroll
          for (int k = 0; k < 8; ++k)
            cfma(zsum, __ldg(p.proj + c0 / 2 + k), make_float2(uv[2 * k], uv[2 * k + 1]));
        } else if (row_ok) {
          ts::store16(out, C, n, c0, uv);
        }
      }
      if (p.z_cell && row_ok) (*p.z_cell)[n] = zsum;
    }
    tc::fence_before();   // this tile's TMEM reads precede the next tile's MMAs
  }
  ok = __syncthreads_and(ok);
  if (!ok) goto fail;
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)G::COLS));
  }
  return;

fail:
  // a bounded wait ran out: record it, give this CTA's MMAs a last bounded
  // chance to finish, release the tensor memory and leave
  if (p.err && tid == 0) atomicOr(p.err, 1);
  tc::bar_wait(&bars[0], phase[0], nullptr);
  tc::bar_wait(&bars[1], phase[1], nullptr);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)G::COLS));
  }
}

// The same step and residual with every field row reaching the SM through
// the copy ring: per tile the segments are the 2d+1 stencil taps of e (rows
// shifted by the tap's offset), then r and a (epilogue 1), s (epilogue 2) and
// e (epilogue 3); the residual takes the taps, r and a; the first
// pre-smoothing step (e = 0) takes r and s.  The segments of one CTA form one
// sequence over its tiles; R of them are in flight, and a buffer is refilled
// right after the block barrier that follows its last read.  Every thread
// waits for a segment's mbarrier itself before reading its own row.
template <int K2, int D, int P, int MODE>
__global__ void __launch_bounds__(ts::THREADS, ts::Ring<K2, P>::PER_SM) k_smooth_tsr(TsParams p) {
  using G = ts::Cfg<K2, P>;
  using RG = ts::Ring<K2, P>;
  constexpr int C = K2 / 2;
  constexpr int NT = 2 * D + 1;
  constexpr int NM = MODE == 0 ? NT + 3 : NT + 1;
  constexpr int R = RG::R;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint64_t full[R];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool has_e = p.e_in != nullptr;
  const int NSEG = MODE == 1 ? NT + 2 : (has_e ? NT + 4 : 2);   // segments per tile
  uint8_t* ring = smem + NM * G::MAT;
  const uint32_t ring_s = tc::smem_u32(ring);

  {
    constexpr int PER = G::MAT / 16;
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (int m = 0; m < NM; ++m) {
      const int gm = (MODE == 0 && m == NT + 2) ? p.wi : m;
      for (int i = tid; i < PER; i += ts::THREADS)
        dst[m * PER + i] = __ldg(p.mats + (size_t)gm * PER + i);
    }
  }
  if (tid == 0) {
    tc::bar_init(&bars[0], 1);
    tc::bar_init(&bars[1], 1);
    for (int b = 0; b < R; ++b) tc::bar_init(&full[b], ts::THREADS);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)G::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t lane = (uint32_t)(32 * warp) << 16;
  const uint32_t tX = tmem, tY = tmem + K2;
  const uint32_t slot0 = tmem + 2 * K2, slot1 = slot0 + G::AW;
  const uint32_t wbase = tc::smem_u32(smem);
  auto mat = [&](int m) { return wbase + (uint32_t)(m * G::MAT); };
  uint32_t phase[2] = {0, 0};
  bool ok = true;
  auto wait_bar = [&](int b) -> bool {
    const bool w = tc::bar_wait(&bars[b], phase[b], p.err);
    phase[b] ^= 1;
    return w;
  };
  const int my_tiles = blockIdx.x < p.items ? (p.items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int g_total = my_tiles * NSEG;
  // the next segment to issue, as (tile of this CTA, index within the tile)
  int g_issued = 0, is_k = 0, is_idx = 0;

  // issue the next segment of this CTA's sequence into ring buffer g_issued % R
  auto issue_next = [&]() {
    const int item = blockIdx.x + is_k * gridDim.x;
    const ts::Tile tv = ts::tile_of(p, item, C);
    const int idx = is_idx;
    const float2* base;
    long long start = tv.n0;
    if (MODE == 0 && !has_e) {
      base = idx == 0 ? tv.r : tv.s;
    } else if (idx < NT) {
      base = tv.e_in;
      if (idx > 0) {
        const int axis = (idx - 1) >> 1;
        const long long stride = axis == 0 ? 1 : (axis == 1 ? tv.nx : (long long)tv.nx * tv.ny);
        start = tv.n0 + ((idx & 1) ? -stride : stride);
      }
    } else {
      const int e = idx - NT;    // 0 r, 1 a, 2 s, 3 e
      base = e == 0 ? tv.r : e == 1 ? tv.a : e == 2 ? tv.s : tv.e_in;
    }
    const int b = g_issued % R;
    ts::copy_segment<K2, P>(ring_s + (uint32_t)(b * RG::SEG), base, start, tv.nodes, tid);
    ts::cp_async_arrive(&full[b]);
    ++g_issued;
    if (++is_idx == NSEG) { is_idx = 0; ++is_k; }
  };
  // refill every buffer whose segment all threads have read (g < g_cons)
  auto top_up = [&](int g_cons) {
    while (g_issued < g_total && g_issued < g_cons + R) issue_next();
  };
  // wait until segment g has landed in its buffer, return the buffer
  auto seg = [&](int g, bool& okk) -> const uint8_t* {
    okk = tc::bar_wait(&full[g % R], (uint32_t)((g / R) & 1), p.err) && okk;
    return ring + (g % R) * RG::SEG;
  };
  top_up(0);

  for (int k = 0; k < my_tiles; ++k) {
    const int item = blockIdx.x + k * gridDim.x;
    const ts::Tile tv = ts::tile_of(p, item, C);
    float2* out = tv.out;
    const long long n = tv.n0 + tid;
    const bool row_ok = n < tv.nodes;
    const long long nc = row_ok ? n : tv.nodes - 1;
    const int gt = k * NSEG;        // first segment of this tile
    int x, y, z;
    node_xyz(nc, tv.nx, tv.ny, x, y, z);
    auto tap_ok = [&](int j) -> bool {
      if (j == 0) return row_ok;
      const int axis = (j - 1) >> 1;
      const int sgn = (j & 1) ? -1 : 1;
      const int c = axis == 0 ? x : (axis == 1 ? y : z);
      const int ext = axis == 0 ? tv.nx : (axis == 1 ? tv.ny : tv.nz);
      return row_ok && c + sgn >= 0 && c + sgn < ext;
    };

    if (has_e) {
      // ---- phase 1: the taps
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const uint32_t slot = (j & 1) ? slot1 : slot0;
        const uint8_t* b = seg(gt + j, ok);
        if (j >= 2) ok = wait_bar(j & 1) && ok;
        const bool v = tap_ok(j);
#pragma unroll
        for (int c0 = 0; c0 < K2; c0 += 16) {
          float t[16];
          ts::ring_read16<K2, P>(b, tid, c0, t);
          if (!v) {
#pragma unroll
            for (int i = 0; i < 16; ++i) t[i] = 0.f;
          }
          ts::put16<K2, P>(slot + lane, c0, t);
        }
        tc::tmem_st_wait();
        tc::fence_before();
        ok = __syncthreads_and(ok);
        if (!ok) goto fail;
        top_up(gt + j + 1);
        if (tid == 0) {
          tc::fence_after();
          ts::gemm<K2, P>(tX, slot, mat(j), j > 0);
          if (j == 0) ts::gemm<K2, P>(tY, slot, mat(NT), false);
          tc::mma_commit(&bars[j & 1]);
        }
      }
      ok = wait_bar((NT - 2) & 1) && ok;
      ok = wait_bar((NT - 1) & 1) && ok;
      tc::fence_after();
      // ---- epilogue 1: t = r - X - a (.) Y
      {
        const uint8_t* rb = seg(gt + NT, ok);
        const uint8_t* ab = seg(gt + NT + 1, ok);
#pragma unroll
        for (int c0 = 0; c0 < K2; c0 += 16) {
          float xv[16], yv[16], rv[16], av[16], t[16];
          tc::tmem_ld16(tX + lane + c0, xv);
          tc::tmem_ld16(tY + lane + c0, yv);
          ts::ring_read16<K2, P>(rb, tid, c0, rv);
          ts::ring_read16<K2, P>(ab, tid, c0, av);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            t[2 * q] = rv[2 * q] - xv[2 * q] - (av[2 * q] * yv[2 * q] - av[2 * q + 1] * yv[2 * q + 1]);
            t[2 * q + 1] = rv[2 * q + 1] - xv[2 * q + 1] -
                           (av[2 * q] * yv[2 * q + 1] + av[2 * q + 1] * yv[2 * q]);
          }
          if constexpr (MODE == 1) {
            if (row_ok) ts::store16(out, C, n, c0, t);
          } else {
            if (!row_ok) {
#pragma unroll
              for (int i = 0; i < 16; ++i) t[i] = 0.f;
            }
            ts::put16<K2, P>(slot0 + lane, c0, t);
          }
        }
      }
      if constexpr (MODE == 1) {
        // r and a are read: free their buffers before the next tile's taps
        tc::fence_before();
        ok = __syncthreads_and(ok);
        if (!ok) goto fail;
        top_up(gt + NT + 2);
      }
    } else {
      const uint8_t* rb = seg(gt, ok);
#pragma unroll
      for (int c0 = 0; c0 < K2; c0 += 16) {
        float rv[16];
        ts::ring_read16<K2, P>(rb, tid, c0, rv);
        if (!row_ok) {
#pragma unroll
          for (int i = 0; i < 16; ++i) rv[i] = 0.f;
        }
        ts::put16<K2, P>(slot0 + lane, c0, rv);
      }
    }

    if constexpr (MODE == 0) {
      const int gs = has_e ? gt + NT + 2 : gt + 1;   // segment of s
      // ---- phase 2: Z = T K~_S^T
      tc::tmem_st_wait();
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) goto fail;
      top_up(gs);
      if (tid == 0) {
        tc::fence_after();
        ts::gemm<K2, P>(tX, slot0, mat(NT + 1), false);
        tc::mma_commit(&bars[0]);
      }
      ok = wait_bar(0) && ok;
      tc::fence_after();
      {
        const uint8_t* sb = seg(gs, ok);
#pragma unroll
        for (int c0 = 0; c0 < K2; c0 += 16) {
          float zv[16], sv[16], zz[16];
          tc::tmem_ld16(tX + lane + c0, zv);
          ts::ring_read16<K2, P>(sb, tid, c0, sv);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            zz[2 * q] = sv[2 * q] * zv[2 * q] - sv[2 * q + 1] * zv[2 * q + 1];
            zz[2 * q + 1] = sv[2 * q] * zv[2 * q + 1] + sv[2 * q + 1] * zv[2 * q];
          }
          if (!row_ok) {
#pragma unroll
            for (int i = 0; i < 16; ++i) zz[i] = 0.f;
          }
          ts::put16<K2, P>(slot1 + lane, c0, zz);
        }
      }
      // ---- phase 3: U = Z W~_i^T; e' = e + U
      tc::tmem_st_wait();
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) goto fail;
      top_up(gs + 1);
      if (tid == 0) {
        tc::fence_after();
        ts::gemm<K2, P>(tY, slot1, mat(NT + 2), false);
        tc::mma_commit(&bars[1]);
      }
      ok = wait_bar(1) && ok;
      tc::fence_after();
      {
        const uint8_t* eb = has_e ? seg(gt + NT + 3, ok) : nullptr;
#pragma unroll
        for (int c0 = 0; c0 < K2; c0 += 16) {
          float uv[16];
          tc::tmem_ld16(tY + lane + c0, uv);
          if (has_e) {
            float ev[16];
            ts::ring_read16<K2, P>(eb, tid, c0, ev);
#pragma unroll
            for (int i = 0; i < 16; ++i) uv[i] += ev[i];
          }
          if (row_ok) ts::store16(out, C, n, c0, uv);
        }
      }
    }
    tc::fence_before();
  }
  ok = __syncthreads_and(ok);
  if (!ok) goto fail;
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)G::COLS));
  }
  return;

fail:
  // a bounded wait ran out: record it, let this thread's copies land, give
  // this CTA's MMAs a last bounded chance to finish, release the tensor memory
  if (p.err && tid == 0) atomicOr(p.err, 1);
  ts::cp_async_wait_all();
  tc::bar_wait(&bars[0], phase[0], nullptr);
  tc::bar_wait(&bars[1], phase[1], nullptr);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)G::COLS));
  }
}

// ---------------------------------------------------------------------------
// Large channel counts (K2 = 64 with TF32x3, K2 = 128 with either precision):
// the weights no longer fit shared memory, so they stream through it.  CTAs
// of 256 threads, as many per SM as their TMEM columns allow (two at K2 = 64,
// one at K2 = 128): thread t owns row 32 (w % 4) + lane of warp w and every
// other 16-column chunk of it (warps 0-3 the even chunks, 4-7 the odd ones).
// Each stencil tap is one A stage, or two K-halves for TF32x3 so that two A
// slots fit beside X and Y.  The stage loop handles two stages per iteration
// so that the two register buffers are named statically: a buffer's loads,
// issued two stages ahead, stay in flight until it is converted (a buffer
// chosen at run time made the compiler wait for each load at once).  The
// weight matrices arrive per (matrix, K-half) unit in a ring of RB
// shared-memory buffers filled by bulk asynchronous copies with
// transaction-count mbarriers; thread 32 issues them after each block
// barrier, beside thread 0's MMAs, and a buffer is refilled once the MMAs
// that read it have committed.  The arithmetic and the phases are those above.
// ---------------------------------------------------------------------------
namespace ts {

template <int K2, int P>
struct Big {
  // K-halves per tap: with TF32x3 the two A slots of a whole tap would not
  // leave room beside X and Y (K2 = 128) or would hold the SM's tensor memory
  // for one CTA alone (K2 = 64); in halves two CTAs fit per SM at K2 = 64
  static constexpr int NH = (P == 1 && K2 >= 64) ? 2 : 1;
  static constexpr int KU = K2 / NH;                          // K of one stage
  static constexpr int AW = P ? 2 * KU : KU / 2;              // TMEM columns per A slot
  static constexpr int NEED = 2 * K2 + 2 * AW;
  static constexpr int COLS = NEED <= 128 ? 128 : NEED <= 256 ? 256 : 512;
  static constexpr int PER_SM = 512 / COLS;                   // CTAs per SM
  static_assert(NEED <= COLS, "TMEM");
  static constexpr int SUB = KU * K2 * (P ? 4 : 2);           // bytes of one K-half (hi or bf16)
  static constexpr int UNIT = P ? 2 * SUB : SUB;              // bytes of one streamed unit
  static constexpr int MATB = P ? 2 * K2 * K2 * 4 : K2 * K2 * 2;
  static constexpr int RB = (PER_SM == 1 ? 192 * 1024 : 96 * 1024) / UNIT;   // ring buffers
  static constexpr int THREADS = 256;
  static constexpr int CPT = KU / 32;                         // 16-column chunks per thread per stage
  static_assert(RB >= 2 && CPT >= 1, "ring and stage shapes");
};

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(dst), "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// The MMAs of one streamed unit: D (+)= A B^T over the unit's K range, A in
// TMEM at a (hi at a, lo at a + KU for TF32x3), B at b in shared memory.
template <int K2, int P>
__device__ __forceinline__ void gemm_unit(uint32_t d, uint32_t a, uint32_t b, bool accumulate) {
  using B = Big<K2, P>;
  constexpr uint32_t lbo = K2 * 16;
  constexpr uint64_t kstep = (2 * lbo) >> 4;
  if constexpr (P == 0) {
    constexpr uint32_t idesc = tc::make_idesc(M, K2);
    const uint64_t b0 = tc::make_desc(b, lbo, 128);
#pragma unroll
    for (int s = 0; s < B::KU / 16; ++s)
      tc::mma_bf16_ts(d, a + 8 * s, b0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
  } else {
    constexpr uint32_t idesc = tc::make_idesc_tf32(M, K2);
    const uint64_t bh0 = tc::make_desc(b, lbo, 128);
    const uint64_t bl0 = bh0 + (B::SUB >> 4);
#pragma unroll
    for (int s = 0; s < B::KU / 8; ++s) {
      const uint32_t ahi = a + 8 * s, alo = a + B::KU + 8 * s;
      tc::mma_tf32_ts(d, alo, bh0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
      tc::mma_tf32_ts(d, ahi, bl0 + s * kstep, idesc, 1u);
      tc::mma_tf32_ts(d, ahi, bh0 + s * kstep, idesc, 1u);
    }
  }
}

}  // namespace ts

template <int K2, int D, int P, int MODE>
__global__ void __launch_bounds__(256, ts::Big<K2, P>::PER_SM) k_smooth_tsb(TsParams p) {
  using B = ts::Big<K2, P>;
  constexpr int C = K2 / 2;
  constexpr int NT = 2 * D + 1;
  constexpr int NH = B::NH, KU = B::KU, RB = B::RB, CPT = B::CPT;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t abar[2];        // A slot s free again (its MMAs done)
  __shared__ uint64_t pbar;           // the MMAs of an epilogue phase done
  __shared__ uint64_t fullb[RB];      // unit landed in ring buffer b
  __shared__ uint64_t emptyb[RB];     // MMAs reading ring buffer b done
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lanei = tid & 31;
  const int row = 32 * (warp & 3) + lanei;
  const int grp = warp >> 2;          // owns chunks q with q % 2 == grp
  const bool has_e = p.e_in != nullptr;
  const int UPT = has_e ? (NT + 1) * NH + (MODE == 0 ? 2 * NH : 0) : 2 * NH;   // units per tile

  if (tid == 0) {
    tc::bar_init(&abar[0], 1);
    tc::bar_init(&abar[1], 1);
    tc::bar_init(&pbar, 1);
    for (int b = 0; b < RB; ++b) {
      tc::bar_init(&fullb[b], 1);
      tc::bar_init(&emptyb[b], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)B::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t lane = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t tX = tmem, tY = tmem + K2;
  const uint32_t slot0 = tmem + 2 * K2, slot1 = slot0 + B::AW;
  const uint32_t ring_s = tc::smem_u32(smem);
  uint32_t aph[2] = {0, 0}, pph = 0;
  bool ok = true;
  auto wait_a = [&](int s) {
    ok = tc::bar_wait(&abar[s], aph[s], p.err) && ok;
    aph[s] ^= 1;
  };
  auto wait_p = [&]() {
    ok = tc::bar_wait(&pbar, pph, p.err) && ok;
    pph ^= 1;
  };
  const int my_tiles = blockIdx.x < p.items ? (p.items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // ---- the weight stream (thread 0): units in order, RB - 1 ahead
  const int u_total = my_tiles * UPT;
  int u_issued = 0, u_done = 0, ui_idx = 0;   // ui_idx: index of the next issue within its tile
  auto unit_of = [&](int idx, int& m, int& h) {
    if (!has_e) {
      m = idx < NH ? NT + 1 : NT + 2;
      h = idx < NH ? idx : idx - NH;
      return;
    }
    if (idx < 2 * NH) {                 // tap 0 with K_A, per K-half
      m = (idx & 1) ? NT : 0;
      h = idx >> 1;
      return;
    }
    const int r = idx - 2 * NH;
    if (r < (NT - 1) * NH) {
      m = 1 + r / NH;
      h = r % NH;
      return;
    }
    const int r2 = r - (NT - 1) * NH;
    m = r2 < NH ? NT + 1 : NT + 2;
    h = r2 < NH ? r2 : r2 - NH;
  };
  auto issue_unit = [&]() {            // thread 0
    const int b = u_issued % RB;
    if (u_issued >= RB) {              // the MMAs of unit u_issued - RB have read buffer b
      ok = tc::bar_wait(&emptyb[b], (uint32_t)(((u_issued / RB) - 1) & 1), p.err) && ok;
    }
    int m, h;
    unit_of(ui_idx, m, h);
    const int gm = m == NT + 2 ? p.wi : m;
    const uint8_t* src = reinterpret_cast<const uint8_t*>(p.mats) + (size_t)gm * B::MATB;
    const uint32_t dst = ring_s + (uint32_t)(b * B::UNIT);
    ts::expect_tx(&fullb[b], (uint32_t)B::UNIT);
    if constexpr (P == 1) {
      ts::bulk_copy(dst, src + (size_t)h * B::SUB, B::SUB, &fullb[b]);
      ts::bulk_copy(dst + B::SUB, src + (size_t)K2 * K2 * 4 + (size_t)h * B::SUB, B::SUB, &fullb[b]);
    } else {
      ts::bulk_copy(dst, src + (size_t)h * B::SUB, B::SUB, &fullb[b]);
    }
    ++u_issued;
    if (++ui_idx == UPT) ui_idx = 0;
  };
  // Thread 32 issues the copies, right after each block barrier, so that
  // thread 0 only waits for weights and issues MMAs.  u_seen counts the
  // units consumed before that barrier; a refill waits for the MMAs of unit
  // u_issued - RB <= u_seen - 2, which thread 0 issued before the barrier.
  int u_seen = 0;
  auto produce = [&](int consumed_now) {   // every thread; only thread 32 acts
    if (tid == 32)
      while (ok && u_issued < u_total && u_issued < u_seen + RB - 1) issue_unit();
    u_seen += consumed_now;
  };
  // MMAs of the next unit (thread 0): A at a, target d
  int u_fail = -1;                     // a unit whose arrival thread 0 gave up on
  auto run_unit = [&](uint32_t d, uint32_t a, bool acc) {
    const int b = u_done % RB;
    if (!tc::bar_wait(&fullb[b], (uint32_t)((u_done / RB) & 1), p.err)) {
      ok = false;
      u_fail = u_done;
    }
    if (ok) {
      tc::fence_after();
      ts::gemm_unit<K2, P>(d, a, ring_s + (uint32_t)(b * B::UNIT), acc);
      tc::mma_commit(&emptyb[b]);
    }
    ++u_done;
  };
  if (tid == 32)
    while (ok && u_issued < u_total && u_issued < RB - 1) issue_unit();

  for (int k = 0; k < my_tiles; ++k) {
    const int item = blockIdx.x + k * gridDim.x;
    const ts::Tile tv = ts::tile_of(p, item, C);
    const float2* r = tv.r;
    const float2* ein = has_e ? tv.e_in : nullptr;
    float2* out = tv.out;
    const long long n = tv.n0 + row;
    const bool row_ok = n < tv.nodes;
    const long long nc = row_ok ? n : tv.nodes - 1;
    int x, y, z;
    node_xyz(nc, tv.nx, tv.ny, x, y, z);
    auto nbr = [&](int j, long long& nb) -> bool {
      if (j == 0) { nb = nc; return row_ok; }
      const int axis = (j - 1) >> 1;
      const int sgn = (j & 1) ? -1 : 1;
      const int c = axis == 0 ? x : (axis == 1 ? y : z);
      const int ext = axis == 0 ? tv.nx : (axis == 1 ? tv.ny : tv.nz);
      const long long stride = axis == 0 ? 1 : (axis == 1 ? tv.nx : (long long)tv.nx * tv.ny);
      nb = nc + sgn * stride;
      return row_ok && c + sgn >= 0 && c + sgn < ext;
    };
    // this thread's chunks of stage (tap j, half h): columns h KU + 32 i + 16 grp
    auto load_stage = [&](float (&v)[CPT * 16], int j, int h) {
      long long nb;
      const bool ok_n = nbr(j, nb);
#pragma unroll
      for (int i = 0; i < CPT; ++i) {
        const int c0 = h * KU + 32 * i + 16 * grp;
        const float4* q = reinterpret_cast<const float4*>(ein + nb * C + c0 / 2);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float4 w = ok_n ? __ldg(q + t) : make_float4(0.f, 0.f, 0.f, 0.f);
          v[16 * i + 4 * t] = w.x;
          v[16 * i + 4 * t + 1] = w.y;
          v[16 * i + 4 * t + 2] = w.z;
          v[16 * i + 4 * t + 3] = w.w;
        }
      }
    };
    // 16 columns at absolute column c of an epilogue operand -> its A slot
    auto put_abs = [&](bool second, int c, const float* v) {
      const int h = c / KU;
      const uint32_t slot = NH == 2 ? (h ? slot1 : slot0) : (second ? slot1 : slot0);
      if constexpr (P == 1) {
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          hi[i] = tc::to_tf32(v[i]);
          lo[i] = tc::to_tf32(v[i] - __uint_as_float(hi[i]));
        }
        tc::tmem_st16(slot + lane + (c - h * KU), hi);
        tc::tmem_st16(slot + lane + KU + (c - h * KU), lo);
      } else {
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) pk[i] = tc::pack_bf16(v[2 * i], v[2 * i + 1]);
        tc::tmem_st8(slot + lane + (c - h * KU) / 2, pk);
      }
    };

    if (has_e) {
      // ---- phase 1: stages q = (tap j, half h)
      constexpr int Q = NT * NH;
      float va[CPT * 16], vb[CPT * 16];
      load_stage(va, 0, 0);
      load_stage(vb, (1 / NH), 1 % NH);
      // two stages per iteration, so that each register buffer is named
      // statically and its loads stay in flight until the buffer is used
      auto stage = [&](int q, float (&cur)[CPT * 16], uint32_t slot) -> bool {
        const int j = q / NH, h = q % NH;
        if (q >= 2) wait_a(q & 1);                 // MMAs of stage q-2 have read this slot
#pragma unroll
        for (int i = 0; i < CPT; ++i) ts::put16<KU, P>(slot + lane, 32 * i + 16 * grp, cur + 16 * i);
        tc::tmem_st_wait();
        if (q + 2 < Q) load_stage(cur, (q + 2) / NH, (q + 2) % NH);
        tc::fence_before();
        ok = __syncthreads_and(ok);
        if (!ok) return false;
        produce(j == 0 ? 2 : 1);
        if (tid == 0) {
          tc::fence_after();
          run_unit(tX, slot, q > 0);
          if (j == 0) run_unit(tY, slot, h > 0);
          tc::mma_commit(&abar[q & 1]);
        }
        return true;
      };
      {
        int q = 0;
        for (; q + 1 < Q; q += 2) {
          if (!stage(q, va, slot0)) goto fail;
          if (!stage(q + 1, vb, slot1)) goto fail;
        }
        if (q < Q && !stage(q, va, slot0)) goto fail;
      }
      wait_a(Q >= 2 ? ((Q - 2) & 1) : 0);
      wait_a((Q - 1) & 1);
      tc::fence_after();
      // ---- epilogue 1: t = r - X - a (.) Y
#pragma unroll
      for (int i = 0; i < K2 / 32; ++i) {
        const int c0 = 32 * i + 16 * grp;
        float xv[16], yv[16], rv[16], av[16], t[16];
        tc::tmem_ld16(tX + lane + c0, xv);
        tc::tmem_ld16(tY + lane + c0, yv);
        ts::load16(rv, r, C, nc, c0);
        ts::load16(av, tv.a, C, nc, c0);
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) {
          t[2 * qq] = rv[2 * qq] - xv[2 * qq] - (av[2 * qq] * yv[2 * qq] - av[2 * qq + 1] * yv[2 * qq + 1]);
          t[2 * qq + 1] = rv[2 * qq + 1] - xv[2 * qq + 1] -
                          (av[2 * qq] * yv[2 * qq + 1] + av[2 * qq + 1] * yv[2 * qq]);
        }
        if constexpr (MODE == 1) {
          if (row_ok) ts::store16(out, C, n, c0, t);
        } else {
          if (!row_ok) {
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) t[qq] = 0.f;
          }
          put_abs(false, c0, t);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < K2 / 32; ++i) {
        const int c0 = 32 * i + 16 * grp;
        float rv[16];
        ts::load16(rv, r, C, nc, c0);
        if (!row_ok) {
#pragma unroll
          for (int qq = 0; qq < 16; ++qq) rv[qq] = 0.f;
        }
        put_abs(false, c0, rv);
      }
    }

    if constexpr (MODE == 0) {
      // ---- phase 2: Z = T K~_S^T; epilogue 2: z = s (.) Z
      tc::tmem_st_wait();
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) goto fail;
      produce(NH);
      if (tid == 0) {
        tc::fence_after();
        for (int h = 0; h < NH; ++h) run_unit(tX, (NH == 2 && h) ? slot1 : slot0, h > 0);
        tc::mma_commit(&pbar);
      }
      wait_p();
      tc::fence_after();
#pragma unroll
      for (int i = 0; i < K2 / 32; ++i) {
        const int c0 = 32 * i + 16 * grp;
        float zv[16], sv[16], zz[16];
        tc::tmem_ld16(tX + lane + c0, zv);
        ts::load16(sv, tv.s, C, nc, c0);
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) {
          zz[2 * qq] = sv[2 * qq] * zv[2 * qq] - sv[2 * qq + 1] * zv[2 * qq + 1];
          zz[2 * qq + 1] = sv[2 * qq] * zv[2 * qq + 1] + sv[2 * qq + 1] * zv[2 * qq];
        }
        if (!row_ok) {
#pragma unroll
          for (int qq = 0; qq < 16; ++qq) zz[qq] = 0.f;
        }
        put_abs(true, c0, zz);
      }
      // ---- phase 3: U = Z W~_i^T; epilogue 3: e' = e + U
      tc::tmem_st_wait();
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) goto fail;
      produce(NH);
      if (tid == 0) {
        tc::fence_after();
        for (int h = 0; h < NH; ++h) run_unit(tY, NH == 2 ? (h ? slot1 : slot0) : slot1, h > 0);
        tc::mma_commit(&pbar);
      }
      wait_p();
      tc::fence_after();
#pragma unroll
      for (int i = 0; i < K2 / 32; ++i) {
        const int c0 = 32 * i + 16 * grp;
        float uv[16];
        tc::tmem_ld16(tY + lane + c0, uv);
        if (has_e) {
          float ev[16];
          ts::load16(ev, ein, C, nc, c0);
#pragma unroll
          for (int qq = 0; qq < 16; ++qq) uv[qq] += ev[qq];
        }
        if (row_ok) ts::store16(out, C, n, c0, uv);
      }
    }
    tc::fence_before();
  }
  ok = __syncthreads_and(ok);
  if (!ok) goto fail;
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)B::COLS));
  }
  return;

fail:
  // a bounded wait ran out: record it; thread 0 lets its weight copies land
  // and its MMAs finish (bounded), then the tensor memory is released
  if (p.err && tid == 0) atomicOr(p.err, 1);
  if (tid == 32) {                     // copies not consumed yet
    for (int u = u_seen; u < u_issued; ++u)
      tc::bar_wait(&fullb[u % RB], (uint32_t)((u / RB) & 1), nullptr);
  }
  if (tid == 0) {
    if (u_fail >= 0)
      tc::bar_wait(&fullb[u_fail % RB], (uint32_t)((u_fail / RB) & 1), nullptr);
    if (u_done > 0)
      tc::bar_wait(&emptyb[(u_done - 1) % RB], (uint32_t)(((u_done - 1) / RB) & 1), nullptr);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)B::COLS));
  }
}

namespace {

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

template <int K2, int D, int P, int MODE>
mcmg_status tsr_launch(TsParams p, int nrhs, cudaStream_t st) {
  using G = ts::Cfg<K2, P>;
  using RG = ts::Ring<K2, P>;
  constexpr int NT = 2 * D + 1;
  constexpr int NM = MODE == 0 ? NT + 3 : NT + 1;
  auto kern = k_smooth_tsr<K2, D, P, MODE>;
  static size_t smem = 0;
  if (smem == 0) {
    // weights and ring; at most PER_SM CTAs on one SM, so that their TMEM
    // always fits: ask for more than the shared memory PER_SM + 1 blocks share
    const size_t need = (size_t)NM * G::MAT + (size_t)RG::R * RG::SEG;
    size_t guard = (size_t)ts::SM_SMEM / (RG::PER_SM + 1) + 16 - 2 * ts::BLOCK_RESERVED;
    size_t s = need > guard ? need : guard;
    s = (s + 127) & ~(size_t)127;
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s));
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    smem = s;
  }
  static_assert(RG::PER_SM >= 1, "ring does not fit");
  if (!p.fields) {
    p.tiles = (int)((p.nodes + ts::M - 1) / ts::M);
    p.items = p.tiles * nrhs;
  }
  const int grid = std::min(p.items, sm_count() * RG::PER_SM);
  kern<<<grid, ts::THREADS, smem, st>>>(p);
  MCMG_CHECK_LAUNCH("smooth_tsr");
  return MCMG_OK;
}

template <int K2, int D, int P, int MODE>
mcmg_status tsb_launch(TsParams p, int nrhs, cudaStream_t st) {
  using B = ts::Big<K2, P>;
  auto kern = k_smooth_tsb<K2, D, P, MODE>;
  static bool attr = false;
  const size_t smem = (size_t)B::RB * B::UNIT;
  if (!attr) {
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  if (!p.fields) {
    p.tiles = (int)((p.nodes + ts::M - 1) / ts::M);
    p.items = p.tiles * nrhs;
  }
  const int grid = std::min(p.items, sm_count() * B::PER_SM);
  kern<<<grid, B::THREADS, smem, st>>>(p);
  MCMG_CHECK_LAUNCH("smooth_tsb");
  return MCMG_OK;
}

template <int K2, int D, int P, int MODE>
mcmg_status ts_launch(TsParams p, int nrhs, cudaStream_t st) {
  using G = ts::Cfg<K2, P>;
  constexpr int NT = 2 * D + 1;
  constexpr int NM = MODE == 0 ? NT + 3 : NT + 1;
  auto kern = k_smooth_ts<K2, D, P, MODE>;
  static size_t smem = 0;
  static int per_sm = 0;
  if (smem == 0) {
    // at most PER_SM CTAs on one SM, so that their TMEM always fits: ask for
    // more than the shared memory PER_SM + 1 blocks could share
    const size_t need = (size_t)NM * G::MAT;
    size_t guard = (size_t)ts::SM_SMEM / (G::PER_SM + 1) + 16 - ts::BLOCK_RESERVED;
    size_t s = need > guard ? need : guard;
    s = (s + 127) & ~(size_t)127;
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s));
    // the whole shared-memory carveout, so that exactly PER_SM such blocks fit
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    smem = s;
    per_sm = G::PER_SM;
  }
  if (!p.fields) {
    p.tiles = (int)((p.nodes + ts::M - 1) / ts::M);
    p.items = p.tiles * nrhs;
  }
  const int grid = std::min(p.items, sm_count() * per_sm);
  kern<<<grid, ts::THREADS, smem, st>>>(p);
  MCMG_CHECK_LAUNCH("smooth_ts");
  return MCMG_OK;
}

template <int D, int P, int MODE>
mcmg_status ts_dispatch(int C, const TsParams& p, int nrhs, cudaStream_t st) {
  switch (C) {
    // measured per shape: the ring wins for BF16 at C = 16 only
    case 8: return ts_launch<16, D, P, MODE>(p, nrhs, st);
    case 16:
      if constexpr (P == 0) return tsr_launch<32, D, P, MODE>(p, nrhs, st);
      else return ts_launch<32, D, P, MODE>(p, nrhs, st);
    case 32:
      if constexpr (P == 0) return ts_launch<64, D, P, MODE>(p, nrhs, st);
      else return tsb_launch<64, D, P, MODE>(p, nrhs, st);
    case 64: return tsb_launch<128, D, P, MODE>(p, nrhs, st);
    default: break;
  }
  set_error("tensor-core step: no variant for C = %d", C);
  return MCMG_ERR_SHAPE;
}

}  // namespace

bool ts_supported(int C, int prec) {
  if (prec == MCMG_BF16 || prec == MCMG_FP32_TC) return C == 8 || C == 16 || C == 32 || C == 64;
  return false;
}

mcmg_status launch_smooth_ts(const Level& L, int step, const float2* r, const float2* e_in,
                             float2* out, int mode, int nrhs, cudaStream_t st) {
  if (mode == 1 && !e_in) {
    set_error("tensor-core residual needs e");
    return MCMG_ERR_ARG;
  }
  TsParams p{};
  p.r = r;
  p.e_in = e_in;
  p.out = out;
  p.a = L.a;
  p.s = L.s;
  p.mats = L.ts_mats;
  p.wi = 2 * L.g.d + 1 + 2 + step;
  p.nx = L.g.nx;
  p.ny = L.g.ny;
  p.nz = L.g.nz;
  p.nodes = L.g.nodes();
  p.err = L.err;
  const bool d3 = L.g.d == 3;
  const bool tf = L.ts_prec == MCMG_FP32_TC;
  if (mode == 0) {
    if (tf) return d3 ? ts_dispatch<3, 1, 0>(L.C, p, nrhs, st) : ts_dispatch<2, 1, 0>(L.C, p, nrhs, st);
    return d3 ? ts_dispatch<3, 0, 0>(L.C, p, nrhs, st) : ts_dispatch<2, 0, 0>(L.C, p, nrhs, st);
  }
  if (tf) return d3 ? ts_dispatch<3, 1, 1>(L.C, p, nrhs, st) : ts_dispatch<2, 1, 1>(L.C, p, nrhs, st);
  return d3 ? ts_dispatch<3, 0, 1>(L.C, p, nrhs, st) : ts_dispatch<2, 0, 1>(L.C, p, nrhs, st);
}

bool ts_fused_io_supported(const Level& L) {
  // the levels whose step runs k_smooth_ts (one thread per row, all channels)
  return L.use_ts && (L.C == 8 || (L.C == 16 && L.ts_prec == MCMG_FP32_TC));
}

mcmg_status launch_smooth_ts_io(const Level& L, int step, const float2* const* r_cell,
                                const float2* lift, const float2* e_in, float2* out,
                                float2* const* z_cell, const float2* proj, int mode,
                                cudaStream_t st) {
  if (!ts_fused_io_supported(L) || (mode == 1 && !e_in) || (mode == 1 && z_cell)) {
    set_error("fused lift / projection not available on this level");
    return MCMG_ERR_ARG;
  }
  TsParams p{};
  p.r_cell = r_cell;
  p.lift = lift;
  p.z_cell = z_cell;
  p.proj = proj;
  p.e_in = e_in;
  p.out = out;
  p.a = L.a;
  p.s = L.s;
  p.mats = L.ts_mats;
  p.wi = 2 * L.g.d + 1 + 2 + step;
  p.nx = L.g.nx;
  p.ny = L.g.ny;
  p.nz = L.g.nz;
  p.nodes = L.g.nodes();
  p.err = L.err;
  const bool d3 = L.g.d == 3;
  const bool tf = L.ts_prec == MCMG_FP32_TC;
  if (mode == 0) {
    if (tf) return d3 ? ts_dispatch<3, 1, 0>(L.C, p, 1, st) : ts_dispatch<2, 1, 0>(L.C, p, 1, st);
    return d3 ? ts_dispatch<3, 0, 0>(L.C, p, 1, st) : ts_dispatch<2, 0, 0>(L.C, p, 1, st);
  }
  if (tf) return d3 ? ts_dispatch<3, 1, 1>(L.C, p, 1, st) : ts_dispatch<2, 1, 1>(L.C, p, 1, st);
  return d3 ? ts_dispatch<3, 0, 1>(L.C, p, 1, st) : ts_dispatch<2, 0, 1>(L.C, p, 1, st);
}

mcmg_status launch_smooth_ts_fields(const Level& L, int step, const TsField* fields_dev,
                                    const TsField* fields_host, int nf, bool has_e, int mode,
                                    cudaStream_t st) {
  if (nf < 1) return MCMG_OK;
  if (mode == 1 && !has_e) {
    set_error("tensor-core residual needs e");
    return MCMG_ERR_ARG;
  }
  TsParams p{};
  p.fields = fields_dev;
  p.nfields = nf;
  p.items = fields_host[nf - 1].first + fields_host[nf - 1].tiles;
  // e_in only marks whether the fields carry e (the descriptors hold the pointers)
  p.e_in = has_e ? fields_host[0].e_in : nullptr;
  p.mats = L.ts_mats;
  p.wi = 2 * L.g.d + 1 + 2 + step;
  p.err = L.err;
  const bool d3 = L.g.d == 3;
  const bool tf = L.ts_prec == MCMG_FP32_TC;
  if (mode == 0) {
    if (tf) return d3 ? ts_dispatch<3, 1, 0>(L.C, p, 1, st) : ts_dispatch<2, 1, 0>(L.C, p, 1, st);
    return d3 ? ts_dispatch<3, 0, 0>(L.C, p, 1, st) : ts_dispatch<2, 0, 0>(L.C, p, 1, st);
  }
  if (tf) return d3 ? ts_dispatch<3, 1, 1>(L.C, p, 1, st) : ts_dispatch<2, 1, 1>(L.C, p, 1, st);
  return d3 ? ts_dispatch<3, 0, 1>(L.C, p, 1, st) : ts_dispatch<2, 0, 1>(L.C, p, 1, st);
}

// Host: a complex C x C matrix M[co][ci] (float2, row-major) -> its real
// 2C x 2C block form as BF16 in the no-swizzle K-major core-matrix layout of
// a B operand (row n = output index, K = input index, 16-byte chunks of 8
// elements, chunk-major).
void pack_ts_bf16(const float2* Mc, int C, uint16_t* out) {
  const int K2 = 2 * C;
  for (int n = 0; n < K2; ++n)
    for (int k = 0; k < K2; ++k) {
      const float2 m = Mc[(size_t)(n >> 1) * C + (k >> 1)];
      float v;
      if ((n & 1) == 0) v = (k & 1) == 0 ? m.x : -m.y;   // re out: Mr re_in - Mi im_in
      else v = (k & 1) == 0 ? m.y : m.x;                 // im out: Mi re_in + Mr im_in
      __nv_bfloat16 b = __float2bfloat16_rn(v);
      const size_t pos = ((size_t)(k >> 3) * K2 + n) * 8 + (k & 7);
      std::memcpy(out + pos, &b, 2);
    }
}

// Host: FP32 -> TF32 bit pattern, round to nearest, ties away from zero
// (the same rounding as the device's cvt.rna.tf32.f32 on finite values).
static float host_tf32(float v) {
  uint32_t b;
  std::memcpy(&b, &v, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &b, 4);
  return r;
}

// Host: a complex C x C matrix M[co][ci] (float2, row-major) -> its real
// 2C x 2C block form as TF32 hi and lo halves, each in the no-swizzle K-major
// core-matrix layout of a B operand (row n = output index, K = input index,
// 16-byte chunks of 4 elements, chunk-major).
void pack_ts_tf32(const float2* Mc, int C, float* out) {
  const int K2 = 2 * C;
  float* hi = out;
  float* lo = out + (size_t)K2 * K2;
  for (int n = 0; n < K2; ++n)
    for (int k = 0; k < K2; ++k) {
      const float2 m = Mc[(size_t)(n >> 1) * C + (k >> 1)];
      float v;
      if ((n & 1) == 0) v = (k & 1) == 0 ? m.x : -m.y;
      else v = (k & 1) == 0 ? m.y : m.x;
      const float h = host_tf32(v);
      const size_t pos = ((size_t)(k >> 2) * K2 + n) * 4 + (k & 3);
      hi[pos] = h;
      lo[pos] = host_tf32(v - h);
    }
}

}  // namespace mcmg
