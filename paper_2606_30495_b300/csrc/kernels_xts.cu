// Restriction and prolongation of the McMg V-cycle (Section 3.2, Algorithm 2)
// on the tcgen05 tensor cores, for levels whose input side has at least 16
// channels (BF16 or FP32-accurate 3xTF32 operands, FP32 accumulation).
//
// Both are sums over 3^d taps of a complex channel-mixing matrix applied to
// a gathered row, i.e. GEMMs over tiles of M = 128 output nodes with
// K = 2 C_in, N = 2 C_out in real block form:
//
//   restriction   r_c[J]  = sum_o R_o x[2J + o]                (27 / 9 taps)
//   prolongation  e[2j+p] += sum_{(J, o): 2J + o = 2j + p} P_o e_c[J]
//
// The prolongation is taken output by output: a tile holds 128 fine nodes of
// one parity class p (fine node 2j + p for 128 consecutive j of the coarse
// lattice), whose taps are fixed: per axis one (J = j, o = 0) when p_a = 0,
// two (J = j, o = +1) and (J = j + 1, o = -1) when p_a = 1.
//
// The structure is that of the streamed-weight smoothing step (kernels_ts.cu):
// 256 threads, thread t owning row 32 (w % 4) + lane of warp w and every
// other 16-column chunk of it; each (tap, K-part) is one A stage gathered
// into registers two stages ahead (two stages per loop iteration, so that
// both register buffers are named statically), converted and written to one
// of two A slots in tensor memory; the weight matrices stream per (tap,
// K-part) unit through a ring of shared-memory buffers filled by bulk
// asynchronous copies that thread 32 issues; thread 0 issues the MMAs.  Each
// tap accumulates apart and the tap partials are summed in FP32 registers;
// the epilogue stores the sum (restriction) or adds it to the fine field
// (prolongation).  Every mbarrier wait is bounded and the block votes on the
// outcome at its next barrier.
//
// Further below: the prolongation in block form (all parity classes of a
// coarse tile in one MMA group) and the restriction from 8 channels with the
// fine lines staged in shared memory.
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "mcmg_internal.cuh"
#include "tcgen05.cuh"
#include "vcycle_kernels.cuh"

namespace mcmg {

namespace xts {

constexpr int M = 128;
constexpr int THREADS = 256;

template <int KI, int KO, int P>  // P: 0 BF16, 1 TF32x3
struct Cfg {
  // A stages of 32 K values (one 16-column chunk per thread)
  static constexpr int KU = 32;
  static constexpr int NH = KI / KU;                          // K parts per tap
  static constexpr int AW = P ? 2 * KU : KU / 2;              // A slot columns
  // two accumulators (taps alternate) and two A slots
  static constexpr int NEED = 2 * KO + 2 * AW;
  static constexpr int COLS = NEED <= 256 ? 256 : 512;
  static constexpr int PER_SM = 512 / COLS;
  static constexpr int SUB = KU * KO * (P ? 4 : 2);           // one K part of one matrix (hi or bf16)
  static constexpr int UNIT = P ? 2 * SUB : SUB;
  static constexpr int MATB = P ? 2 * KO * KI * 4 : KO * KI * 2;
  static constexpr int RING = PER_SM == 1 ? 192 * 1024 : 96 * 1024;
  static constexpr int RB = RING / UNIT;
  static constexpr int NCH = (KO + 31) / 32;                  // output chunks per thread
  static_assert(KI % KU == 0 && RB >= 2 && NEED <= COLS, "transfer shape");
};

// K of one stage's weight matrix: a tap's 2 C_in, or two taps' for the
// restriction from 8 channels
__host__ __device__ constexpr int stage_k(int ki, int dir) { return dir == 0 && ki == 16 ? 32 : ki; }

struct XParams {
  const float2* src;      // restriction: fine x; prolongation: coarse e_c
  float2* dst;            // restriction: coarse r_c (written); prolongation: fine e (+=)
  const uint4* mats;      // [3^d taps] matrices in the operand layout, MATB bytes each
  int fx, fy, fz;         // fine grid
  int cx, cy, cz;         // coarse grid
  long long src_nodes, dst_nodes;   // per field
  int tiles;              // coarse-lattice tiles per field (per parity class)
  int items;
  int* err;
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

// 16 FP32 values -> A slot columns c0 .. c0+15 (TF32 hi at c0, lo at KU + c0;
// or 8 packed BF16 pairs at c0 / 2)
template <int KU, int P>
__device__ __forceinline__ void put16(uint32_t slot, int c0, const float* v) {
  if constexpr (P == 1) {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      hi[i] = tc::to_tf32(v[i]);
      lo[i] = tc::to_tf32(v[i] - __uint_as_float(hi[i]));
    }
    tc::tmem_st16(slot + c0, hi);
    tc::tmem_st16(slot + KU + c0, lo);
  } else {
    uint32_t pk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) pk[i] = tc::pack_bf16(v[2 * i], v[2 * i + 1]);
    tc::tmem_st8(slot + c0 / 2, pk);
  }
}

// The MMAs of one streamed unit: D (+)= A B^T over the unit's K range.
template <int KI, int KO, int P>
__device__ __forceinline__ void gemm_unit(uint32_t d, uint32_t a, uint32_t b, bool accumulate) {
  using G = Cfg<KI, KO, P>;
  constexpr uint32_t lbo = KO * 16;       // B rows are the KO outputs
  constexpr uint64_t kstep = (2 * lbo) >> 4;
  if constexpr (P == 0) {
    constexpr uint32_t idesc = tc::make_idesc(M, KO);
    const uint64_t b0 = tc::make_desc(b, lbo, 128);
#pragma unroll
    for (int s = 0; s < G::KU / 16; ++s)
      tc::mma_bf16_ts(d, a + 8 * s, b0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
  } else {
    constexpr uint32_t idesc = tc::make_idesc_tf32(M, KO);
    const uint64_t bh0 = tc::make_desc(b, lbo, 128);
    const uint64_t bl0 = bh0 + (G::SUB >> 4);
#pragma unroll
    for (int s = 0; s < G::KU / 8; ++s) {
      const uint32_t ahi = a + 8 * s, alo = a + G::KU + 8 * s;
      tc::mma_tf32_ts(d, alo, bh0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
      tc::mma_tf32_ts(d, ahi, bl0 + s * kstep, idesc, 1u);
      tc::mma_tf32_ts(d, ahi, bh0 + s * kstep, idesc, 1u);
    }
  }
}

// Tap `idx` of an item: its weight index t (taps ((oz+1)*3+(oy+1))*3+(ox+1))
// and the gather offsets.  Restriction: idx enumerates the 3^D offsets o and
// the gathered fine node is 2J + o.  Prolongation of parity class p: the
// odd axes of p take o = +1 (source J = j) or o = -1 (J = j + 1) by the bits
// of idx; even axes take o = 0.
template <int D, int DIR>
__device__ __forceinline__ void tap_of(int cls, int idx, int& t, int (&o)[3], int (&dj)[3]) {
  if constexpr (DIR == 0) {
    int r = idx;
    o[0] = r % 3 - 1;
    r /= 3;
    o[1] = r % 3 - 1;
    r /= 3;
    o[2] = D == 3 ? r - 1 : 0;
    dj[0] = dj[1] = dj[2] = 0;
  } else {
    int bit = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dj[a] = 0;
      o[a] = 0;
      if (a < D && ((cls >> a) & 1)) {
        const bool minus = (idx >> bit) & 1;
        ++bit;
        o[a] = minus ? -1 : 1;
        dj[a] = minus ? 1 : 0;
      }
    }
  }
  t = D == 3 ? ((o[2] + 1) * 3 + (o[1] + 1)) * 3 + (o[0] + 1) : (o[1] + 1) * 3 + (o[0] + 1);
}

template <int D>
__host__ __device__ constexpr int popc_cls(int cls) {
  return (cls & 1) + ((cls >> 1) & 1) + (D == 3 ? ((cls >> 2) & 1) : 0);
}

}  // namespace xts

template <int KI, int KO, int D, int P, int DIR>
__global__ void __launch_bounds__(xts::THREADS, xts::Cfg<xts::stage_k(KI, DIR), KO, P>::PER_SM)
    k_transfer_ts(xts::XParams p) {
  // restriction from 8 channels: two taps per stage, each thread group (grp)
  // gathering the 16 floats of one of the two fine rows, against the pair's
  // matrices concatenated along K (KI = 16 per tap, 32 per stage)
  constexpr bool PAIR = DIR == 0 && KI == 16;
  constexpr int KIE = xts::stage_k(KI, DIR);       // K of one stage's weights
  using G = xts::Cfg<KIE, KO, P>;
  constexpr int CI = KI / 2, CO = KO / 2;
  constexpr int NH = G::NH, KU = G::KU, RB = G::RB, NCH = G::NCH;
  constexpr int T3 = D == 3 ? 27 : 9;
  constexpr int NCLS = DIR == 1 ? (1 << D) : 1;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t abar[2];
  __shared__ uint64_t fullb[RB];
  __shared__ uint64_t emptyb[RB];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lanei = tid & 31;
  const int row = 32 * (warp & 3) + lanei;
  const int grp = warp >> 2;

  if (tid == 0) {
    tc::bar_init(&abar[0], 1);
    tc::bar_init(&abar[1], 1);
    for (int b = 0; b < RB; ++b) {
      tc::bar_init(&fullb[b], 1);
      tc::bar_init(&emptyb[b], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)G::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t lane = (uint32_t)(32 * (warp & 3)) << 16;
  // accumulators: tap t into column tmem + (t & 1) KO; A slots after them
  const uint32_t slot0 = tmem + 2 * KO, slot1 = slot0 + G::AW;
  const uint32_t ring_s = tc::smem_u32(smem);
  uint32_t aph[2] = {0, 0};
  bool ok = true;
  auto wait_a = [&](int s) {
    ok = tc::bar_wait(&abar[s], aph[s], p.err) && ok;
    aph[s] ^= 1;
  };
  const int my_items = blockIdx.x < p.items ? (p.items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // taps of an item: all 3^D for the restriction, 2^(odd axes) for a class
  auto item_class = [&](int item) -> int {
    if constexpr (DIR == 0) return 0;
    else return (item / p.tiles) % NCLS;
  };
  auto item_taps = [&](int item) -> int {
    if constexpr (DIR == 0) return PAIR ? (T3 + 1) / 2 : T3;
    else return 1 << xts::popc_cls<D>(item_class(item));
  };
  // ---- weight stream (thread 0): units (tap, K part) of every item in order
  int u_issued = 0, u_done = 0;
  int ui_k = 0, ui_idx = 0;           // next unit: item of this CTA, unit within it
  int u_left = 0;                     // units of this CTA not yet issued
  for (int k = 0; k < my_items; ++k) u_left += item_taps(blockIdx.x + k * gridDim.x) * NH;
  const int u_total = u_left;
  auto issue_unit = [&]() {
    const int b = u_issued % RB;
    if (u_issued >= RB)
      ok = tc::bar_wait(&emptyb[b], (uint32_t)(((u_issued / RB) - 1) & 1), p.err) && ok;
    const int item = blockIdx.x + ui_k * gridDim.x;
    const int tap = ui_idx / NH, h = ui_idx % NH;
    int t = tap, o[3], dj[3];
    if constexpr (!PAIR) xts::tap_of<D, DIR>(item_class(item), tap, t, o, dj);
    const uint8_t* src = reinterpret_cast<const uint8_t*>(p.mats) + (size_t)t * G::MATB;
    const uint32_t dst = ring_s + (uint32_t)(b * G::UNIT);
    xts::expect_tx(&fullb[b], (uint32_t)G::UNIT);
    xts::bulk_copy(dst, src + (size_t)h * G::SUB, G::SUB, &fullb[b]);
    if constexpr (P == 1)
      xts::bulk_copy(dst + G::SUB, src + (size_t)KO * KIE * 4 + (size_t)h * G::SUB, G::SUB,
                     &fullb[b]);
    ++u_issued;
    if (++ui_idx == item_taps(item) * NH) { ui_idx = 0; ++ui_k; }
  };
  // thread 32 issues the copies after each block barrier (one unit per
  // stage); u_seen counts the units consumed before that barrier, and a
  // refill waits for the MMAs of unit u_issued - RB <= u_seen - 2, which
  // thread 0 issued before the barrier
  int u_seen = 0;
  auto produce = [&]() {               // every thread; only thread 32 acts
    if (tid == 32)
      while (ok && u_issued < u_total && u_issued < u_seen + RB - 1) issue_unit();
    ++u_seen;
  };
  int u_fail = -1;                     // a unit whose arrival thread 0 gave up on
  auto run_unit = [&](uint32_t d, uint32_t a, bool acc) {   // thread 0
    const int b = u_done % RB;
    if (!tc::bar_wait(&fullb[b], (uint32_t)((u_done / RB) & 1), p.err)) {
      ok = false;
      u_fail = u_done;
    }
    if (ok) {
      tc::fence_after();
      xts::gemm_unit<KIE, KO, P>(d, a, ring_s + (uint32_t)(b * G::UNIT), acc);
      tc::mma_commit(&emptyb[b]);
    }
    ++u_done;
  };
  if (tid == 32)
    while (ok && u_issued < u_total && u_issued < RB - 1) issue_unit();

  for (int k = 0; k < my_items; ++k) {
    const int item = blockIdx.x + k * gridDim.x;
    const int per_field = p.tiles * NCLS;
    const int field = item / per_field;
    const int within = item - field * per_field;
    const int cls = DIR == 1 ? within / p.tiles : 0;
    const int tile = within - cls * p.tiles;
    const float2* src = p.src + (size_t)field * (size_t)p.src_nodes * CI;
    float2* dst = p.dst + (size_t)field * (size_t)p.dst_nodes * CO;
    const long long cnodes = (long long)p.cx * p.cy * p.cz;
    const long long j = (long long)tile * xts::M + row;      // coarse-lattice node of this row
    const bool row_ok = j < cnodes;
    int jx, jy, jz;
    node_xyz(row_ok ? j : 0, p.cx, p.cy, jx, jy, jz);
    // the gathered source row of tap `tap`: fine 2J + o (restriction) or
    // coarse j + dj (prolongation)
    auto source = [&](int tap, long long& s) -> bool {
      int t, o[3], dj[3];
      xts::tap_of<D, DIR>(cls, tap, t, o, dj);
      if constexpr (DIR == 0) {
        const int fxx = 2 * jx + o[0], fyy = 2 * jy + o[1], fzz = 2 * jz + o[2];
        s = ((long long)fzz * p.fy + fyy) * p.fx + fxx;
        return row_ok && fxx >= 0 && fxx < p.fx && fyy >= 0 && fyy < p.fy && fzz >= 0 &&
               fzz < p.fz;
      } else {
        const int cxx = jx + dj[0], cyy = jy + dj[1], czz = jz + dj[2];
        s = ((long long)czz * p.cy + cyy) * p.cx + cxx;
        return row_ok && cxx < p.cx && cyy < p.cy && czz < p.cz;
      }
    };
    auto load_stage = [&](float (&v)[16], int q) {
      long long s = 0;
      const int stap = PAIR ? 2 * q + grp : q / NH;      // PAIR: NH = 1
      const bool ok_n = (!PAIR || stap < T3) && source(stap, s);
      const int c0 = PAIR ? 0 : (q % NH) * KU + 16 * grp;
      const float4* qp = reinterpret_cast<const float4*>(src + s * CI + c0 / 2);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 w = ok_n ? __ldg(qp + u) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * u] = w.x;
        v[4 * u + 1] = w.y;
        v[4 * u + 2] = w.z;
        v[4 * u + 3] = w.w;
      }
    };
    // The tensor cores accumulate in FP32 with truncation, an error that
    // grows with the number of MMAs summed into one accumulator (27 taps x
    // 3 KI / 8 of them would reach ~2e-5).  Each tap therefore sums into an
    // accumulator of its own (taps alternate between two), and the tap
    // partials are added here in FP32 with rounding to nearest.
    float acc[NCH * 16];
#pragma unroll
    for (int i = 0; i < NCH * 16; ++i) acc[i] = 0.f;
    auto fold = [&](int t) {
      const uint32_t dcol = tmem + lane + (uint32_t)((t & 1) * KO);
#pragma unroll
      for (int i = 0; i < NCH; ++i) {
        const int c0 = 32 * i + 16 * grp;
        if (c0 < KO) {
          float dv[16];
          tc::tmem_ld16(dcol + c0, dv);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[16 * i + u] += dv[u];
        }
      }
    };
    const int TAPS = item_taps(item);
    const int Q = TAPS * NH;                // stages of this item (>= 1)
    // two stages per iteration, so that each register buffer is named
    // statically and its loads stay in flight until the buffer is used
    auto stage = [&](int q, float (&cur)[16], uint32_t slot) -> bool {
      const int tap = q / NH, h = q - (q / NH) * NH;
      if (q >= 2) wait_a(q & 1);
      // the MMAs of stage q - 2 and all before it are complete: tap - 2's
      // accumulator is final and is about to be reused by this tap
      if (h == 0 && tap >= 2) {
        tc::fence_after();
        fold(tap - 2);
      }
      xts::put16<KU, P>(slot + lane, 16 * grp, cur);
      tc::tmem_st_wait();
      if (q + 2 < Q) load_stage(cur, q + 2);
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) return false;
      produce();
      if (tid == 0) {
        tc::fence_after();
        run_unit(tmem + (uint32_t)((tap & 1) * KO), slot, h > 0);
        tc::mma_commit(&abar[q & 1]);
      }
      return true;
    };
    float va[16], vb[16];
    load_stage(va, 0);
    if (Q > 1) load_stage(vb, 1);
    {
      int q = 0;
      for (; q + 1 < Q; q += 2) {
        if (!stage(q, va, slot0)) goto fail;
        if (!stage(q + 1, vb, slot1)) goto fail;
      }
      if (q < Q && !stage(q, va, slot0)) goto fail;
    }
    if (Q >= 2) wait_a((Q - 2) & 1);
    wait_a((Q - 1) & 1);
    tc::fence_after();
    if (TAPS >= 2) fold(TAPS - 2);
    fold(TAPS - 1);
    // ---- epilogue: store the sum (restriction) or add it to the fine field
    {
      long long o_row;
      if constexpr (DIR == 0) {
        o_row = j;
      } else {
        const int px = cls & 1, py = (cls >> 1) & 1, pz = D == 3 ? (cls >> 2) & 1 : 0;
        o_row = ((long long)(2 * jz + pz) * p.fy + (2 * jy + py)) * p.fx + (2 * jx + px);
      }
#pragma unroll
      for (int i = 0; i < NCH; ++i) {
        const int c0 = 32 * i + 16 * grp;
        if (c0 < KO && row_ok) {
          float4* op = reinterpret_cast<float4*>(dst + o_row * CO + c0 / 2);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float4 w = make_float4(acc[16 * i + 4 * u], acc[16 * i + 4 * u + 1],
                                   acc[16 * i + 4 * u + 2], acc[16 * i + 4 * u + 3]);
            if constexpr (DIR == 1) {
              const float4 e = op[u];
              w.x += e.x;
              w.y += e.y;
              w.z += e.z;
              w.w += e.w;
            }
            op[u] = w;
          }
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
                 "r"((uint32_t)G::COLS));
  }
}


// ---------------------------------------------------------------------------
// Prolongation in block form: an item is a tile of 128 coarse nodes j and
// all 2^d parity classes of their fine nodes 2j + p.  The stages are the 2^d
// source rows e_c[j + s] (s in {0,1}^d; per K part), and each stage is ONE
// MMA group of N = 2^d x 2C columns: the block of class p holds P_o with
// o = p - 2s per axis (-1, 0 or +1) when s is inside p (s_a <= p_a), zeros
// otherwise.  So the 27 (class, tap) products of a 3D block run as 8 wide
// MMA groups instead of 27 narrow ones, and every source row is gathered
// once instead of once per class.  Each class accumulates 2^d x K/8 x 3 MMAs
// at most (fine for the truncating accumulation, no fold).
// ---------------------------------------------------------------------------
namespace xts {

template <int KI, int KO, int D, int P>
struct BlockCfg {
  static constexpr int NCLS = 1 << D;
  static constexpr int N = NCLS * KO;                         // MMA N: all classes
  static constexpr int KU = 32;
  static constexpr int NH = KI / KU;
  static constexpr int AW = P ? 2 * KU : KU / 2;
  static constexpr int NEED = N + 2 * AW;
  static constexpr int COLS = NEED <= 256 ? 256 : 512;
  static constexpr int PER_SM = 512 / COLS;
  static constexpr int SUB = KU * N * (P ? 4 : 2);
  static constexpr int UNIT = P ? 2 * SUB : SUB;
  static constexpr int MATB = P ? 2 * N * KI * 4 : N * KI * 2;  // one source's stacked matrix
  static constexpr int RB = (PER_SM == 1 ? 192 * 1024 : 96 * 1024) / UNIT;
  static_assert(KI % KU == 0 && N <= 256 && RB >= 3 && NEED <= COLS, "block prolongation shape");
};

// D (+)= A B^T over one unit (KU of K), N output columns
template <int N, int KU, int SUB, int P>
__device__ __forceinline__ void gemm_n(uint32_t d, uint32_t a, uint32_t b, bool accumulate) {
  constexpr uint32_t lbo = N * 16;
  constexpr uint64_t kstep = (2 * lbo) >> 4;
  if constexpr (P == 0) {
    constexpr uint32_t idesc = tc::make_idesc(M, N);
    const uint64_t b0 = tc::make_desc(b, lbo, 128);
#pragma unroll
    for (int s = 0; s < KU / 16; ++s)
      tc::mma_bf16_ts(d, a + 8 * s, b0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
  } else {
    constexpr uint32_t idesc = tc::make_idesc_tf32(M, N);
    const uint64_t bh0 = tc::make_desc(b, lbo, 128);
    const uint64_t bl0 = bh0 + (SUB >> 4);
#pragma unroll
    for (int s = 0; s < KU / 8; ++s) {
      const uint32_t ahi = a + 8 * s, alo = a + KU + 8 * s;
      tc::mma_tf32_ts(d, alo, bh0 + s * kstep, idesc, (accumulate || s > 0) ? 1u : 0u);
      tc::mma_tf32_ts(d, ahi, bl0 + s * kstep, idesc, 1u);
      tc::mma_tf32_ts(d, ahi, bh0 + s * kstep, idesc, 1u);
    }
  }
}

}  // namespace xts

template <int KI, int KO, int D, int P>
__global__ void __launch_bounds__(xts::THREADS, xts::BlockCfg<KI, KO, D, P>::PER_SM)
    k_prolong_block_ts(xts::XParams p) {
  using G = xts::BlockCfg<KI, KO, D, P>;
  constexpr int CI = KI / 2, CO = KO / 2;
  constexpr int NH = G::NH, KU = G::KU, RB = G::RB, NCLS = G::NCLS, N = G::N;
  constexpr int UPI = NCLS * NH;                  // units (= stages) per item
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t abar[2];
  __shared__ uint64_t fullb[RB];
  __shared__ uint64_t emptyb[RB];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lanei = tid & 31;
  const int row = 32 * (warp & 3) + lanei;
  const int grp = warp >> 2;

  if (tid == 0) {
    tc::bar_init(&abar[0], 1);
    tc::bar_init(&abar[1], 1);
    for (int b = 0; b < RB; ++b) {
      tc::bar_init(&fullb[b], 1);
      tc::bar_init(&emptyb[b], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)G::COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t lane = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t tD = tmem, slot0 = tmem + N, slot1 = slot0 + G::AW;
  const uint32_t ring_s = tc::smem_u32(smem);
  uint32_t aph[2] = {0, 0};
  bool ok = true;
  auto wait_a = [&](int s) {
    ok = tc::bar_wait(&abar[s], aph[s], p.err) && ok;
    aph[s] ^= 1;
  };
  const int my_items = blockIdx.x < p.items ? (p.items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // ---- weight stream: unit u of an item = (source u / NH, K part u % NH);
  // thread 32 issues after each block barrier, u_seen = units consumed before it
  const int u_total = my_items * UPI;
  int u_issued = 0, u_done = 0, u_seen = 0, u_fail = -1;
  auto issue_unit = [&]() {
    const int b = u_issued % RB;
    if (u_issued >= RB)
      ok = tc::bar_wait(&emptyb[b], (uint32_t)(((u_issued / RB) - 1) & 1), p.err) && ok;
    const int w = u_issued % UPI, src_i = w / NH, h = w % NH;
    const uint8_t* src = reinterpret_cast<const uint8_t*>(p.mats) + (size_t)src_i * G::MATB;
    const uint32_t dst = ring_s + (uint32_t)(b * G::UNIT);
    xts::expect_tx(&fullb[b], (uint32_t)G::UNIT);
    xts::bulk_copy(dst, src + (size_t)h * G::SUB, G::SUB, &fullb[b]);
    if constexpr (P == 1)
      xts::bulk_copy(dst + G::SUB, src + (size_t)N * KI * 4 + (size_t)h * G::SUB, G::SUB,
                     &fullb[b]);
    ++u_issued;
  };
  auto produce = [&]() {
    if (tid == 32)
      while (ok && u_issued < u_total && u_issued < u_seen + RB - 1) issue_unit();
    ++u_seen;
  };
  auto run_unit = [&](uint32_t a, bool acc) {   // thread 0
    const int b = u_done % RB;
    if (!tc::bar_wait(&fullb[b], (uint32_t)((u_done / RB) & 1), p.err)) {
      ok = false;
      u_fail = u_done;
    }
    if (ok) {
      tc::fence_after();
      xts::gemm_n<N, KU, G::SUB, P>(tD, a, ring_s + (uint32_t)(b * G::UNIT), acc);
      tc::mma_commit(&emptyb[b]);
    }
    ++u_done;
  };
  if (tid == 32)
    while (ok && u_issued < u_total && u_issued < RB - 1) issue_unit();

  const long long cnodes = (long long)p.cx * p.cy * p.cz;
  for (int k = 0; k < my_items; ++k) {
    const int item = blockIdx.x + k * gridDim.x;
    const int field = item / p.tiles;
    const int tile = item - field * p.tiles;
    const float2* src = p.src + (size_t)field * (size_t)p.src_nodes * CI;
    float2* dst = p.dst + (size_t)field * (size_t)p.dst_nodes * CO;
    const long long j = (long long)tile * xts::M + row;
    const bool row_ok = j < cnodes;
    int jx, jy, jz;
    node_xyz(row_ok ? j : 0, p.cx, p.cy, jx, jy, jz);
    // stage q: source s = q / NH (row j + s), columns (q % NH) KU + 16 grp
    auto load_stage = [&](float (&v)[16], int q) {
      const int sv = q / NH;
      const int dx = sv & 1, dy = (sv >> 1) & 1, dz = D == 3 ? (sv >> 2) & 1 : 0;
      const bool ok_n = row_ok && jx + dx < p.cx && jy + dy < p.cy && jz + dz < p.cz;
      const long long sidx = ((long long)(jz + dz) * p.cy + (jy + dy)) * p.cx + (jx + dx);
      const int c0 = (q % NH) * KU + 16 * grp;
      const float4* qp = reinterpret_cast<const float4*>(src + (ok_n ? sidx : 0) * CI + c0 / 2);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 w = ok_n ? __ldg(qp + u) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * u] = w.x;
        v[4 * u + 1] = w.y;
        v[4 * u + 2] = w.z;
        v[4 * u + 3] = w.w;
      }
    };
    // two stages per iteration: both register buffers named statically
    auto stage = [&](int q, float (&cur)[16], uint32_t slot) -> bool {
      if (q >= 2) wait_a(q & 1);
      xts::put16<KU, P>(slot + lane, 16 * grp, cur);
      tc::tmem_st_wait();
      if (q + 2 < UPI) load_stage(cur, q + 2);
      tc::fence_before();
      ok = __syncthreads_and(ok);
      if (!ok) return false;
      produce();
      if (tid == 0) {
        tc::fence_after();
        run_unit(slot, q > 0);
        tc::mma_commit(&abar[q & 1]);
      }
      return true;
    };
    float va[16], vb[16];
    load_stage(va, 0);
    if (UPI > 1) load_stage(vb, 1);
    {
      int q = 0;
      for (; q + 1 < UPI; q += 2) {
        if (!stage(q, va, slot0)) goto fail;
        if (!stage(q + 1, vb, slot1)) goto fail;
      }
      if (q < UPI && !stage(q, va, slot0)) goto fail;
    }
    if (UPI >= 2) wait_a((UPI - 2) & 1);
    wait_a((UPI - 1) & 1);
    tc::fence_after();
    // ---- epilogue: e[2j + p] += D[class p]; the thread group grp takes the
    // classes whose highest parity bit equals grp
#pragma unroll
    for (int pc = 0; pc < NCLS / 2; ++pc) {
      const int pcls = grp * (NCLS / 2) + pc;
      const int px = pcls & 1, py = (pcls >> 1) & 1, pz = D == 3 ? (pcls >> 2) & 1 : 0;
      const long long o_row =
          ((long long)(2 * jz + pz) * p.fy + (2 * jy + py)) * p.fx + (2 * jx + px);
#pragma unroll
      for (int c = 0; c < KO / 16; ++c) {
        float dv[16];
        tc::tmem_ld16(tD + lane + (uint32_t)(pcls * KO + 16 * c), dv);
        if (row_ok) {
          float4* op = reinterpret_cast<float4*>(dst + o_row * CO + 8 * c);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 e = op[u];
            op[u] = make_float4(e.x + dv[4 * u], e.y + dv[4 * u + 1], e.z + dv[4 * u + 2],
                                e.w + dv[4 * u + 3]);
          }
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
  if (p.err && tid == 0) atomicOr(p.err, 1);
  if (tid == 32) {
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
                 "r"((uint32_t)G::COLS));
  }
}

// ---------------------------------------------------------------------------
// Restriction from 8 channels with the fine lines staged in shared memory.
//
// The per-tap gather above reads, for one tap, every other fine node of a
// line (64 bytes per lane at a 128-byte stride), so each warp load touches
// 32 cache lines.  Here a stage is one (o_y, o_z): for each warp's 32 coarse
// nodes J (consecutive along x, one coarse line) the fine nodes
// 2 J_x0 - 1 .. 2 J_x0 + 63 of fine line (2 J_y + o_y, 2 J_z + o_z) are
// staged in shared memory by coalesced 16-byte asynchronous copies that all
// threads of the pipeline issue (zero-filled outside the grid), and the three
// taps o_x = -1, 0, +1 are read from there by three thread groups (tap o_x in
// group o_x + 1: fine node 2 J + o_x is slot 2 (J_x - J_x0) + o_x + 1 of the
// segment).  A stage is K = 48 (three taps of 2 x 8) against
// [R_(-1) | R_0 | R_(+1)] of its (o_y, o_z); all 3^(d-1) stage matrices stay
// in shared memory for the whole kernel.  Two independent tile pipelines of
// 384 threads share the CTA (and its 512 tensor-memory columns and the
// weights), each with its own ring of staged stages, A slots, accumulators
// and named barrier, so one pipeline's MMA and fold latency overlaps the
// other's work.  Each stage sums into its own accumulator (stages alternate
// between two) and the partials are added in FP32 registers, as in
// k_transfer_ts; the fold of a tile's last stages and its store happen during
// the next tile's first stages.
// ---------------------------------------------------------------------------
namespace xts {

template <int KO, int D, int P>
struct LineCfg {
  static constexpr int KS = 48;                       // K of a stage: three taps of 2 x 8
  static constexpr int S = D == 3 ? 9 : 3;            // stages (o_y, o_z) per tile
  static constexpr int PIPES = 2;
  static constexpr int PT = 384;                      // threads per pipeline: 3 taps x 4 warps
  static constexpr int THREADS = PIPES * PT;
  static constexpr int AW = P ? 2 * KS : KS / 2;      // A slot columns (TF32 hi + lo, or BF16 pairs)
  static constexpr int COLS = 256;                    // tensor memory per pipeline
  static constexpr int MATB = P ? 2 * KO * KS * 4 : KO * KS * 2;   // one stage's matrix
  static constexpr int CH = 65 * 4;                   // 16-byte chunks of a warp's 65 fine nodes
  static constexpr int SEGU = 33 * 8;                 // their 16-byte units in shared memory
  static constexpr int DBUF = 4 * SEGU * 16;          // one staged stage: four warp segments
  static constexpr int NBUF = 3;                      // staged stages per pipeline
  static constexpr int LPT = (4 * CH + PT - 1) / PT;  // chunks one thread stages per stage
  static constexpr int WBYTES = S * MATB;
  static constexpr int SMEM = WBYTES + PIPES * NBUF * DBUF;
  static_assert(2 * KO + 2 * AW <= COLS && SMEM <= 226 * 1024 && MATB % 16 == 0 &&
                    WBYTES % 16 == 0,
                "line restriction shape");
};

// 16-byte unit of chunk c of fine slot s in a staged segment: slots pair up
// in 128-byte rows, and the half and the chunk are XOR-swizzled by the row,
// so that the 8 lanes of a quarter warp reading slots 2 l + g (consecutive l)
// reach 8 different bank groups
__device__ __forceinline__ int line_unit(int s, int c) {
  const int row = s >> 1;
  return 8 * row + 4 * ((s & 1) ^ (row & 1)) + (c ^ ((row >> 1) & 3));
}

// AND of `v` over the `n` threads of named barrier `id` (a barrier for them)
__device__ __forceinline__ bool bar_and(bool v, int id, int n) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// 16 bytes global -> shared, asynchronous; `bytes` 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}

// one arrival on `bar` once this thread's earlier asynchronous copies have landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(tc::smem_u32(bar))
               : "memory");
}

}  // namespace xts

template <int KO, int D, int P>
__global__ void __launch_bounds__(xts::LineCfg<KO, D, P>::THREADS, 1)
    k_restrict_lines_ts(xts::XParams p) {
  using G = xts::LineCfg<KO, D, P>;
  constexpr int S = G::S, KS = G::KS, NBUF = G::NBUF, CO = KO / 2, LPT = G::LPT;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t wbar;
  __shared__ uint64_t dfull[G::PIPES][NBUF];
  __shared__ uint64_t abar[G::PIPES][2];
  __shared__ uint32_t tmem_base_sh;
  const int tid = threadIdx.x;
  const int pi = tid / G::PT, lt = tid - pi * G::PT;
  const int lw = lt >> 5, lanei = lt & 31;
  const int g = lw >> 2;               // tap o_x = g - 1
  const int ws = lw & 3;               // warp segment: rows 32 ws .. 32 ws + 31
  const int row = 32 * ws + lanei;

  if (tid == 0) {
    tc::bar_init(&wbar, 1);
    for (int q = 0; q < G::PIPES; ++q) {
      for (int b = 0; b < NBUF; ++b) tc::bar_init(&dfull[q][b], G::PT);
      tc::bar_init(&abar[q][0], 1);
      tc::bar_init(&abar[q][1], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     tc::smem_u32(&tmem_base_sh)),
                 "r"((uint32_t)(G::PIPES * G::COLS)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base_sh + (uint32_t)(pi * G::COLS);
  const uint32_t lane = (uint32_t)(32 * ws) << 16;
  const uint32_t slot0 = tmem + 2 * KO;          // A slots after the two accumulators
  const uint32_t wts = tc::smem_u32(smem);
  const int ring_off = G::WBYTES + pi * NBUF * G::DBUF;
  if (tid == 0) {                                // the stage matrices, once
    xts::expect_tx(&wbar, (uint32_t)G::WBYTES);
    for (int st = 0; st < S; ++st)
      xts::bulk_copy(wts + (uint32_t)(st * G::MATB),
                     reinterpret_cast<const uint8_t*>(p.mats) + (size_t)st * G::MATB,
                     (uint32_t)G::MATB, &wbar);
  }
  const int NV = G::PIPES * (int)gridDim.x;
  const int vp = pi * (int)gridDim.x + (int)blockIdx.x;
  const int my_items = vp < p.items ? (p.items - 1 - vp) / NV + 1 : 0;
  const int Q = my_items * S;                    // stages of this pipeline
  const long long cnodes = (long long)p.cx * p.cy * p.cz;
  const int bar_id = 1 + pi;
  bool ok = true;
  uint32_t aph[2] = {0, 0};
  int q_issued = 0, q_fail = -1, q_commit = -1;

  // ---- staging: this thread copies chunks lt + PT k (k < LPT) of each
  // stage's 4 x CH; per item it keeps, for each, the 16-byte index of the
  // chunk at (o_y, o_z) = (0, 0) and flags: bit 0 its segment exists, bit 1
  // J_y0 = 0, bit 2 J_z0 = 0, bit 3 its fine node is inside (x >= 0)
  long long cbase[LPT];
  int cflag[LPT];
  int cache_kk = -1;
  auto plan = [&](int kk) {
    const int item = vp + kk * NV;
    const int field = item / p.tiles, tile = item - field * p.tiles;
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int i = lt + G::PT * k;
      const int w = i / G::CH, within = i - w * G::CH;
      const int sl = within >> 2, c = within & 3;
      const long long j0 = (long long)tile * xts::M + 32 * w;
      cflag[k] = 0;
      cbase[k] = 0;
      if (i < 4 * G::CH && j0 < cnodes) {
        int jx0, jy0, jz0;
        node_xyz(j0, p.cx, p.cy, jx0, jy0, jz0);
        const long long node =
            ((long long)(2 * jz0) * p.fy + 2 * jy0) * p.fx + 2 * jx0 - 1 + sl;
        cbase[k] = ((long long)field * p.src_nodes + node) * 4 + c;
        cflag[k] = 1 | (jy0 == 0 ? 2 : 0) | (jz0 == 0 ? 4 : 0) | (jx0 > 0 || sl > 0 ? 8 : 0);
      }
    }
    cache_kk = kk;
  };
  auto issue = [&](int q) {            // every thread: its chunks of stage q
    const int kk = q / S, st = q - kk * S;
    if (kk != cache_kk) plan(kk);
    const int oy = st % 3 - 1, oz = D == 3 ? st / 3 - 1 : 0;
    const long long delta = ((long long)oz * p.fy + oy) * p.fx * 4;
    const int b = q % NBUF;
    const uint32_t dst0 = wts + (uint32_t)(ring_off + b * G::DBUF);
    const float4* src = reinterpret_cast<const float4*>(p.src);
#pragma unroll
    for (int k = 0; k < LPT; ++k) {
      const int i = lt + G::PT * k;
      if (i < 4 * G::CH) {
        const int w = i / G::CH, within = i - w * G::CH;
        const uint32_t dst = dst0 + (uint32_t)(16 * (w * G::SEGU + xts::line_unit(within >> 2, within & 3)));
        const int f = cflag[k];
        const bool in = (f & 1) && (f & 8) && !(oy < 0 && (f & 2)) && !(oz < 0 && (f & 4));
        xts::cp_async16(dst, in ? src + cbase[k] + delta : src, in ? 16u : 0u);
      }
    }
    xts::cp_async_arrive(&dfull[pi][b]);
  };
  for (; q_issued < Q && q_issued < NBUF; ++q_issued) issue(q_issued);

  // ---- per-thread sums of the stage partials (groups 0 and 1: columns
  // 16 g .. 16 g + 15 of the KO outputs)
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  auto fold = [&](int par) {
    if (16 * g < KO) {
      float dv[16];
      tc::tmem_ld16(tmem + lane + (uint32_t)(par * KO + 16 * g), dv);
#pragma unroll
      for (int u = 0; u < 16; ++u) acc[u] += dv[u];
    }
  };
  auto store = [&](int kk) {            // the sums of this pipeline's item kk
    const int item = vp + kk * NV;
    const int field = item / p.tiles, tile = item - field * p.tiles;
    const long long j = (long long)tile * xts::M + row;
    if (16 * g < KO && j < cnodes) {
      float4* op = reinterpret_cast<float4*>(p.dst + (size_t)field * (size_t)p.dst_nodes * CO +
                                             (size_t)j * CO + 8 * g);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        op[u] = make_float4(acc[4 * u], acc[4 * u + 1], acc[4 * u + 2], acc[4 * u + 3]);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  };
  auto retire = [&](int qd) {           // stage qd's MMAs are complete: fold, store at a tile's end
    ok = tc::bar_wait(&abar[pi][qd & 1], aph[qd & 1], p.err) && ok;
    aph[qd & 1] ^= 1;
    tc::fence_after();
    fold(qd & 1);
    if (qd % S == S - 1) store(qd / S);
  };
  // the staged slot of this thread's A row: fine node 2 J + o_x
  const int rslot = 2 * lanei + g;

  // the pipeline leaves its loops only together, on a failed vote
  for (int kk = 0; kk < my_items && q_fail < 0; ++kk) {
    for (int st = 0; st < S; ++st) {
      const int q = kk * S + st;
      const int b = q % NBUF;
      if (q >= 2) retire(q - 2);
      ok = tc::bar_wait(&dfull[pi][b], (uint32_t)((q / NBUF) & 1), p.err) && ok;
      const uint8_t* rp = smem + ring_off + b * G::DBUF + ws * (G::SEGU * 16);
      float4 c4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        c4[u] = *reinterpret_cast<const float4*>(rp + 16 * xts::line_unit(rslot, u));
      const uint32_t slot = slot0 + (uint32_t)((q & 1) * G::AW);
      if constexpr (P == 1) {
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const float x[8] = {c4[2 * hf].x, c4[2 * hf].y, c4[2 * hf].z, c4[2 * hf].w,
                              c4[2 * hf + 1].x, c4[2 * hf + 1].y, c4[2 * hf + 1].z,
                              c4[2 * hf + 1].w};
          uint32_t hi[8], lo[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            hi[i] = tc::to_tf32(x[i]);
            lo[i] = tc::to_tf32(x[i] - __uint_as_float(hi[i]));
          }
          tc::tmem_st8(slot + lane + (uint32_t)(16 * g + 8 * hf), hi);
          tc::tmem_st8(slot + lane + (uint32_t)(KS + 16 * g + 8 * hf), lo);
        }
      } else {
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          pk[2 * i] = tc::pack_bf16(c4[i].x, c4[i].y);
          pk[2 * i + 1] = tc::pack_bf16(c4[i].z, c4[i].w);
        }
        tc::tmem_st8(slot + lane + (uint32_t)(8 * g), pk);
      }
      tc::tmem_st_wait();
      tc::fence_before();
      ok = xts::bar_and(ok, bar_id, G::PT);
      if (!ok) {
        q_fail = q;
        break;
      }
      // every thread of the pipeline has read buffer b: it takes stage q + NBUF
      if (q_issued < Q) issue(q_issued++);
      if (lt == 0) {
        tc::fence_after();
        if (q == 0 && !tc::bar_wait(&wbar, 0, p.err)) ok = false;
        if (ok) {
          const uint32_t d = tmem + (uint32_t)((q & 1) * KO);
          const uint32_t bw = wts + (uint32_t)(st * G::MATB);
          constexpr uint32_t lbo = KO * 16;
          constexpr uint64_t kstep = (2 * lbo) >> 4;
          if constexpr (P == 1) {
            constexpr uint32_t idesc = tc::make_idesc_tf32(xts::M, KO);
            const uint64_t bh0 = tc::make_desc(bw, lbo, 128);
            const uint64_t bl0 = bh0 + ((KO * KS * 4) >> 4);
#pragma unroll
            for (int k8 = 0; k8 < KS / 8; ++k8) {
              const uint32_t ahi = slot + 8 * k8, alo = slot + KS + 8 * k8;
              tc::mma_tf32_ts(d, alo, bh0 + k8 * kstep, idesc, k8 > 0 ? 1u : 0u);
              tc::mma_tf32_ts(d, ahi, bl0 + k8 * kstep, idesc, 1u);
              tc::mma_tf32_ts(d, ahi, bh0 + k8 * kstep, idesc, 1u);
            }
          } else {
            constexpr uint32_t idesc = tc::make_idesc(xts::M, KO);
            const uint64_t b0 = tc::make_desc(bw, lbo, 128);
#pragma unroll
            for (int k16 = 0; k16 < KS / 16; ++k16)
              tc::mma_bf16_ts(d, slot + 8 * k16, b0 + k16 * kstep, idesc, k16 > 0 ? 1u : 0u);
          }
        }
        tc::mma_commit(&abar[pi][q & 1]);
        q_commit = q;
      }
    }
  }
  if (q_fail < 0) ok = xts::bar_and(ok, bar_id, G::PT);
  if (q_fail < 0 && ok) {                // the last two stages
    if (Q >= 2) retire(Q - 2);
    if (Q >= 1) retire(Q - 1);
    tc::fence_before();
    ok = xts::bar_and(ok, bar_id, G::PT);
  }
  if (!ok) {
    if (p.err && lt == 0) atomicOr(p.err, 1);
    if (lt == 0 && q_commit >= 0)
      tc::bar_wait(&abar[pi][q_commit & 1], (uint32_t)((q_commit >> 1) & 1), nullptr);
    tc::fence_before();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");   // this thread's copies have landed
  if (tid == 0) tc::bar_wait(&wbar, 0, nullptr);       // and the weight copies
  __syncthreads();
  if (tid < 32) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base_sh),
                 "r"((uint32_t)(G::PIPES * G::COLS)));
  }
}

namespace {

int xsm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

template <int KI, int KO, int D, int P, int DIR>
mcmg_status xts_launch(xts::XParams p, int nrhs, cudaStream_t st) {
  using G = xts::Cfg<xts::stage_k(KI, DIR), KO, P>;
  auto kern = k_transfer_ts<KI, KO, D, P, DIR>;
  static bool attr = false;
  // ring; at most PER_SM CTAs on one SM so that their tensor memory fits
  const size_t guard = (size_t)(228 * 1024) / (G::PER_SM + 1) + 16 - 2048;
  size_t smem = std::max((size_t)G::RB * G::UNIT, guard);
  smem = (smem + 127) & ~(size_t)127;
  if (!attr) {
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  const long long cn = (long long)p.cx * p.cy * p.cz;
  p.tiles = (int)((cn + xts::M - 1) / xts::M);
  p.items = p.tiles * (DIR == 1 ? (1 << D) : 1) * nrhs;
  const int grid = std::min(p.items, xsm_count() * G::PER_SM);
  kern<<<grid, xts::THREADS, smem, st>>>(p);
  MCMG_CHECK_LAUNCH(DIR == 0 ? "restrict_ts" : "prolong_ts");
  return MCMG_OK;
}

template <int KI, int KO, int D, int P>
mcmg_status block_launch(xts::XParams p, int nrhs, cudaStream_t st) {
  using G = xts::BlockCfg<KI, KO, D, P>;
  auto kern = k_prolong_block_ts<KI, KO, D, P>;
  static bool attr = false;
  const size_t guard = (size_t)(228 * 1024) / (G::PER_SM + 1) + 16 - 2048;
  size_t smem = std::max((size_t)G::RB * G::UNIT, guard);
  smem = (smem + 127) & ~(size_t)127;
  if (!attr) {
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  const long long cn = (long long)p.cx * p.cy * p.cz;
  p.tiles = (int)((cn + xts::M - 1) / xts::M);
  p.items = p.tiles * nrhs;
  const int grid = std::min(p.items, xsm_count() * G::PER_SM);
  kern<<<grid, xts::THREADS, smem, st>>>(p);
  MCMG_CHECK_LAUNCH("prolong_block_ts");
  return MCMG_OK;
}

template <int D, int P, int DIR>
mcmg_status xts_channels(int CI, int CO, const xts::XParams& p, int nrhs, cudaStream_t st) {
  // (input channels, output channels): restriction C -> C', prolongation C' -> C
#define XTS_CASE(ci, co)                                          \
  if (CI == ci && CO == co) return xts_launch<2 * ci, 2 * co, D, P, DIR>(p, nrhs, st);
  if constexpr (DIR == 0) {
    XTS_CASE(8, 16) XTS_CASE(8, 8) XTS_CASE(16, 32) XTS_CASE(16, 16) XTS_CASE(32, 64)
    XTS_CASE(32, 32) XTS_CASE(64, 64)
  } else {
    XTS_CASE(16, 8) XTS_CASE(16, 16) XTS_CASE(32, 16) XTS_CASE(32, 32) XTS_CASE(64, 32)
    XTS_CASE(64, 64)
  }
#undef XTS_CASE
  set_error("tensor-core transfer: no variant for %d -> %d channels", CI, CO);
  return MCMG_ERR_SHAPE;
}

}  // namespace

bool xts_supported(const Level& L, bool restrict_) {
  if (!L.use_ts || !L.ts_R || !L.ts_P) return false;
  const int CI = restrict_ ? L.C : L.Cn, CO = restrict_ ? L.Cn : L.C;
  if (restrict_)
    return (CI == 8 && (CO == 16 || CO == 8)) || (CI == 16 && (CO == 32 || CO == 16)) ||
           (CI == 32 && (CO == 64 || CO == 32)) || (CI == 64 && CO == 64);
  return (CI == 16 && (CO == 8 || CO == 16)) || (CI == 32 && (CO == 16 || CO == 32)) ||
         (CI == 64 && (CO == 32 || CO == 64));
}

mcmg_status launch_transfer_ts(const Level& L, bool restrict_, const float2* src, float2* dst,
                               int nrhs, cudaStream_t st) {
  if (!xts_supported(L, restrict_)) {
    set_error("tensor-core transfer not available on this level");
    return MCMG_ERR_SHAPE;
  }
  const Grid gc = L.g.coarse();
  xts::XParams p{};
  p.src = src;
  p.dst = dst;
  p.mats = restrict_ ? L.ts_R : L.ts_P;
  p.fx = L.g.nx;
  p.fy = L.g.ny;
  p.fz = L.g.nz;
  p.cx = gc.nx;
  p.cy = gc.ny;
  p.cz = gc.nz;
  p.src_nodes = restrict_ ? L.g.nodes() : gc.nodes();
  p.dst_nodes = restrict_ ? gc.nodes() : L.g.nodes();
  p.err = L.err;
  const int CI = restrict_ ? L.C : L.Cn, CO = restrict_ ? L.Cn : L.C;
  const bool d3 = L.g.d == 3, tf = L.ts_prec == MCMG_FP32_TC;
  if (restrict_) {
    if (tf) return d3 ? xts_channels<3, 1, 0>(CI, CO, p, nrhs, st) : xts_channels<2, 1, 0>(CI, CO, p, nrhs, st);
    return d3 ? xts_channels<3, 0, 0>(CI, CO, p, nrhs, st) : xts_channels<2, 0, 0>(CI, CO, p, nrhs, st);
  }
  if (tf) return d3 ? xts_channels<3, 1, 1>(CI, CO, p, nrhs, st) : xts_channels<2, 1, 1>(CI, CO, p, nrhs, st);
  return d3 ? xts_channels<3, 0, 1>(CI, CO, p, nrhs, st) : xts_channels<2, 0, 1>(CI, CO, p, nrhs, st);
}

// Block prolongation: (C_n, C) with C_n in {16, 32, 64}, C = C_n or C_n / 2,
// and all 2^d classes in one MMA (2^d x 2C <= 256 columns).
bool xts_block_pair(int d, int Cn, int C) {
  if (!((Cn == 16 || Cn == 32 || Cn == 64) && (C == Cn || 2 * C == Cn))) return false;
  return (1 << d) * 2 * C <= 256;
}

bool xts_block_supported(const Level& L) {
  return L.use_ts && L.ts_Pb && xts_block_pair(L.g.d, L.Cn, L.C);
}

namespace {
template <int D, int P>
mcmg_status block_channels(int Cn, int C, const xts::XParams& p, int nrhs, cudaStream_t st) {
#define XTB_CASE(cn, c)                                                            \
  if (Cn == cn && C == c) {                                                         \
    if constexpr ((1 << D) * 2 * c <= 256) return block_launch<2 * cn, 2 * c, D, P>(p, nrhs, st); \
  }
  XTB_CASE(16, 8) XTB_CASE(16, 16) XTB_CASE(32, 16) XTB_CASE(32, 32) XTB_CASE(64, 32)
  XTB_CASE(64, 64)
#undef XTB_CASE
  set_error("block prolongation: no variant for %d -> %d channels", Cn, C);
  return MCMG_ERR_SHAPE;
}
}  // namespace

mcmg_status launch_prolong_block_ts(const Level& L, const float2* ec, float2* e, int nrhs,
                                    cudaStream_t st) {
  if (!xts_block_supported(L)) {
    set_error("block prolongation not available on this level");
    return MCMG_ERR_SHAPE;
  }
  const Grid gc = L.g.coarse();
  xts::XParams p{};
  p.src = ec;
  p.dst = e;
  p.mats = L.ts_Pb;
  p.fx = L.g.nx;
  p.fy = L.g.ny;
  p.fz = L.g.nz;
  p.cx = gc.nx;
  p.cy = gc.ny;
  p.cz = gc.nz;
  p.src_nodes = gc.nodes();
  p.dst_nodes = L.g.nodes();
  p.err = L.err;
  const bool d3 = L.g.d == 3, tf = L.ts_prec == MCMG_FP32_TC;
  if (tf) return d3 ? block_channels<3, 1>(L.Cn, L.C, p, nrhs, st) : block_channels<2, 1>(L.Cn, L.C, p, nrhs, st);
  return d3 ? block_channels<3, 0>(L.Cn, L.C, p, nrhs, st) : block_channels<2, 0>(L.Cn, L.C, p, nrhs, st);
}

// Line-staged restriction from 8 channels: C_n in {8, 16}, and a coarse x
// extent that is a multiple of 32, so that each warp's 32 coarse nodes lie
// on one coarse line.
bool xts_lines_pair(int C, int Cn, int cx) {
  return C == 8 && (Cn == 16 || Cn == 8) && cx >= 32 && cx % 32 == 0;
}

bool xts_lines_supported(const Level& L) {
  return L.use_ts && L.ts_R3 && xts_lines_pair(L.C, L.Cn, L.g.coarse().nx);
}

namespace {
template <int KO, int D, int P>
mcmg_status lines_launch(xts::XParams p, int nrhs, cudaStream_t st) {
  using G = xts::LineCfg<KO, D, P>;
  auto kern = k_restrict_lines_ts<KO, D, P>;
  static bool attr = false;
  // one CTA per SM (it allocates all 512 tensor-memory columns)
  const size_t smem = std::max((size_t)G::SMEM, (size_t)120 * 1024);
  if (!attr) {
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  const long long cn = (long long)p.cx * p.cy * p.cz;
  p.tiles = (int)((cn + xts::M - 1) / xts::M);
  p.items = p.tiles * nrhs;
  const int grid = std::min((p.items + G::PIPES - 1) / G::PIPES, xsm_count());
  kern<<<grid, G::THREADS, smem, st>>>(p);
  MCMG_CHECK_LAUNCH("restrict_lines_ts");
  return MCMG_OK;
}
}  // namespace

mcmg_status launch_restrict_lines_ts(const Level& L, const float2* src, float2* dst, int nrhs,
                                     cudaStream_t st) {
  if (!xts_lines_supported(L)) {
    set_error("line-staged restriction not available on this level");
    return MCMG_ERR_SHAPE;
  }
  // the bulk copies of the fine lines need a 16-byte aligned field
  if (reinterpret_cast<uintptr_t>(src) % 16) return launch_transfer_ts(L, true, src, dst, nrhs, st);
  const Grid gc = L.g.coarse();
  xts::XParams p{};
  p.src = src;
  p.dst = dst;
  p.mats = L.ts_R3;
  p.fx = L.g.nx;
  p.fy = L.g.ny;
  p.fz = L.g.nz;
  p.cx = gc.nx;
  p.cy = gc.ny;
  p.cz = gc.nz;
  p.src_nodes = L.g.nodes();
  p.dst_nodes = gc.nodes();
  p.err = L.err;
  const bool d3 = L.g.d == 3, tf = L.ts_prec == MCMG_FP32_TC;
  if (L.Cn == 16) {
    if (tf) return d3 ? lines_launch<32, 3, 1>(p, nrhs, st) : lines_launch<32, 2, 1>(p, nrhs, st);
    return d3 ? lines_launch<32, 3, 0>(p, nrhs, st) : lines_launch<32, 2, 0>(p, nrhs, st);
  }
  if (tf) return d3 ? lines_launch<16, 3, 1>(p, nrhs, st) : lines_launch<16, 2, 1>(p, nrhs, st);
  return d3 ? lines_launch<16, 3, 0>(p, nrhs, st) : lines_launch<16, 2, 0>(p, nrhs, st);
}

// Host: a complex Cout x Cin matrix M[co][ci] (float2, row-major) -> its real
// block form (N = 2 Cout rows, K = 2 Cin) as a B operand in the no-swizzle
// K-major core-matrix layout: BF16 (chunks of 8 K-elements) or TF32 hi and lo
// halves (chunks of 4), [hi][lo].
void pack_ts_rect(const float2* Mc, int Cout, int Cin, bool tf32, void* out) {
  const int N = 2 * Cout, K = 2 * Cin;
  auto rna = [](float v) {
    uint32_t b;
    std::memcpy(&b, &v, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
  };
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < K; ++k) {
      const float2 m = Mc[(size_t)(n >> 1) * Cin + (k >> 1)];
      float v;
      if ((n & 1) == 0) v = (k & 1) == 0 ? m.x : -m.y;
      else v = (k & 1) == 0 ? m.y : m.x;
      if (tf32) {
        float* hi = static_cast<float*>(out);
        float* lo = hi + (size_t)N * K;
        const size_t pos = ((size_t)(k >> 2) * N + n) * 4 + (k & 3);
        const float h = rna(v);
        hi[pos] = h;
        lo[pos] = rna(v - h);
      } else {
        uint16_t* o = static_cast<uint16_t*>(out);
        const __nv_bfloat16 bv = __float2bfloat16_rn(v);
        const size_t pos = ((size_t)(k >> 3) * N + n) * 8 + (k & 7);
        std::memcpy(o + pos, &bv, 2);
      }
    }
}

}  // namespace mcmg
