// Tensor-core (tcgen05) forms of the two contractions on sm_103a.
//
// GEMM1  X_k[i, j] = sum_r (a_k[r] Psi[r, i]) Psi[r, j]     (H-breve', §II.C)
//        upper-part tiles only; the whole grid reduction runs inside one
//        tile, in segments of 1024 rows whose TMEM results are summed in FP32
//        registers; the a_k weighting is applied to the A rows between their
//        TMA load and the MMAs, which read the weighted A from tensor memory.
//        Three forms: 256 x 256 tiles on a CTA pair (cta_group::2, M = 256
//        MMAs, each CTA holding half of the A and B rows; the default),
//        128 x 256 tiles on one CTA, and 128 x 128 tiles with one or two
//        directions.
// GEMM2  drho_k(r) = factor * sum_j Psi[r, j] (sum_{i <= j} Psi[r, i] X''_k[i, j])
//        tile 128 (r) x 256 (j); for each j-block the i-reduction stops at the
//        block's end (X'' is zero below the diagonal); two TMEM accumulators so
//        the row-dot epilogue of one j-block overlaps the MMAs of the next.
//        Psi X'' only ever lives in tensor memory.  With one direction at
//        N_s >= 2048 an item's j-blocks are split into parts run by
//        neighbouring CTAs (FP64 part sums, added by k_g2_combine).
//
// Both: operands K-major in 64-byte-swizzled shared memory, loaded by TMA;
// one thread issues tcgen05.mma, accumulators (FP32) in tensor memory, read
// back with tcgen05.ld.  Precisions: split BF16x3 (a = a_hi + a_lo, three
// bf16 products a_hi b_hi + a_hi b_lo + a_lo b_hi) and TF32.  Persistent
// grids (one CTA per SM) over work items; every wait is bounded (4 s), after
// which the kernel raises the timeout status bit, drains its own copies and
// MMAs, frees its tensor memory and returns.
#include "lrdm_internal.h"
#include "tc_problem.h"
#include "tc_ptx.cuh"

#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <stdio.h>
#include <stdlib.h>

namespace lrdm {
namespace {

constexpr int BM = 128;                 // MMA M = tensor-memory lanes
constexpr int ROWB = 64;                // bytes per swizzled smem row (64-byte swizzle)
constexpr int KSTEPS = ROWB / 32;       // 32-byte MMA K steps per row
constexpr int TILE_A = BM * ROWB;       // 8 KB per operand part
constexpr int NTHREADS = 192;           // warp 0 TMA, warp 1 MMA, warps 2-5 math / epilogue
constexpr uint64_t WAIT_NS = 4000000000ull;
constexpr uint16_t PAIR_MASK = 0x3;           // both CTAs of a pair (cluster ranks 0, 1)

template <int PREC>
struct Tr;
template <>
struct Tr<LRDM_BF16X3> {
  static constexpr int BK = 32;          // bf16 per 64-byte row
  static constexpr int PARTS = 2;        // hi, lo
};
template <>
struct Tr<LRDM_TF32> {
  static constexpr int BK = 16;          // fp32 per 64-byte row
  static constexpr int PARTS = 1;
};

// GEMM2 configuration for j-tile width BN2 (128 or 256): the B operand is
// loaded as BN2 / 128 boxes of 128 rows; deeper pipelines for the narrow tile.
template <int PREC, int BN2>
struct G2Cfg {
  static constexpr int PARTS = Tr<PREC>::PARTS, BK = Tr<PREC>::BK;
  // state chunks of BK per stage: TF32 takes two 16-state chunks (the
  // operand boxes), so that a stage holds four MMAs as BF16x3's holds six
  static constexpr int SUB = PREC == LRDM_TF32 ? 2 : 1;
  static constexpr int TILE_B2 = BN2 * ROWB;
  static constexpr int CHUNK = PARTS * (TILE_A + TILE_B2);      // A and B parts of one chunk
  static constexpr int SB = SUB * CHUNK;
  static constexpr int STAGES = BN2 == 256 ? 4 : 6;
  static constexpr int SMEM = STAGES * SB + 1024 + 512;
  static constexpr uint32_t IDESC = ptx::idesc_make(PREC == LRDM_BF16X3 ? 1 : 2, BM, BN2);
};


struct Bars {
  uint64_t* full;      // [STAGES] TMA landed
  uint64_t* empty;     // [STAGES] MMAs done with the stage
  uint64_t* ready;     // [STAGES] A tile scaled (GEMM1 only)
  uint64_t* acc_full;  // [2]
  uint64_t* acc_empty; // [2]
  uint64_t* drain;     // [1]
  uint32_t* tmem_slot;
  volatile int* abort;
};

template <int STAGES>
__device__ __forceinline__ Bars carve(uint8_t* tail) {
  Bars b;
  uint64_t* p = reinterpret_cast<uint64_t*>(tail);
  b.full = p;
  b.empty = p + STAGES;
  b.ready = p + 2 * STAGES;
  b.acc_full = p + 3 * STAGES;
  b.acc_empty = p + 3 * STAGES + 2;
  b.drain = p + 3 * STAGES + 4;
  b.tmem_slot = reinterpret_cast<uint32_t*>(p + 3 * STAGES + 5);
  b.abort = reinterpret_cast<volatile int*>(p + 3 * STAGES + 6);
  return b;
}

__device__ __forceinline__ bool wait1(uint64_t* bar, uint32_t parity, const Bars& B, int* status) {
  return ptx::mbar_wait(bar, parity, B.abort, status, WAIT_NS, STATUS_TIMEOUT);
}
// Warp-uniform bounded wait: lane 0 polls, and the whole warp takes its result
// (__syncwarp orders the other lanes' later shared-memory reads after it).
__device__ __forceinline__ bool waitw(uint64_t* bar, uint32_t parity, const Bars& B, int* status) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = ptx::mbar_wait(bar, parity, B.abort, status, WAIT_NS, STATUS_TIMEOUT);
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}
// Wait that ignores the abort flag (used to drain in-flight work on exit).
__device__ __forceinline__ void wait_drain(uint64_t* bar, uint32_t parity) {
  volatile int never = 0;
  ptx::mbar_wait(bar, parity, &never, nullptr, 200000000ull, 0);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int PREC, int BN2>
__device__ __forceinline__ void issue_stage_mmas(uint32_t d, uint32_t sa, uint32_t first) {
  using C = G2Cfg<PREC, BN2>;
  constexpr int PARTS = Tr<PREC>::PARTS;
  const uint32_t a0 = sa, a1 = sa + TILE_A;
  const uint32_t b0 = sa + PARTS * TILE_A, b1 = b0 + C::TILE_B2;
#pragma unroll
  for (int kk = 0; kk < KSTEPS; ++kk) {     // 32-byte K steps along the swizzled row
    const uint32_t off = kk * 32;
    const uint32_t acc = (first && kk == 0) ? 0u : 1u;
    if (PREC == LRDM_BF16X3) {
      ptx::mma_f16(d, ptx::desc_k_sw64(a0 + off), ptx::desc_k_sw64(b0 + off), C::IDESC, acc);
      ptx::mma_f16(d, ptx::desc_k_sw64(a0 + off), ptx::desc_k_sw64(b1 + off), C::IDESC, 1);
      ptx::mma_f16(d, ptx::desc_k_sw64(a1 + off), ptx::desc_k_sw64(b0 + off), C::IDESC, 1);
    } else {
      ptx::mma_tf32(d, ptx::desc_k_sw64(a0 + off), ptx::desc_k_sw64(b0 + off), C::IDESC, acc);
    }
  }
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Round alignment of the persistent grids.  A CTA (or CTA pair) takes the
// items b, b + n, b + 2n, ... of a launch; the items of a round that stream
// the same operand rows (the directions of one projection tile, the
// direction group of one response row block) share them through L2 only
// while they reach the same rows at about the same time.  Over long items
// the static assignment lets the start times drift apart by a sixth of an
// item (2.6 ms of 15.8 ms in the projection at 96^3), far more rows than L2
// holds, and the shared rows are read again from HBM.  So the producers count
// the rounds whose loads they have issued in one grid-wide counter (zeroed
// before the launch) and start a round only when every producer has issued
// the previous one.  The host enables it only when all items of a launch
// have the same length; the wait is bounded (ALIGN_NS), after which a
// producer stops aligning, so no result ever depends on it.
constexpr uint64_t ALIGN_NS = 20000000ull;

// Arrivals the counter holds once rounds 0..r are issued, for `items` items
// over `units` grid units with `per_unit` producers each.
__device__ __forceinline__ unsigned round_target(int r, int items, int units, int per_unit) {
  unsigned t = 0;
  for (int q = 0; q <= r; ++q) {
    const int a = items - q * units;
    t += (unsigned)per_unit * (unsigned)(a >= units ? units : (a > 0 ? a : 0));
  }
  return t;
}

// ===========================================================================
// GEMM2: response contraction with the row-dot epilogue
// ===========================================================================

// One grouped launch covers several problems (systems / spin channels); slot
// q of the launch is problem pid[q] with K[q] directions, items
// [begin[q], begin[q + 1]).  Slots are ordered by decreasing item cost.
struct G2Params {
  const TcProblem* probs;
  int nslot;
  int begin[TC_MAX_SLOTS + 1];
  int pid[TC_MAX_SLOTS];
  int K[TC_MAX_SLOTS];
  int kgroup[TC_MAX_SLOTS];         // directions that share one Psi row block side by side
  double factor[TC_MAX_SLOTS];
  const void* v[TC_MAX_SLOTS];
  long long v_stride[TC_MAX_SLOTS];
  void* out[TC_MAX_SLOTS];
  long long out_stride[TC_MAX_SLOTS];
  int nR[TC_MAX_SLOTS];             // row blocks processed (the problem's nR; fewer when tuning)
  // j-tile parts: with nsplit > 1 a (row block, direction) item becomes nsplit
  // items, part p taking the j-tiles jl[jb[p] .. jb[p + 1]) and writing its
  // FP64 sum to the problem's part buffer (summed by k_g2_combine)
  int nsplit[TC_MAX_SLOTS];
  int jb[TC_MAX_SLOTS][G2_MAX_SPLIT + 1];
  unsigned char jl[TC_MAX_SLOTS][G2_MAX_NJ];
  int out_io, out_is_io;
  int* status;
  unsigned* sync;                   // round counter (zero at launch), or null: no alignment
};

__device__ __forceinline__ int find_slot(const int* begin, int nslot, int item) {
  int q = 0;
  while (q + 1 < nslot && item >= begin[q + 1]) ++q;
  return q;
}

// Item order within a problem: groups of kgroup directions, row block,
// direction within the group, j-tile part -- the items of one row block run
// side by side and share its Psi rows through L2, while only kgroup matrices
// X''_k compete for L2 at a time.  [j0, j1) indexes the item's j-tiles
// (through jl when the problem's items are split into parts).
template <int BN2>
__device__ __forceinline__ const TcProblem* g2_item(const G2Params& P, int item, int& q, int& k,
                                                    int& R, int& jp, int& j0, int& j1) {
  q = find_slot(P.begin, P.nslot, item);
  const TcProblem* pr = P.probs + P.pid[q];
  const int local = item - P.begin[q];
  const int G = P.kgroup[q], K = P.K[q], S = P.nsplit[q];
  const int per = P.nR[q] * G * S;
  const int kg = local / per;
  const int rem = local - kg * per;
  const int g = min(G, K - kg * G);
  R = rem / (g * S);
  const int t = rem - R * g * S;
  k = kg * G + t / S;
  jp = t - (t / S) * S;
  if (S > 1) {
    j0 = P.jb[q][jp];
    j1 = P.jb[q][jp + 1];
  } else {
    j0 = 0;
    j1 = (pr->ns_pad + BN2 - 1) / BN2;
  }
  return pr;
}

__device__ __forceinline__ int g2_tile(const G2Params& P, int q, int jj) {
  return P.nsplit[q] > 1 ? (int)P.jl[q][jj] : jj;
}

// Row-dot of one j-tile: sum over the tile's BN2 columns of this thread's
// TMEM lane (row r of Psi X'') times Psi[r, j] (bf16 hi + lo, or FP32).
template <int PREC, int BN2>
__device__ __forceinline__ float g2_tile_dot(uint32_t tb, int J, long long r, long long Ng, int ns_pad,
                                             const void* psi0, const void* psi1) {
  float part = 0.f;
#pragma unroll 1
  for (int c = 0; c < BN2 / 32; ++c) {
    float v[32];
    ptx::tmem_ld32(tb + c * 32, v);
    const int j0 = J * BN2 + c * 32;
    if (r < Ng && j0 < ns_pad) {
      const long long o = r * ns_pad + j0;
      if (PREC == LRDM_BF16X3) {
        const uint4* ph = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(psi0) + o);
        const uint4* pl = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(psi1) + o);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint4 h = __ldg(ph + u), l = __ldg(pl + u);
          const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            part += v[u * 8 + 2 * e] * (bf_lo(hw[e]) + bf_lo(lw[e]));
            part += v[u * 8 + 2 * e + 1] * (bf_hi(hw[e]) + bf_hi(lw[e]));
          }
        }
      } else {
        const float4* pf = reinterpret_cast<const float4*>(static_cast<const float*>(psi0) + o);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 x = __ldg(pf + u);
          part += v[u * 4] * x.x + v[u * 4 + 1] * x.y + v[u * 4 + 2] * x.z + v[u * 4 + 3] * x.w;
        }
      }
    }
  }
  return part;
}

// The epilogue's result for row r: out = factor * drho (- v) in the io dtype,
// the FP32 sum, or (items split into j-tile parts) the FP64 part sum.
__device__ __forceinline__ void g2_store(const G2Params& P, const TcProblem* pr, int q, int k, int jp,
                                         long long r, double acc_row) {
  const long long Ng = pr->Ng;
  if (r >= Ng) return;
  if (P.nsplit[q] > 1) {
    pr->part[((long long)jp * P.K[q] + k) * Ng + r] = P.factor[q] * acc_row;
    return;
  }
  const double d = P.factor[q] * acc_row;
  const long long o = (long long)k * P.out_stride[q] + r;
  if (P.out_is_io) {
    const long long ov = (long long)k * P.v_stride[q] + r;
    if (P.out_io == LRDM_DTYPE_F64)
      static_cast<double*>(P.out[q])[o] = d - static_cast<const double*>(P.v[q])[ov];
    else
      static_cast<float*>(P.out[q])[o] = (float)(d - (double)static_cast<const float*>(P.v[q])[ov]);
  } else {
    static_cast<float*>(P.out[q])[o] = (float)d;
  }
}

template <int PREC, int BN2>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm2_tc(const __grid_constant__ G2Params P) {
  using C = G2Cfg<PREC, BN2>;
  constexpr int STAGES = C::STAGES, PARTS = C::PARTS, BK = C::BK;
  constexpr int SB = C::SB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Bars B = carve<STAGES>(smem + STAGES * SB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = P.begin[P.nslot];

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&B.full[s], 1);
      ptx::mbar_init(&B.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&B.acc_full[a], 1);
      ptx::mbar_init(&B.acc_empty[a], 4);
    }
    ptx::mbar_init(B.drain, 1);
    *B.abort = 0;
    ptx::fence_barrier_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 1) {
    ptx::tmem_alloc(B.tmem_slot, 2 * BN2);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *B.tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    for (int q = 0; q < P.nslot; ++q) {
      const TcProblem* pr = P.probs + P.pid[q];
      ptx::tmap_acquire(&pr->g2a0);
      ptx::tmap_acquire(&pr->g2b0);
      if (PARTS == 2) {
        ptx::tmap_acquire(&pr->g2a1);
        ptx::tmap_acquire(&pr->g2b1);
      }
    }
    int s = 0;
    uint32_t ph = 0;
    int pending[STAGES];
    for (int i = 0; i < STAGES; ++i) pending[i] = -1;
    // round alignment (equal-length items only, as set by the host): the
    // CTAs of a direction group share their row block's Psi rows, and all
    // row blocks of a direction its X'' tiles, through L2
    bool align = P.sync != nullptr;
    int round = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x, ++round) {
      if (align && round > 0 &&
          !ptx::counter_wait_geq(P.sync, round_target(round - 1, items, gridDim.x, 1), ALIGN_NS))
        align = false;
      int q, k, R, jp, j0, j1;
      const TcProblem* pr = g2_item<BN2>(P, item, q, k, R, jp, j0, j1);
      const int ns_pad = pr->ns_pad;
      const CUtensorMap *mA0 = &pr->g2a0, *mA1 = &pr->g2a1, *mB0 = &pr->g2b0, *mB1 = &pr->g2b1;
      bool ok = true;
      for (int jj = j0; jj < j1 && ok; ++jj) {
        const int J = g2_tile(P, q, jj);
        const int nch = min((J + 1) * BN2, ns_pad) / (BK * C::SUB);     // stages
        const int nbox = min(BN2, ns_pad - J * BN2) / 128;      // 128-row boxes of B in this j-tile
        for (int ic = 0; ic < nch; ++ic) {
          if (!wait1(&B.empty[s], ph ^ 1, B, P.status)) { ok = false; break; }
          ptx::mbar_arrive_expect_tx(&B.full[s], C::SUB * PARTS * (TILE_A + nbox * 128 * ROWB));
#pragma unroll
          for (int c = 0; c < C::SUB; ++c) {
            uint8_t* st = smem + s * SB + c * C::CHUNK;
            const int i0 = (ic * C::SUB + c) * BK;              // first state of the chunk
            ptx::tma_load_2d(st, mA0, &B.full[s], i0, R * BM);
            if (PARTS == 2) ptx::tma_load_2d(st + TILE_A, mA1, &B.full[s], i0, R * BM);
            for (int hb = 0; hb < nbox; ++hb) {
              ptx::tma_load_3d(st + PARTS * TILE_A + hb * 128 * ROWB, mB0, &B.full[s], i0,
                               J * BN2 + hb * 128, k);
              if (PARTS == 2)
                ptx::tma_load_3d(st + PARTS * TILE_A + C::TILE_B2 + hb * 128 * ROWB, mB1, &B.full[s],
                                 i0, J * BN2 + hb * 128, k);
            }
          }
          pending[s] = (int)ph;
          if (++s == STAGES) { s = 0; ph ^= 1; }
        }
      }
      if (!ok) break;
      if (P.sync) ptx::counter_add_release(P.sync, 1);         // this round's loads are issued
    }
    for (int i = 0; i < STAGES; ++i)
      if (pending[i] >= 0) wait_drain(&B.full[i], (uint32_t)pending[i]);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int s = 0, a = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      int q, k, R, jp, j0, j1;
      const TcProblem* pr = g2_item<BN2>(P, item, q, k, R, jp, j0, j1);
      const int ns_pad = pr->ns_pad;
      for (int jj = j0; jj < j1 && ok; ++jj) {
        const int J = g2_tile(P, q, jj);
        if (!wait1(&B.acc_empty[a], aph ^ 1, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * BN2);
        const int nch = min((J + 1) * BN2, ns_pad) / (BK * C::SUB);     // stages
        for (int ic = 0; ic < nch; ++ic) {
          if (!wait1(&B.full[s], ph, B, P.status)) { ok = false; break; }
          ptx::tc_fence_after();
#pragma unroll
          for (int c = 0; c < C::SUB; ++c)
            issue_stage_mmas<PREC, BN2>(d, ptx::smem_u32(smem + s * SB + c * C::CHUNK), ic == 0 && c == 0);
          ptx::mma_commit(&B.empty[s]);
          if (++s == STAGES) { s = 0; ph ^= 1; }
        }
        if (!ok) break;
        ptx::mma_commit(&B.acc_full[a]);
        if (++a == 2) { a = 0; aph ^= 1; }
      }
    }
    ptx::mma_commit(B.drain);
    wait_drain(B.drain, 0);
  } else if (warp >= 2) {
    // ---------------- row-dot epilogue (TMEM lane quarter = warp % 4) ----------------
    const int lq = warp & 3;
    const int row = lq * 32 + lane;
    int a = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      int q, k, R, jp, j0, j1;
      const TcProblem* pr = g2_item<BN2>(P, item, q, k, R, jp, j0, j1);
      const int ns_pad = pr->ns_pad;
      const long long Ng = pr->Ng;
      const void* psi0 = pr->psi0;
      const void* psi1 = pr->psi1;
      const long long r = (long long)R * BM + row;
      double acc_row = 0.0;
      for (int jj = j0; jj < j1; ++jj) {
        const int J = g2_tile(P, q, jj);
        if (!waitw(&B.acc_full[a], aph, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(a * BN2);
        const float part = g2_tile_dot<PREC, BN2>(tb, J, r, Ng, ns_pad, psi0, psi1);
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&B.acc_empty[a]);
        acc_row += (double)part;
        if (++a == 2) { a = 0; aph ^= 1; }
      }
      if (!ok) break;
      g2_store(P, pr, q, k, jp, r, acc_row);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 2 * BN2);
  }
}

// ===========================================================================
// GEMM2 on CTA pairs (cta_group::2): 256 grid rows x 256-wide j-tiles
// ===========================================================================
//
// A cluster of two CTAs on neighbouring SMs computes the response of a
// 256-row block: CTA r loads (TMA) the Psi rows of the 128-row block
// 2 R2 + r (the A rows) and the X'' rows of its half of each 256-wide j-tile
// (states J 256 + 128 r .. + 127, the B rows); one thread of the even CTA
// issues M = 256, N = 256 pair MMAs with both operands in shared memory, and
// each CTA's tensor memory receives its 128 rows x 256 columns (two
// accumulators, so the row-dot epilogue of one j-tile overlaps the MMAs of
// the next).  Per SM that halves the X'' bytes loaded and read per MMA
// against the single-CTA kernel.  The odd CTA's MMA thread relays its stage
// arrivals: it waits for its own full barrier and arrives on the even CTA's
// (pfull, one arrival); the MMA commits are multicast to both CTAs' empty and
// acc-full barriers; the epilogue warps of both CTAs arrive on the even CTA's
// acc-empty barrier (8 arrivals).  Items: as k_gemm2_tc with P.nR = the
// number of 256-row blocks.

template <int PREC>
struct G2PCfg {
  static constexpr int PARTS = Tr<PREC>::PARTS, BK = Tr<PREC>::BK;
  static constexpr int SUB = PREC == LRDM_TF32 ? 2 : 1;
  static constexpr int BN2 = 256;                       // j-tile width (both CTAs)
  static constexpr int TILE_B = 128 * ROWB;             // this CTA's 128 X'' rows, one part
  static constexpr int CHUNK = PARTS * (TILE_A + TILE_B);
  static constexpr int SB = SUB * CHUNK;
  static constexpr int STAGES = 6;
  static constexpr int SMEM = STAGES * SB + 1024 + 512;
  static constexpr uint32_t IDESC = ptx::idesc_make(PREC == LRDM_BF16X3 ? 1 : 2, 256, 256);
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

template <int PREC>
__device__ __forceinline__ void issue_g2p_mmas(uint32_t d, uint32_t sa, uint32_t first) {
  using C = G2PCfg<PREC>;
  constexpr int PARTS = Tr<PREC>::PARTS;
  const uint32_t a0 = sa, a1 = sa + TILE_A;
  const uint32_t b0 = sa + PARTS * TILE_A, b1 = b0 + C::TILE_B;
#pragma unroll
  for (int kk = 0; kk < KSTEPS; ++kk) {
    const uint32_t off = kk * 32;
    const uint32_t acc = (first && kk == 0) ? 0u : 1u;
    if (PREC == LRDM_BF16X3) {
      ptx::mma_f16_pair(d, ptx::desc_k_sw64(a0 + off), ptx::desc_k_sw64(b0 + off), C::IDESC, acc);
      ptx::mma_f16_pair(d, ptx::desc_k_sw64(a0 + off), ptx::desc_k_sw64(b1 + off), C::IDESC, 1);
      ptx::mma_f16_pair(d, ptx::desc_k_sw64(a1 + off), ptx::desc_k_sw64(b0 + off), C::IDESC, 1);
    } else {
      ptx::mma_tf32_pair(d, ptx::desc_k_sw64(a0 + off), ptx::desc_k_sw64(b0 + off), C::IDESC, acc);
    }
  }
}

// Launched in clusters of two CTAs.
template <int PREC>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_gemm2_pair(const __grid_constant__ G2Params P) {
  using C = G2PCfg<PREC>;
  constexpr int STAGES = C::STAGES, PARTS = C::PARTS, BK = C::BK, SB = C::SB, BN2 = C::BN2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Bars B = carve<STAGES>(smem + STAGES * SB);   // ready[] serves as the relayed full barrier
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = P.begin[P.nslot];
  const int rank = (int)ptx::cluster_ctarank();
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&B.full[s], 1);
      ptx::mbar_init(&B.empty[s], 1);
      ptx::mbar_init(&B.ready[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&B.acc_full[a], 1);
      ptx::mbar_init(&B.acc_empty[a], 8);
    }
    ptx::mbar_init(B.drain, 1);
    *B.abort = 0;
    ptx::fence_barrier_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 1) {
    ptx::tmem_alloc_pair(B.tmem_slot, 2 * BN2);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();
  ptx::tc_fence_after();
  const uint32_t tmem = *B.tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    for (int q = 0; q < P.nslot; ++q) {
      const TcProblem* pr = P.probs + P.pid[q];
      ptx::tmap_acquire(&pr->g2a0);
      ptx::tmap_acquire(&pr->g2b0);
      if (PARTS == 2) {
        ptx::tmap_acquire(&pr->g2a1);
        ptx::tmap_acquire(&pr->g2b1);
      }
    }
    int s = 0;
    uint32_t ph = 0;
    int pending[STAGES];
    for (int i = 0; i < STAGES; ++i) pending[i] = -1;
    bool align = P.sync != nullptr;
    int round = 0;
    for (int item = pair; item < items; item += npairs, ++round) {
      if (align && round > 0 &&
          !ptx::counter_wait_geq(P.sync, round_target(round - 1, items, npairs, 2), ALIGN_NS))
        align = false;
      int q, k, R2, jp, j0, j1;
      const TcProblem* pr = g2_item<BN2>(P, item, q, k, R2, jp, j0, j1);
      const int ns_pad = pr->ns_pad;
      const int rb = 2 * R2 + rank;                       // this CTA's 128-row block (past the end: zero fill)
      bool ok = true;
      for (int jj = j0; jj < j1 && ok; ++jj) {
        const int J = g2_tile(P, q, jj);
        const int nch = min((J + 1) * BN2, ns_pad) / (BK * C::SUB);
        for (int ic = 0; ic < nch; ++ic) {
          if (!wait1(&B.empty[s], ph ^ 1, B, P.status)) { ok = false; break; }
          ptx::mbar_arrive_expect_tx(&B.full[s], SB);
#pragma unroll
          for (int c = 0; c < C::SUB; ++c) {
            uint8_t* st = smem + s * SB + c * C::CHUNK;
            const int i0 = (ic * C::SUB + c) * BK;
            ptx::tma_load_2d(st, &pr->g2a0, &B.full[s], i0, rb * BM);
            if (PARTS == 2) ptx::tma_load_2d(st + TILE_A, &pr->g2a1, &B.full[s], i0, rb * BM);
            ptx::tma_load_3d(st + PARTS * TILE_A, &pr->g2b0, &B.full[s], i0, J * BN2 + rank * 128, k);
            if (PARTS == 2)
              ptx::tma_load_3d(st + PARTS * TILE_A + C::TILE_B, &pr->g2b1, &B.full[s], i0,
                               J * BN2 + rank * 128, k);
          }
          pending[s] = (int)ph;
          if (++s == STAGES) { s = 0; ph ^= 1; }
        }
      }
      if (!ok) break;
      if (P.sync) ptx::counter_add_release(P.sync, 1);
    }
    for (int i = 0; i < STAGES; ++i)
      if (pending[i] >= 0) wait_drain(&B.full[i], (uint32_t)pending[i]);
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- MMA issuer (even CTA) ----------------
    int s = 0, a = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    for (int item = pair; item < items && ok; item += npairs) {
      int q, k, R2, jp, j0, j1;
      const TcProblem* pr = g2_item<BN2>(P, item, q, k, R2, jp, j0, j1);
      const int ns_pad = pr->ns_pad;
      for (int jj = j0; jj < j1 && ok; ++jj) {
        const int J = g2_tile(P, q, jj);
        if (!wait1(&B.acc_empty[a], aph ^ 1, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(a * BN2);
        const int nch = min((J + 1) * BN2, ns_pad) / (BK * C::SUB);
        for (int ic = 0; ic < nch; ++ic) {
          if (!wait1(&B.full[s], ph, B, P.status) || !wait1(&B.ready[s], ph, B, P.status)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
#pragma unroll
          for (int c = 0; c < C::SUB; ++c)
            issue_g2p_mmas<PREC>(d, ptx::smem_u32(smem + s * SB + c * C::CHUNK), ic == 0 && c == 0);
          ptx::mma_commit_pair_mc(&B.empty[s], PAIR_MASK);
          if (++s == STAGES) { s = 0; ph ^= 1; }
        }
        if (!ok) break;
        ptx::mma_commit_pair_mc(&B.acc_full[a], PAIR_MASK);
        if (++a == 2) { a = 0; aph ^= 1; }
      }
    }
    ptx::mma_commit_pair(B.drain);
    wait_drain(B.drain, 0);
  } else if (warp == 1 && lane == 0) {
    // ---------------- stage relay (odd CTA): its stages landed -> even CTA ----------------
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int item = pair; item < items && ok; item += npairs) {
      int q, k, R2, jp, j0, j1;
      const TcProblem* pr = g2_item<BN2>(P, item, q, k, R2, jp, j0, j1);
      const int ns_pad = pr->ns_pad;
      for (int jj = j0; jj < j1 && ok; ++jj) {
        const int J = g2_tile(P, q, jj);
        const int nch = min((J + 1) * BN2, ns_pad) / (BK * C::SUB);
        for (int ic = 0; ic < nch; ++ic) {
          if (!wait1(&B.full[s], ph, B, P.status)) { ok = false; break; }
          ptx::mbar_arrive_cluster(&B.ready[s], 0);
          if (++s == STAGES) { s = 0; ph ^= 1; }
        }
      }
    }
  } else if (warp >= 2) {
    // ---------------- row-dot epilogue (both CTAs; TMEM lane quarter = warp % 4) ----------------
    const int lq = warp & 3;
    const int row = lq * 32 + lane;
    int a = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int item = pair; item < items && ok; item += npairs) {
      int q, k, R2, jp, j0, j1;
      const TcProblem* pr = g2_item<BN2>(P, item, q, k, R2, jp, j0, j1);
      const int ns_pad = pr->ns_pad;
      const long long Ng = pr->Ng;
      const long long r = (long long)(2 * R2 + rank) * BM + row;
      double acc_row = 0.0;
      for (int jj = j0; jj < j1; ++jj) {
        const int J = g2_tile(P, q, jj);
        if (!waitw(&B.acc_full[a], aph, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(a * BN2);
        const float part = g2_tile_dot<PREC, BN2>(tb, J, r, Ng, ns_pad, pr->psi0, pr->psi1);
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive_cluster(&B.acc_empty[a], 0);
        acc_row += (double)part;
        if (++a == 2) { a = 0; aph ^= 1; }
      }
      if (!ok) break;
      g2_store(P, pr, q, k, jp, r, acc_row);
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, 2 * BN2);
  }
}

// ===========================================================================
// GEMM1: projection, direction weights applied on the way into tensor memory
// ===========================================================================
//
// One work item = one 128 x 128 tile (I <= J) of X for a pair of directions
// (k0, k0 + 1), reduced over the whole grid.  Per stage the TMA brings the
// raw Psi^T rows of block I (A) and block J (B) and both directions' weights;
// eight warps form a_k o A for the two directions, split it into bf16 hi / lo
// (or round it to TF32) and store it in tensor memory, from where the MMAs
// read their A operand (B stays in shared memory).  One A / B load thus
// serves two directions, and shared memory sees no write-back of the
// weighted tile.
//
// The tensor cores' FP32 accumulation truncates, and over a reduction of
// 10^5-10^6 rows that bias reaches ~1e-3 of the result; so the reduction is
// segmented: each segment of SEG stages (1024 rows) accumulates from zero in
// TMEM, after which the same eight warps add it into FP32 running sums held
// in registers (round-to-nearest) before the next segment starts.
//
// TMEM columns: [0, 256) the accumulators of the two directions (128 each);
// [256, 512) the weighted-A ring, one slot of 2 x ACOLS columns per stage.

// Warps 0-7 (warpgroups 0, 1): weighting + accumulation, 224 registers each
// after reallocation; warpgroup 2: warp 8 TMA, warp 9 MMA and TMEM owner,
// warps 10-11 idle, 56 registers each.  Launch: 384 x 168 = 64512 registers =
// 256 x 224 + 128 x 56; per SM sub-partition (warps w, w + 4, w + 8):
// 2 x 32 x 224 + 32 x 56 = 16128 <= 16384.
constexpr int G1_THREADS = 384;
constexpr int G1_REG_MATH = 224, G1_REG_CTRL = 56;
static_assert(256 * G1_REG_MATH + 128 * G1_REG_CTRL == G1_THREADS * 168, "register split");
constexpr int G1_BN = 128;              // square-tile width (j) = tile height (i)
constexpr int G1_TILE = G1_BN * ROWB;   // 8 KB per operand part (128 rows x 64 bytes)
constexpr int G1_ACOL = 256;            // first TMEM column of the weighted-A ring

// NB = MMA N: 128 -> 128 x 128 tiles (I <= J), one or two directions per tile,
// the accumulators of the two directions side by side; 256 -> 128 x 256
// tiles (128-row blocks I below the end of 256-wide block J), one direction.
template <int PREC, int NB>
struct G1Cfg {
  static constexpr int PARTS = Tr<PREC>::PARTS, BK = Tr<PREC>::BK;
  // grid-row chunks of BK rows per stage: TF32 takes two 16-row chunks (the
  // operand layouts' box), so that a stage holds four MMAs as BF16x3's holds six
  static constexpr int SUB = PREC == LRDM_TF32 ? 2 : 1;
  static constexpr int STAGES = 4;
  static constexpr int MAXD = NB == 256 ? 1 : 2;               // directions per tile at most
  // TMEM columns of one direction's weighted A per stage: bf16 packs two
  // elements per column and has two parts (hi, lo); tf32 one element per column
  static constexpr int ACOLS = BK * SUB;
  static constexpr int SLOT = MAXD * ACOLS;
  static constexpr int A_CHUNK = BM * BK * 4;                   // FP32 A rows of one chunk
  static constexpr int A_BYTES = A_CHUNK * SUB;
  static constexpr int B_TILE = NB * ROWB;                      // one part of the B rows of one chunk
  static constexpr int B_CHUNK = PARTS * B_TILE;
  static constexpr int B_OFF = A_BYTES;
  static constexpr int SC_OFF = B_OFF + SUB * B_CHUNK;
  static constexpr int STRIDE = SC_OFF + 1024;                  // 1024-aligned stages
  static constexpr int SMEM = STAGES * STRIDE + 1024 + 512;
  static constexpr int SEG = 1024 / (BK * SUB);                  // stages per accumulation segment
  static constexpr int LAG = STAGES - 1;                         // stages weighted ahead of a flush
  static constexpr uint32_t IDESC = ptx::idesc_make(PREC == LRDM_BF16X3 ? 1 : 2, BM, NB);
  static_assert(G1_ACOL + STAGES * SLOT <= 512, "TMEM budget");
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
  static_assert(LAG <= STAGES, "flush lag");
};

struct G1Params {
  const TcProblem* probs;
  int nslot;
  int begin[TC_MAX_SLOTS + 1];
  int pid[TC_MAX_SLOTS];
  int K[TC_MAX_SLOTS];
  float* X[TC_MAX_SLOTS];           // [nsplit][K][ns_pad][ns_pad] per slot
  int nsplit[TC_MAX_SLOTS];         // grid-row ranges per slot (partial X summed by the consumers)
  int dpt;                          // directions per tile (1 or 2)
  int nch_lim;                      // > 0: reduce over the first nch_lim stages only (tuning)
  int stall;                        // test only: CTA 0 never publishes its first weighted stage
  int* status;
  unsigned* sync;                   // pair form: round counter (zero at launch), or null
};

// Stages of the grid reduction: chunks of BK rows (nch_lim caps them for
// tuning), SUB chunks per stage.
template <int SUB>
__device__ __forceinline__ int g1_nch(const G1Params& P, const TcProblem* pr) {
  return (P.nch_lim > 0 ? min(P.nch_lim, pr->nch) : pr->nch) / SUB;
}

// Stages [rb, re) of row range `split` of slot q.
template <int SUB>
__device__ __forceinline__ void g1_range(const G1Params& P, const TcProblem* pr, int q, int split,
                                         int& rb, int& re) {
  const long long n = g1_nch<SUB>(P, pr);
  rb = (int)(n * split / P.nsplit[q]);
  re = (int)(n * (split + 1) / P.nsplit[q]);
}

// Item -> slot q, row range `split`, first direction k0, directions nd, tile
// (I, J).  Row ranges run slowest (each is a full set of items over its part
// of the grid; small K is split so that enough items exist); direction
// groups run fastest: the items of one tile run side by side on different SMs
// and stream the same Psi^T rows through L2; tiles go column by column, so
// neighbouring tiles share their B rows.  NB = 128: column J holds I = 0..J;
// NB = 256: column J (256 wide) holds the 128-row blocks I < min(2 J + 2, nI).
template <int NB>
__device__ __forceinline__ const TcProblem* g1_item(const G1Params& P, int item, int& q, int& k0,
                                                    int& nd, int& I, int& J, int& split) {
  q = find_slot(P.begin, P.nslot, item);
  const TcProblem* pr = P.probs + P.pid[q];
  int idx = item - P.begin[q];
  const int K = P.K[q], dpt = NB == 256 ? 1 : P.dpt;
  const int npair = (K + dpt - 1) / dpt;
  const int per_split = (NB == 256 ? pr->ntiles_w : pr->ntiles) * npair;
  split = idx / per_split;                  // row range of the grid reduction (outermost)
  idx -= split * per_split;
  int t = idx / npair;
  const int pp = idx - t * npair;
  k0 = dpt * pp;
  nd = min(dpt, K - k0);
  int j = 0;
  if (NB == 256) {
    const int nI = pr->nI;
    for (;;) {
      const int cnt = min(2 * (j + 1), nI);
      if (t < cnt) break;
      t -= cnt;
      ++j;
    }
  } else {
    while (t > j) {
      t -= j + 1;
      ++j;
    }
  }
  J = j;
  I = t;
  return pr;
}

// The weighted A operand of one stage for this thread's row: elements
// [BK/2 h, BK/2 h + BK/2) of the FP32 row times each direction's weights,
// split into bf16 hi / lo (or rounded to TF32) and stored at TMEM address ta
// (this warp's lane quarter, first column of the stage's slot).  Packed FP32
// pair arithmetic (two elements per instruction).
template <int PREC, class C>
__device__ __forceinline__ void weight_stage_c(uint32_t st, int row, int h, int nd, uint32_t ta) {
  if (PREC == LRDM_BF16X3) {
    // A rows of 32 FP32 = 128 bytes, 128-byte swizzle: chunk c sits at c ^ (row % 8)
    const uint32_t ra = st + row * 128;
    const int sw = row & 7;
    uint64_t xp[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint4 v = ptx::lds128(ra + (((4 * h + u) ^ sw) << 4));
      xp[2 * u] = ptx::f2_pack(v.x, v.y);
      xp[2 * u + 1] = ptx::f2_pack(v.z, v.w);
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (d >= nd) break;
      const uint32_t sc = st + C::SC_OFF + d * C::BK * C::SUB * 4 + h * 16 * 4;
      uint32_t oh[8], ol[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint4 w = ptx::lds128(sc + u * 16);
        const uint64_t y0 = ptx::f2_mul(xp[2 * u], ptx::f2_pack(w.x, w.y));
        const uint64_t y1 = ptx::f2_mul(xp[2 * u + 1], ptx::f2_pack(w.z, w.w));
        const uint32_t h0 = ptx::bf2_from_f2(y0), h1 = ptx::bf2_from_f2(y1);
        oh[2 * u] = h0;
        oh[2 * u + 1] = h1;
        ol[2 * u] = ptx::bf2_from_f2(ptx::f2_sub(y0, ptx::f2_from_bf2(h0)));
        ol[2 * u + 1] = ptx::bf2_from_f2(ptx::f2_sub(y1, ptx::f2_from_bf2(h1)));
      }
      ptx::tmem_st8(ta + d * C::ACOLS + h * 8, oh);          // hi: columns [0, 16) of the direction
      ptx::tmem_st8(ta + d * C::ACOLS + 16 + h * 8, ol);     // lo: columns [16, 32)
    }
  } else {
    // per chunk c of 16 grid rows: A rows of 16 FP32 = 64 bytes, 64-byte
    // swizzle: 16-byte unit u sits at u ^ ((row / 2) % 4)
#pragma unroll
    for (int c = 0; c < C::SUB; ++c) {
    const uint32_t ra = st + c * C::A_CHUNK + row * ROWB;
    const int sw = (row >> 1) & 3;
    uint64_t xp[4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint4 v = ptx::lds128(ra + (((2 * h + u) ^ sw) << 4));
      xp[2 * u] = ptx::f2_pack(v.x, v.y);
      xp[2 * u + 1] = ptx::f2_pack(v.z, v.w);
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (d >= nd) break;
      const uint32_t sc = st + C::SC_OFF + d * C::BK * C::SUB * 4 + c * C::BK * 4 + h * 8 * 4;
      uint32_t o[8];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const uint4 w = ptx::lds128(sc + u * 16);
        const uint64_t y0 = ptx::f2_mul(xp[2 * u], ptx::f2_pack(w.x, w.y));
        const uint64_t y1 = ptx::f2_mul(xp[2 * u + 1], ptx::f2_pack(w.z, w.w));
        o[4 * u] = __float_as_uint(tf32_round(__uint_as_float((uint32_t)y0)));
        o[4 * u + 1] = __float_as_uint(tf32_round(__uint_as_float((uint32_t)(y0 >> 32))));
        o[4 * u + 2] = __float_as_uint(tf32_round(__uint_as_float((uint32_t)y1)));
        o[4 * u + 3] = __float_as_uint(tf32_round(__uint_as_float((uint32_t)(y1 >> 32))));
      }
      ptx::tmem_st8(ta + d * C::ACOLS + c * C::BK + h * 8, o);
    }
    }
  }
}

template <int PREC, int NB>
__device__ __forceinline__ void weight_stage(uint32_t st, int row, int h, int nd, uint32_t ta) {
  weight_stage_c<PREC, G1Cfg<PREC, NB>>(st, row, h, nd, ta);
}

// The MMAs of one stage: for each direction d, D_d (+)= A'_d B^T over the
// stage's BK grid rows (three bf16 products for the split form).
template <int PREC, int NB>
__device__ __forceinline__ void issue_g1_mmas(uint32_t tmem, uint32_t aslot, uint32_t sb, int nd,
                                              bool first) {
  using C = G1Cfg<PREC, NB>;
#pragma unroll
  for (int d = 0; d < C::MAXD; ++d) {
    if (d >= nd) break;
    const uint32_t dt = tmem + d * G1_BN;
    const uint32_t at = tmem + aslot + d * C::ACOLS;
#pragma unroll
    for (int c = 0; c < C::SUB; ++c) {        // chunks of BK grid rows
      const uint32_t bc = sb + c * C::B_CHUNK;
#pragma unroll
      for (int kk = 0; kk < KSTEPS; ++kk) {   // 32-byte K steps along the swizzled B row
        const uint32_t acc = (first && c == 0 && kk == 0) ? 0u : 1u;
        const uint64_t b0 = ptx::desc_k_sw64(bc + kk * 32);
        if (PREC == LRDM_BF16X3) {
          const uint64_t b1 = ptx::desc_k_sw64(bc + C::B_TILE + kk * 32);
          ptx::mma_f16_ta(dt, at + kk * 8, b0, C::IDESC, acc);        // hi x hi
          ptx::mma_f16_ta(dt, at + kk * 8, b1, C::IDESC, 1);          // hi x lo
          ptx::mma_f16_ta(dt, at + 16 + kk * 8, b0, C::IDESC, 1);     // lo x hi
        } else {
          ptx::mma_tf32_ta(dt, at + c * C::BK + kk * 8, b0, C::IDESC, acc);
        }
      }
    }
  }
}

// ---- the roles of k_gemm1_tc ----

template <int PREC, int NB>
__device__ __forceinline__ void g1_producer(const G1Params& P, uint8_t* smem, const Bars& B, int items) {
  using C = G1Cfg<PREC, NB>;
  constexpr int STAGES = C::STAGES, PARTS = C::PARTS, BK = C::BK, SB = C::STRIDE;
  for (int q = 0; q < P.nslot; ++q) {
    const TcProblem* pr = P.probs + P.pid[q];
    ptx::tmap_acquire(&pr->g1a);
    ptx::tmap_acquire(&pr->g1b0);
    if (PARTS == 2) ptx::tmap_acquire(&pr->g1b1);
  }
  int s = 0;
  uint32_t ph = 0;
  int pending[STAGES];
  for (int i = 0; i < STAGES; ++i) pending[i] = -1;
  bool ok = true;
  for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
    int q, k0, nd, I, J, sp;
    const TcProblem* pr = g1_item<NB>(P, item, q, k0, nd, I, J, sp);
    int rb, re;
    g1_range<C::SUB>(P, pr, q, sp, rb, re);
    const float* w0 = pr->a + (long long)k0 * pr->a_stride;
    const long long wstride = pr->a_stride;
    const CUtensorMap *ma = &pr->g1a, *mb0 = &pr->g1b0, *mb1 = &pr->g1b1;
    constexpr int SUB = C::SUB;
    const uint32_t tx = C::A_BYTES + SUB * C::B_CHUNK + nd * BK * SUB * 4;
    for (int rc = rb; rc < re; ++rc) {
      if (!wait1(&B.empty[s], ph ^ 1, B, P.status)) { ok = false; break; }
      uint8_t* st = smem + s * SB;
      ptx::mbar_arrive_expect_tx(&B.full[s], tx);
#pragma unroll
      for (int c = 0; c < SUB; ++c) {
        const int ch = rc * SUB + c;           // chunk of BK grid rows
        ptx::tma_load_4d(st + c * C::A_CHUNK, ma, &B.full[s], 0, 0, ch, I);
        // B rows: NB / 128 consecutive state blocks (a block past the last one
        // of the matrix reads the zero fill; those columns are never stored)
#pragma unroll
        for (int hb = 0; hb < NB / 128; ++hb) {
          uint8_t* bd = st + C::B_OFF + c * C::B_CHUNK + hb * G1_TILE;
          ptx::tma_load_4d(bd, mb0, &B.full[s], 0, 0, ch, J * (NB / 128) + hb);
          if (PARTS == 2) ptx::tma_load_4d(bd + C::B_TILE, mb1, &B.full[s], 0, 0, ch, J * (NB / 128) + hb);
        }
      }
      for (int d = 0; d < nd; ++d)
        ptx::bulk_load(st + C::SC_OFF + d * BK * SUB * 4, w0 + d * wstride + (long long)rc * BK * SUB,
                       BK * SUB * 4, &B.full[s]);
      pending[s] = (int)ph;
      if (++s == STAGES) { s = 0; ph ^= 1; }
    }
  }
  for (int i = 0; i < STAGES; ++i)
    if (pending[i] >= 0) wait_drain(&B.full[i], (uint32_t)pending[i]);
}

template <int PREC, int NB>
__device__ __forceinline__ void g1_mma(const G1Params& P, uint8_t* smem, const Bars& B, int items,
                                       uint32_t tmem) {
  using C = G1Cfg<PREC, NB>;
  constexpr int STAGES = C::STAGES, SB = C::STRIDE, SEG = C::SEG;
  int s = 0;
  uint32_t ph = 0, aph = 0;
  bool ok = true;
  for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
    int q, k0, nd, I, J, sp;
    const TcProblem* pr = g1_item<NB>(P, item, q, k0, nd, I, J, sp);
    int rb, re;
    g1_range<C::SUB>(P, pr, q, sp, rb, re);
    const int nseg = (re - rb + SEG - 1) / SEG;
    for (int sg = 0; sg < nseg && ok; ++sg) {
      if (!wait1(&B.acc_empty[0], aph ^ 1, B, P.status)) { ok = false; break; }
      ptx::tc_fence_after();
      const int r0 = rb + sg * SEG, r1 = min(re, r0 + SEG);
      for (int rc = r0; rc < r1; ++rc) {
        if (!wait1(&B.ready[s], ph, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        issue_g1_mmas<PREC, NB>(tmem, (uint32_t)(G1_ACOL + s * C::SLOT),
                            ptx::smem_u32(smem + s * SB) + C::B_OFF, nd, rc == r0);
        ptx::mma_commit(&B.empty[s]);
        if (++s == STAGES) { s = 0; ph ^= 1; }
      }
      if (!ok) break;
      ptx::mma_commit(&B.acc_full[0]);
      aph ^= 1;
    }
  }
  ptx::mma_commit(B.drain);
  wait_drain(B.drain, 0);
}

// Weighting into tensor memory, segment accumulation and the tile epilogue
// (warps 0-7; warp w serves TMEM lane quarter w % 4 and element half /
// direction w / 4).
template <int PREC, int NB>
__device__ __forceinline__ void g1_math(const G1Params& P, uint8_t* smem, const Bars& B, int items,
                                        uint32_t tmem, int warp, int lane) {
  using C = G1Cfg<PREC, NB>;
  constexpr int STAGES = C::STAGES, SB = C::STRIDE, SEG = C::SEG, LAG = C::LAG;
  const int lq = warp & 3;
  const int h = warp >> 2;
  const int row = lq * 32 + lane;
  const uint32_t tq = tmem + ((uint32_t)(lq * 32) << 16);
  int s = 0;
  uint32_t ph = 0, aph = 0;
  bool ok = true;
  float sum[128];
  // test only: the MMA thread of CTA 0 then waits for a stage that is never
  // published, and its bounded wait ends the launch with a timeout status
  bool stall = P.stall != 0 && blockIdx.x == 0;
  for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
    int q, k0, nd, I, J, sp;
    const TcProblem* pr = g1_item<NB>(P, item, q, k0, nd, I, J, sp);
    int rb, re;
    g1_range<C::SUB>(P, pr, q, sp, rb, re);
    const int ns = pr->ns, ns_pad = pr->ns_pad;
    const int nseg = (re - rb + SEG - 1) / SEG;
#pragma unroll
    for (int c = 0; c < 128; ++c) sum[c] = 0.f;
    int flushed = 0;                      // segments already added into sum[]
    for (int rc = rb; rc < re; ++rc) {
      if (!waitw(&B.full[s], ph, B, P.status)) { ok = false; break; }
      weight_stage<PREC, NB>(ptx::smem_u32(smem + s * SB), row, h, nd,
                         tq + (uint32_t)(G1_ACOL + s * C::SLOT));
      ptx::tmem_wait_st();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0 && !stall) ptx::mbar_arrive(&B.ready[s]);
      stall = false;
      if (++s == STAGES) { s = 0; ph ^= 1; }
      // add a finished segment into the running sums once the weighting is
      // LAG stages past its end (those stages are ready when the MMAs resume)
      const int ready_seg = (rc - rb + 1 - LAG) / SEG;
      const bool last = rc + 1 == re;
      while (flushed < nseg && (flushed < ready_seg || last)) {
        if (!waitw(&B.acc_full[0], aph, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        if (NB == 256 || h < nd) {        // columns [128 h, 128 h + 128) of the accumulators
          const uint32_t ta = tq + (uint32_t)(h * 128);
#pragma unroll
          for (int c8 = 0; c8 < 8; ++c8) {
            float v[16];
            ptx::tmem_ld16(ta + c8 * 16, v);
#pragma unroll
            for (int e = 0; e < 16; ++e) sum[c8 * 16 + e] += v[e];
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&B.acc_empty[0]);
        aph ^= 1;
        ++flushed;
      }
      if (!ok) break;
    }
    if (!ok) break;
    // epilogue: X[i][j] and X[j][i] for i <= j of this tile; NB = 128: the
    // columns of direction k0 + h, NB = 256: columns 128 h.. of direction k0
    const int i = I * G1_BN + row;
    if ((NB == 256 || h < nd) && i < ns) {
      float* Xk = P.X[q] + ((long long)sp * P.K[q] + k0 + (NB == 256 ? 0 : h)) * ns_pad * ns_pad;
      const int j0 = J * NB + (NB == 256 ? h * 128 : 0);
#pragma unroll
      for (int c = 0; c < 128; ++c) {
        const int j = j0 + c;
        if (j >= i && j < ns) {
          Xk[(long long)i * ns_pad + j] = sum[c];
          Xk[(long long)j * ns_pad + i] = sum[c];
        }
      }
    }
  }
}

template <int PREC, int NB>
__global__ void __launch_bounds__(G1_THREADS, 1)
    k_gemm1_tc(const __grid_constant__ G1Params P) {
  using C = G1Cfg<PREC, NB>;
  constexpr int STAGES = C::STAGES, SB = C::STRIDE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Bars B = carve<STAGES>(smem + STAGES * SB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = P.begin[P.nslot];

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&B.full[s], 1);
      ptx::mbar_init(&B.empty[s], 1);
      ptx::mbar_init(&B.ready[s], 8);
    }
    ptx::mbar_init(&B.acc_full[0], 1);       // segment accumulated
    ptx::mbar_init(&B.acc_empty[0], 8);      // segment added to the running sums
    ptx::mbar_init(B.drain, 1);
    *B.abort = 0;
    ptx::fence_barrier_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 9) {
    ptx::tmem_alloc(B.tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *B.tmem_slot;
  if (warp >= 8) {
    ptx::setmaxnreg_dec<G1_REG_CTRL>();
    if (warp == 8 && lane == 0) g1_producer<PREC, NB>(P, smem, B, items);
    else if (warp == 9 && lane == 0) g1_mma<PREC, NB>(P, smem, B, items, tmem);
  } else {
    ptx::setmaxnreg_inc<G1_REG_MATH>();
    g1_math<PREC, NB>(P, smem, B, items, tmem, warp, lane);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 9) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512);
  }
}

// ===========================================================================
// GEMM1 on CTA pairs (cta_group::2): 256 x 256 tiles, one direction
// ===========================================================================
//
// A cluster of two CTAs on neighbouring SMs computes one 256 x 256 tile
// (I2, J) of X_k, I2 <= J in 256-state blocks, with M = 256 pair MMAs: CTA r
// of the pair loads (by TMA) and weights the FP32 Psi^T rows of the 128-state
// block 2 I2 + r into its own tensor memory (the A rows of the MMA), and loads
// the bf16 hi / lo (or TF32) Psi^T rows of the 128-state block 2 J + r (its
// half of the B rows).  One thread of the even CTA issues the MMAs; each CTA's
// tensor memory receives its 128 rows x 256 columns of the accumulator.  Per
// SM that halves the B rows loaded and read per MMA, against the 128 x 256
// single-CTA tile, for the same MMA work.
//
// Barriers: full[s] (each CTA, its own TMA bytes); ready[s] and acc_empty
// (even CTA, 16 arrivals: the 8 math warps of both CTAs); empty[s] and
// acc_full (both CTAs, one arrival each from the multicast MMA commit); drain
// (even CTA).  The reduction is segmented as in k_gemm1_tc.

template <int PREC>
struct G1PCfg {
  static constexpr int PARTS = Tr<PREC>::PARTS, BK = Tr<PREC>::BK;
  static constexpr int SUB = PREC == LRDM_TF32 ? 2 : 1;
  static constexpr int STAGES = 6;
  static constexpr int ACOLS = BK * SUB;
  static constexpr int SLOT = ACOLS;
  static constexpr int A_CHUNK = BM * BK * 4;
  static constexpr int A_BYTES = A_CHUNK * SUB;
  static constexpr int B_TILE = 128 * ROWB;                     // this CTA's 128 B rows, one part
  static constexpr int B_CHUNK = PARTS * B_TILE;
  static constexpr int B_OFF = A_BYTES;
  static constexpr int SC_OFF = B_OFF + SUB * B_CHUNK;
  static constexpr int STRIDE = SC_OFF + 1024;
  static constexpr int SMEM = STAGES * STRIDE + 1024 + 512;
  static constexpr int SEG = 1024 / (BK * SUB);
  static constexpr int LAG = STAGES - 1;
  static constexpr int TX = A_BYTES + SUB * B_CHUNK + BK * SUB * 4;   // TMA bytes per stage and CTA
  static constexpr uint32_t IDESC = ptx::idesc_make(PREC == LRDM_BF16X3 ? 1 : 2, 256, 256);
  static_assert(G1_ACOL + STAGES * SLOT <= 512, "TMEM budget");
  static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

// Pair item -> slot q, row range `split`, direction k, tile (I2, J): row
// ranges outermost, then tiles column by column (column J holds I2 = 0..J),
// directions fastest (the pairs working on one tile stream the same Psi^T
// rows through L2).
__device__ __forceinline__ const TcProblem* g1p_item(const G1Params& P, int item, int& q, int& k,
                                                     int& I2, int& J, int& split) {
  q = find_slot(P.begin, P.nslot, item);
  const TcProblem* pr = P.probs + P.pid[q];
  int idx = item - P.begin[q];
  const int K = P.K[q];
  const int per_split = pr->ntiles_p * K;
  split = idx / per_split;
  idx -= split * per_split;
  int t = idx / K;
  k = idx - t * K;
  int j = 0;
  while (t > j) {
    t -= j + 1;
    ++j;
  }
  J = j;
  I2 = t;
  return pr;
}

template <int PREC>
__device__ __forceinline__ void issue_g1p_mmas(uint32_t tmem, uint32_t aslot, uint32_t sb, bool first) {
  using C = G1PCfg<PREC>;
  const uint32_t at = tmem + aslot;
#pragma unroll
  for (int c = 0; c < C::SUB; ++c) {
    const uint32_t bc = sb + c * C::B_CHUNK;
#pragma unroll
    for (int kk = 0; kk < KSTEPS; ++kk) {
      const uint32_t acc = (first && c == 0 && kk == 0) ? 0u : 1u;
      const uint64_t b0 = ptx::desc_k_sw64(bc + kk * 32);
      if (PREC == LRDM_BF16X3) {
        const uint64_t b1 = ptx::desc_k_sw64(bc + C::B_TILE + kk * 32);
        ptx::mma_f16_ta_pair(tmem, at + kk * 8, b0, C::IDESC, acc);        // hi x hi
        ptx::mma_f16_ta_pair(tmem, at + kk * 8, b1, C::IDESC, 1);          // hi x lo
        ptx::mma_f16_ta_pair(tmem, at + 16 + kk * 8, b0, C::IDESC, 1);     // lo x hi
      } else {
        ptx::mma_tf32_ta_pair(tmem, at + c * C::BK + kk * 8, b0, C::IDESC, acc);
      }
    }
  }
}

template <int PREC>
__device__ __forceinline__ void g1p_producer(const G1Params& P, uint8_t* smem, const Bars& B, int items,
                                             int rank, int pair, int npairs) {
  using C = G1PCfg<PREC>;
  constexpr int STAGES = C::STAGES, PARTS = C::PARTS, BK = C::BK, SUB = C::SUB;
  for (int q = 0; q < P.nslot; ++q) {
    const TcProblem* pr = P.probs + P.pid[q];
    ptx::tmap_acquire(&pr->g1a);
    ptx::tmap_acquire(&pr->g1b0);
    if (PARTS == 2) ptx::tmap_acquire(&pr->g1b1);
  }
  int s = 0;
  uint32_t ph = 0;
  int pending[STAGES];
  for (int i = 0; i < STAGES; ++i) pending[i] = -1;
  bool ok = true;
  bool align = P.sync != nullptr;
  int round = 0;
  for (int item = pair; item < items && ok; item += npairs, ++round) {
    if (align && round > 0 && !ptx::counter_wait_geq(P.sync, round_target(round - 1, items, npairs, 2), ALIGN_NS))
      align = false;
    int q, k, I2, J, sp;
    const TcProblem* pr = g1p_item(P, item, q, k, I2, J, sp);
    int rb, re;
    g1_range<SUB>(P, pr, q, sp, rb, re);
    const float* w0 = pr->a + (long long)k * pr->a_stride;
    const int ia = 2 * I2 + rank, ib = 2 * J + rank;   // 128-state blocks (past the end: zero fill)
    for (int rc = rb; rc < re; ++rc) {
      if (!wait1(&B.empty[s], ph ^ 1, B, P.status)) { ok = false; break; }
      uint8_t* st = smem + s * C::STRIDE;
      ptx::mbar_arrive_expect_tx(&B.full[s], C::TX);
#pragma unroll
      for (int c = 0; c < SUB; ++c) {
        const int ch = rc * SUB + c;
        ptx::tma_load_4d(st + c * C::A_CHUNK, &pr->g1a, &B.full[s], 0, 0, ch, ia);
        uint8_t* bd = st + C::B_OFF + c * C::B_CHUNK;
        ptx::tma_load_4d(bd, &pr->g1b0, &B.full[s], 0, 0, ch, ib);
        if (PARTS == 2) ptx::tma_load_4d(bd + C::B_TILE, &pr->g1b1, &B.full[s], 0, 0, ch, ib);
      }
      ptx::bulk_load(st + C::SC_OFF, w0 + (long long)rc * BK * SUB, BK * SUB * 4, &B.full[s]);
      pending[s] = (int)ph;
      if (++s == STAGES) { s = 0; ph ^= 1; }
    }
    if (P.sync && ok) ptx::counter_add_release(P.sync, 1);     // this round's loads are issued
  }
  for (int i = 0; i < STAGES; ++i)
    if (pending[i] >= 0) wait_drain(&B.full[i], (uint32_t)pending[i]);
}

// The MMA thread's waits on barriers that both CTAs' math warps arrive on:
// the CTA-scope try_wait (which suspends the thread between polls; the
// cluster-scope form spins and takes issue slots from the math warps that
// share its sub-partition), paired with the default-semantics remote arrive.
__device__ __forceinline__ bool wait_cl(uint64_t* bar, uint32_t parity, const Bars& B, int* status) {
  return ptx::mbar_wait(bar, parity, B.abort, status, WAIT_NS, STATUS_TIMEOUT);
}

// MMA issue (even CTA of the pair only).
template <int PREC>
__device__ __forceinline__ void g1p_mma(const G1Params& P, uint8_t* smem, const Bars& B, int items,
                                        uint32_t tmem, int pair, int npairs) {
  using C = G1PCfg<PREC>;
  constexpr int STAGES = C::STAGES, SEG = C::SEG;
  int s = 0;
  uint32_t ph = 0, aph = 0;
  bool ok = true;
  for (int item = pair; item < items && ok; item += npairs) {
    int q, k, I2, J, sp;
    const TcProblem* pr = g1p_item(P, item, q, k, I2, J, sp);
    int rb, re;
    g1_range<C::SUB>(P, pr, q, sp, rb, re);
    const int nseg = (re - rb + SEG - 1) / SEG;
    for (int sg = 0; sg < nseg && ok; ++sg) {
      if (!wait_cl(&B.acc_empty[0], aph ^ 1, B, P.status)) { ok = false; break; }
      ptx::tc_fence_after();
      const int r0 = rb + sg * SEG, r1 = min(re, r0 + SEG);
      for (int rc = r0; rc < r1; ++rc) {
        if (!wait_cl(&B.ready[s], ph, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        issue_g1p_mmas<PREC>(tmem, (uint32_t)(G1_ACOL + s * C::SLOT),
                             ptx::smem_u32(smem + s * C::STRIDE) + C::B_OFF, rc == r0);
        ptx::mma_commit_pair_mc(&B.empty[s], PAIR_MASK);
        if (++s == STAGES) { s = 0; ph ^= 1; }
      }
      if (!ok) break;
      ptx::mma_commit_pair_mc(&B.acc_full[0], PAIR_MASK);
      aph ^= 1;
    }
  }
  ptx::mma_commit_pair(B.drain);
  wait_drain(B.drain, 0);
}

// Weighting into this CTA's tensor memory, segment accumulation and the tile
// epilogue (warps 0-7 of both CTAs; warp w serves TMEM lane quarter w % 4 and
// element half / accumulator column half w / 4).
template <int PREC>
__device__ __forceinline__ void g1p_math(const G1Params& P, uint8_t* smem, const Bars& B, int items,
                                         uint32_t tmem, int warp, int lane, int rank, int pair,
                                         int npairs) {
  using C = G1PCfg<PREC>;
  constexpr int STAGES = C::STAGES, SEG = C::SEG, LAG = C::LAG;
  const int lq = warp & 3;
  const int h = warp >> 2;
  const int row = lq * 32 + lane;
  const uint32_t tq = tmem + ((uint32_t)(lq * 32) << 16);
  int s = 0;
  uint32_t ph = 0, aph = 0;
  bool ok = true;
  float sum[128];
  bool stall = P.stall != 0 && blockIdx.x == 0;
  for (int item = pair; item < items && ok; item += npairs) {
    int q, k, I2, J, sp;
    const TcProblem* pr = g1p_item(P, item, q, k, I2, J, sp);
    int rb, re;
    g1_range<C::SUB>(P, pr, q, sp, rb, re);
    const int ns = pr->ns, ns_pad = pr->ns_pad;
    const int nseg = (re - rb + SEG - 1) / SEG;
#pragma unroll
    for (int c = 0; c < 128; ++c) sum[c] = 0.f;
    int flushed = 0;
    for (int rc = rb; rc < re; ++rc) {
      if (!waitw(&B.full[s], ph, B, P.status)) { ok = false; break; }
      weight_stage_c<PREC, C>(ptx::smem_u32(smem + s * C::STRIDE), row, h, 1,
                              tq + (uint32_t)(G1_ACOL + s * C::SLOT));
      ptx::tmem_wait_st();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0 && !stall) ptx::mbar_arrive_cluster(&B.ready[s], 0);
      stall = false;
      if (++s == STAGES) { s = 0; ph ^= 1; }
      const int ready_seg = (rc - rb + 1 - LAG) / SEG;
      const bool last = rc + 1 == re;
      while (flushed < nseg && (flushed < ready_seg || last)) {
        if (!waitw(&B.acc_full[0], aph, B, P.status)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t ta = tq + (uint32_t)(h * 128);
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
          float v[16];
          ptx::tmem_ld16(ta + c8 * 16, v);
#pragma unroll
          for (int e = 0; e < 16; ++e) sum[c8 * 16 + e] += v[e];
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive_cluster(&B.acc_empty[0], 0);
        aph ^= 1;
        ++flushed;
      }
      if (!ok) break;
    }
    if (!ok) break;
    const int i = (2 * I2 + rank) * BM + row;
    if (i < ns) {
      float* Xk = P.X[q] + ((long long)sp * P.K[q] + k) * ns_pad * ns_pad;
      const int j0 = J * 256 + h * 128;
#pragma unroll
      for (int c = 0; c < 128; ++c) {
        const int j = j0 + c;
        if (j >= i && j < ns) {
          Xk[(long long)i * ns_pad + j] = sum[c];
          Xk[(long long)j * ns_pad + i] = sum[c];
        }
      }
    }
  }
}

// Launched in clusters of two CTAs (an even number of CTAs, one per SM).
template <int PREC>
__global__ void __launch_bounds__(G1_THREADS, 1)
    k_gemm1_pair(const __grid_constant__ G1Params P) {
  using C = G1PCfg<PREC>;
  constexpr int STAGES = C::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const Bars B = carve<STAGES>(smem + STAGES * C::STRIDE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = P.begin[P.nslot];
  const int rank = (int)ptx::cluster_ctarank();
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&B.full[s], 1);
      ptx::mbar_init(&B.empty[s], 1);
      ptx::mbar_init(&B.ready[s], 16);
    }
    ptx::mbar_init(&B.acc_full[0], 1);
    ptx::mbar_init(&B.acc_empty[0], 16);
    ptx::mbar_init(B.drain, 1);
    *B.abort = 0;
    ptx::fence_barrier_init();
    ptx::fence_proxy_async_smem();
  }
  if (warp == 9) {
    ptx::tmem_alloc_pair(B.tmem_slot, 512);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();          // both CTAs' barriers initialised before any remote arrive
  ptx::tc_fence_after();
  const uint32_t tmem = *B.tmem_slot;
  if (warp >= 8) {
    ptx::setmaxnreg_dec<G1_REG_CTRL>();
    if (warp == 8 && lane == 0) g1p_producer<PREC>(P, smem, B, items, rank, pair, npairs);
    else if (warp == 9 && lane == 0 && rank == 0) g1p_mma<PREC>(P, smem, B, items, tmem, pair, npairs);
  } else {
    ptx::setmaxnreg_inc<G1_REG_MATH>();
    g1p_math<PREC>(P, smem, B, items, tmem, warp, lane, rank, pair, npairs);
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();          // the even CTA's MMAs into this CTA's memory are complete
  if (warp == 9) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc_pair(tmem, 512);
  }
}

// ===========================================================================
// host side
// ===========================================================================

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // the driver entry point is the same for every device; initialised once
  // (thread-safe static initialisation)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// Map of rank 2-4 over a row-major array; box inner extent = 64 bytes,
// 64-byte swizzle (matching desc_k_sw64).
bool make_map(CUtensorMap* m, const void* base, int elem_bytes, int rank, const uint64_t* dims,
              const uint64_t* strides_bytes, const uint32_t* box,
              CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_64B) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t gd[4];
  cuuint64_t gs[3];
  cuuint32_t bx[4], es[4] = {1, 1, 1, 1};
  for (int i = 0; i < rank; ++i) {
    gd[i] = dims[i];
    bx[i] = box[i];
  }
  for (int i = 0; i < rank - 1; ++i) gs[i] = strides_bytes[i];
  CUresult r = fn(m, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  rank, const_cast<void*>(base), gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Function attributes and device properties are per device: the records
// below are kept per device ordinal (cached values are plain queries, so two
// host threads that race on a first call store the same value).
constexpr int MAX_DEV = 64;

int cur_dev() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int num_sms() {
  static std::atomic<int> cache[MAX_DEV];
  const int dev = cur_dev();
  int n = dev >= 0 && dev < MAX_DEV ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (n <= 0) n = 148;
  if (dev >= 0 && dev < MAX_DEV) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// One bit per device: the kernel's dynamic shared-memory limit has been raised.
struct DevMask {
  std::atomic<unsigned long long> bits{0};
};

template <typename Kern>
cudaError_t set_smem(Kern k, int bytes, DevMask& done) {
  const int dev = cur_dev();
  const unsigned long long bit = dev >= 0 && dev < MAX_DEV ? 1ull << dev : 0ull;
  if (bit && (done.bits.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.bits.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Builds the descriptor of one (system, channel) for the tensor-core kernels.
template <int PREC>
bool build_problem(const Channel& c, const SysState& S, int ch, TcProblem& pr) {
  constexpr int BK = Tr<PREC>::BK;
  const int eb = PREC == LRDM_BF16X3 ? 2 : 4;
  memset(&pr, 0, sizeof(pr));
  // GEMM1: Psi^T tile-major [ns_pad/128][Ng_pad/BK][128][BK]: a box (A or B
  // operand of one stage) is one contiguous 8 KB tile.
  const void* t0 = PREC == LRDM_BF16X3 ? (const void*)c.psiT_hi : (const void*)c.psiT32;
  const void* t1 = PREC == LRDM_BF16X3 ? (const void*)c.psiT_lo : (const void*)c.psiT32;
  const void* ta = PREC == LRDM_BF16X3 ? (const void*)c.psiTf : (const void*)c.psiT32;
  const uint64_t d1[4] = {(uint64_t)BK, 128, (uint64_t)(S.Ng_pad / BK), (uint64_t)(c.ns_pad / 128)};
  const uint64_t s1[3] = {(uint64_t)BK * eb, (uint64_t)128 * BK * eb, (uint64_t)128 * S.Ng_pad * eb};
  const uint64_t sa[3] = {(uint64_t)BK * 4, (uint64_t)128 * BK * 4, (uint64_t)128 * S.Ng_pad * 4};
  const uint32_t bA1[4] = {(uint32_t)BK, 128, 1, 1};
  // FP32 A rows: BK * 4 bytes (128 for bf16 mode -> 128-byte swizzle, 64 for TF32)
  const CUtensorMapSwizzle swa = BK * 4 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  // GEMM2: Psi rows [Ng_pad][ns_pad] (A) and X'' [k_max][j][i] (B).
  const void* r0 = PREC == LRDM_BF16X3 ? (const void*)c.psiR_hi : (const void*)c.psiR32;
  const void* r1 = PREC == LRDM_BF16X3 ? (const void*)c.psiR_lo : (const void*)c.psiR32;
  const void* x0 = c.Xpp;
  const void* x1 = PREC == LRDM_BF16X3 ? c.Xpp_lo : c.Xpp;
  const uint64_t dA2[2] = {(uint64_t)c.ns_pad, (uint64_t)S.Ng_pad};
  const uint64_t sA2[1] = {(uint64_t)c.ns_pad * eb};
  const uint32_t bA2[2] = {(uint32_t)BK, (uint32_t)BM};
  const uint64_t dB2[3] = {(uint64_t)c.ns_pad, (uint64_t)c.ns_pad, (uint64_t)S.kmax};
  const uint64_t sB2[2] = {(uint64_t)c.ns_pad * eb, (uint64_t)c.ns_pad * c.ns_pad * eb};
  const uint32_t bB2[3] = {(uint32_t)BK, 128, 1};            // GEMM2 B: 128-row boxes
  if (!make_map(&pr.g1a, ta, 4, 4, d1, sa, bA1, swa) || !make_map(&pr.g1b0, t0, eb, 4, d1, s1, bA1) ||
      !make_map(&pr.g1b1, t1, eb, 4, d1, s1, bA1) ||
      !make_map(&pr.g2a0, r0, eb, 2, dA2, sA2, bA2) || !make_map(&pr.g2a1, r1, eb, 2, dA2, sA2, bA2) ||
      !make_map(&pr.g2b0, x0, eb, 3, dB2, sB2, bB2) || !make_map(&pr.g2b1, x1, eb, 3, dB2, sB2, bB2))
    return false;
  pr.Ng = S.Ng;
  pr.a_stride = (long long)S.nspin * S.Ng_pad;
  pr.a = static_cast<const float*>(S.a) + (size_t)ch * S.Ng_pad;
  pr.psi0 = r0;
  pr.psi1 = r1;
  pr.ns = c.ns;
  pr.ns_pad = c.ns_pad;
  pr.nI = c.ns_pad / BM;
  pr.NJ = (c.ns_pad + 255) / 256;        // GEMM2 j-tiles at the default width
  pr.ntiles = pr.nI * (pr.nI + 1) / 2;    // GEMM1 128 x 128 tiles with I <= J
  pr.ntiles_w = 0;                          // GEMM1 128 x 256 tiles (I below the end of J)
  for (int j = 0; 256 * j < c.ns_pad; ++j) pr.ntiles_w += 2 * (j + 1) < pr.nI ? 2 * (j + 1) : pr.nI;
  pr.ntiles_p = pr.NJ * (pr.NJ + 1) / 2;    // GEMM1 256 x 256 pair tiles with I <= J
  pr.nch = (int)(S.Ng_pad / BK);
  pr.nR = (int)(S.Ng_pad / BM);
  pr.kmax = S.kmax;
  return true;
}

// Slots in decreasing order of per-item cost (longest items first, so that a
// persistent grid's round-robin assignment ends evenly).
void order_slots(const TcEntry* e, int n, int gemm, int* order) {
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 1; i < n; ++i) {
    int t = order[i], j = i;
    auto cost = [&](int x) {
      const TcProblem& p = *e[x].host;
      return gemm == 1 ? (double)p.nch / (e[x].split > 1 ? e[x].split : 1) : (double)p.ns_pad * p.ns_pad;
    };
    while (j > 0 && cost(order[j - 1]) < cost(t)) {
      order[j] = order[j - 1];
      --j;
    }
    order[j] = t;
  }
}

template <int PREC, int NB>
cudaError_t gemm1_group(const TcEntry* e, int n, int* status, cudaStream_t st, const TcTune& t,
                        int nch_lim, int stall) {
  static DevMask attr;
  const int smem = G1Cfg<PREC, NB>::SMEM;
  cudaError_t err = set_smem(k_gemm1_tc<PREC, NB>, smem, attr);
  if (err != cudaSuccess) return err;
  const int dpt = NB == 256 ? 1 : (t.g1_dpt == 1 ? 1 : 2);
  for (int base = 0; base < n; base += TC_MAX_SLOTS) {
    const int m = n - base < TC_MAX_SLOTS ? n - base : TC_MAX_SLOTS;
    int order[TC_MAX_SLOTS];
    order_slots(e + base, m, 1, order);
    G1Params P;
    memset(&P, 0, sizeof(P));
    P.status = status;
    P.dpt = dpt;
    P.nch_lim = nch_lim;
    P.stall = base == 0 ? stall : 0;
    int items = 0, q = 0;
    for (int u = 0; u < m; ++u) {
      const TcEntry& x = e[base + order[u]];
      if (x.K <= 0) continue;
      P.probs = x.dev_base;
      P.pid[q] = x.pid;
      P.K[q] = x.K;
      P.X[q] = static_cast<float*>(x.X);
      P.nsplit[q] = x.split > 1 ? x.split : 1;
      P.begin[q] = items;
      items += (NB == 256 ? x.host->ntiles_w : x.host->ntiles) * ((x.K + dpt - 1) / dpt) * P.nsplit[q];
      ++q;
    }
    P.nslot = q;
    P.begin[q] = items;
    if (items == 0) continue;
    const int grid = items < num_sms() ? items : num_sms();
    k_gemm1_tc<PREC, NB><<<grid, G1_THREADS, smem, st>>>(P);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Clusters of two that fit on the device at once with the pair kernel's
// shared memory (one CTA per SM), per device.
// Clusters of two that fit on the device at once with a pair kernel's
// shared memory and block size (one CTA per SM), per device (cache: one
// entry per device for that kernel).
template <typename Kern>
int cluster_pairs(Kern kern, int smem, int threads, DevMask& attr, std::atomic<int>* cache,
                  const char* what) {
  const int dev = cur_dev();
  int n = dev >= 0 && dev < MAX_DEV ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  if (set_smem(kern, smem, attr) != cudaSuccess) {   // the occupancy query needs the shared-memory limit
    cudaGetLastError();
    return num_sms() / 2 - 2;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * (num_sms() / 2), 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = num_sms() / 2 - 2;
  }
  if (n > num_sms() / 2) n = num_sms() / 2;
  if (dev >= 0 && dev < MAX_DEV) cache[dev].store(n, std::memory_order_relaxed);
  // LRDM_DEBUG=1 in the environment reports the persistent grid of the pair kernels
  if (getenv("LRDM_DEBUG"))
    fprintf(stderr, "liblrdm: device %d: pair %s grid of %d CTA pairs (%d SMs)\n", dev, what, n, num_sms());
  return n;
}

template <int PREC>
struct PairKernels {
  static DevMask g1_attr, g2_attr;
  static std::atomic<int> g1_cache[MAX_DEV], g2_cache[MAX_DEV];
};
template <int PREC>
DevMask PairKernels<PREC>::g1_attr;
template <int PREC>
DevMask PairKernels<PREC>::g2_attr;
template <int PREC>
std::atomic<int> PairKernels<PREC>::g1_cache[MAX_DEV];
template <int PREC>
std::atomic<int> PairKernels<PREC>::g2_cache[MAX_DEV];

template <int PREC>
cudaError_t pair_attr() {
  return set_smem(k_gemm1_pair<PREC>, G1PCfg<PREC>::SMEM, PairKernels<PREC>::g1_attr);
}

template <int PREC>
int pair_clusters() {
  return cluster_pairs(k_gemm1_pair<PREC>, G1PCfg<PREC>::SMEM, G1_THREADS, PairKernels<PREC>::g1_attr,
                       PairKernels<PREC>::g1_cache, "projection");
}

template <int PREC>
int pair_clusters_g2() {
  return cluster_pairs(k_gemm2_pair<PREC>, G2PCfg<PREC>::SMEM, NTHREADS, PairKernels<PREC>::g2_attr,
                       PairKernels<PREC>::g2_cache, "response");
}

template <int PREC>
cudaError_t gemm1_pair_group(const TcEntry* e, int n, int* status, cudaStream_t st, int nch_lim,
                             int stall, unsigned* sync) {
  const int smem = G1PCfg<PREC>::SMEM;
  cudaError_t err = pair_attr<PREC>();
  if (err != cudaSuccess) return err;
  for (int base = 0; base < n; base += TC_MAX_SLOTS) {
    const int m = n - base < TC_MAX_SLOTS ? n - base : TC_MAX_SLOTS;
    int order[TC_MAX_SLOTS];
    order_slots(e + base, m, 1, order);
    G1Params P;
    memset(&P, 0, sizeof(P));
    P.status = status;
    P.dpt = 1;
    P.nch_lim = nch_lim;
    P.stall = base == 0 ? stall : 0;
    int items = 0, q = 0;
    long long len0 = -1;
    bool equal = true;                // all items of the launch equally long (round alignment)
    for (int u = 0; u < m; ++u) {
      const TcEntry& x = e[base + order[u]];
      if (x.K <= 0) continue;
      P.probs = x.dev_base;
      P.pid[q] = x.pid;
      P.K[q] = x.K;
      P.X[q] = static_cast<float*>(x.X);
      P.nsplit[q] = x.split > 1 ? x.split : 1;
      P.begin[q] = items;
      items += x.host->ntiles_p * x.K * P.nsplit[q];
      const long long nch = nch_lim > 0 && nch_lim < x.host->nch ? nch_lim : x.host->nch;
      const long long len = nch * 1024 / P.nsplit[q];
      if (len0 >= 0 && len != len0) equal = false;
      len0 = len;
      ++q;
    }
    P.nslot = q;
    P.begin[q] = items;
    if (items == 0) continue;
    P.sync = equal ? sync : nullptr;
    const int clusters = pair_clusters<PREC>();
    const int pairs = items < clusters ? items : clusters;
    if (P.sync && (err = cudaMemsetAsync(P.sync, 0, sizeof(unsigned), st)) != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * pairs, 1, 1);
    cfg.blockDim = dim3(G1_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if ((err = cudaLaunchKernelEx(&cfg, k_gemm1_pair<PREC>, P)) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Sum of a split GEMM2's part sums in part order, then as the unsplit
// epilogue: out = sum - v in the io dtype (out_is_io) or FP32 sum.
__global__ void k_g2_combine(const double* __restrict__ part, int nsplit, int K, long long Ng,
                             const void* __restrict__ v, long long v_stride, void* __restrict__ out,
                             long long out_stride, int out_io, int out_is_io) {
  const long long n = (long long)K * Ng;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / Ng);
    const long long r = i - (long long)k * Ng;
    double d = 0.0;
    for (int p = 0; p < nsplit; ++p) d += part[((long long)p * K + k) * Ng + r];
    const long long o = (long long)k * out_stride + r;
    if (out_is_io) {
      const long long ov = (long long)k * v_stride + r;
      if (out_io == LRDM_DTYPE_F64)
        static_cast<double*>(out)[o] = d - static_cast<const double*>(v)[ov];
      else
        static_cast<float*>(out)[o] = (float)(d - (double)static_cast<const float*>(v)[ov]);
    } else {
      static_cast<float*>(out)[o] = (float)d;
    }
  }
}

// j-tile parts of a GEMM2 problem with K directions.  Every CTA streams its
// row block's Psi rows once per j-tile; with one direction at N_s >= 2048 the
// row blocks of one wave (2 MB each in bf16 hi / lo) outgrow L2, where a
// group of directions would share each row block side by side.  Splitting
// each (row block, direction) item into parts over its j-tiles puts the parts
// of one row block side by side instead: 4 parts (2 when 4 do not balance).
// The tiles are dealt largest first to the part with the least work (tile J
// holds min((J + 1) BN2, ns_pad) states); since the round-robin item order
// gives each CTA the same part throughout, a split whose largest part exceeds
// the mean by more than 5 % is not used.  At two directions a split measured
// no faster than the pair sharing the row block.
int g2_partition(const TcProblem& pr, int K, int BN2, int* jb, unsigned char* jl) {
  const int NJ = (pr.ns_pad + BN2 - 1) / BN2;
  if (K != 1 || pr.ns_pad < 2048 || NJ > G2_MAX_NJ || pr.part == nullptr) return 1;
  for (int S = 4; S >= 2; S /= 2) {
    if (S > NJ || S * K > G2_MAX_SPLIT) continue;
    long long load[G2_MAX_SPLIT] = {0, 0, 0, 0};
    int owner[G2_MAX_NJ];
    for (int J = NJ - 1; J >= 0; --J) {
      int best = 0;
      for (int p = 1; p < S; ++p)
        if (load[p] < load[best]) best = p;
      owner[J] = best;
      load[best] += (long long)std::min((J + 1) * BN2, pr.ns_pad) + 64;   // + epilogue
    }
    long long mx = 0, tot = 0;
    for (int p = 0; p < S; ++p) {
      mx = std::max(mx, load[p]);
      tot += load[p];
    }
    if (20 * mx * S > 21 * tot) continue;              // max > 1.05 x mean
    int m = 0;
    for (int p = 0; p < S; ++p) {
      jb[p] = m;
      for (int J = 0; J < NJ; ++J)
        if (owner[J] == p) jl[m++] = (unsigned char)J;
    }
    jb[S] = m;
    return S;
  }
  return 1;
}

template <int PREC, int BN2>
cudaError_t gemm2_group(const TcEntry* e, int n, int out_io, int out_is_io, int* status,
                        cudaStream_t st, const TcTune& t, int nR_lim, int* launches, unsigned* sync) {
  static DevMask attr;
  const int smem = G2Cfg<PREC, BN2>::SMEM;
  cudaError_t err = set_smem(k_gemm2_tc<PREC, BN2>, smem, attr);
  if (err != cudaSuccess) return err;
  const int kg = t.g2_kgroup == 1 || t.g2_kgroup == 4 ? t.g2_kgroup : 2;
  for (int base = 0; base < n; base += TC_MAX_SLOTS) {
    const int m = n - base < TC_MAX_SLOTS ? n - base : TC_MAX_SLOTS;
    int order[TC_MAX_SLOTS];
    order_slots(e + base, m, 2, order);
    G2Params P;
    memset(&P, 0, sizeof(P));
    const TcProblem* hp[TC_MAX_SLOTS] = {};
    P.out_io = out_io;
    P.out_is_io = out_is_io;
    P.status = status;
    int items = 0, q = 0;
    for (int u = 0; u < m; ++u) {
      const TcEntry& x = e[base + order[u]];
      if (x.K <= 0) continue;
      P.probs = x.dev_base;
      P.pid[q] = x.pid;
      P.K[q] = x.K;
      P.kgroup[q] = x.K < kg ? x.K : kg;
      P.factor[q] = x.factor;
      P.v[q] = x.v;
      P.v_stride[q] = x.v_stride;
      P.out[q] = x.out;
      P.out_stride[q] = x.out_stride;
      P.nR[q] = nR_lim > 0 && nR_lim < x.host->nR ? nR_lim : x.host->nR;
      P.nsplit[q] = g2_partition(*x.host, x.K, BN2, P.jb[q], P.jl[q]);
      hp[q] = x.host;
      P.begin[q] = items;
      items += P.nR[q] * x.K * P.nsplit[q];
      ++q;
    }
    P.nslot = q;
    P.begin[q] = items;
    if (items == 0) continue;
    // round alignment only where every item has the same length: one problem, unsplit items
    P.sync = sync && q == 1 && P.nsplit[0] == 1 ? sync : nullptr;
    if (P.sync && (err = cudaMemsetAsync(P.sync, 0, sizeof(unsigned), st)) != cudaSuccess) return err;
    const int grid = items < num_sms() ? items : num_sms();
    k_gemm2_tc<PREC, BN2><<<grid, NTHREADS, smem, st>>>(P);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (launches) ++*launches;
    for (int u = 0; u < q; ++u) {
      if (P.nsplit[u] <= 1) continue;
      const long long nk = (long long)P.K[u] * hp[u]->Ng;
      const int blocks = (int)std::min<long long>((nk + 255) / 256, 4LL * num_sms());
      k_g2_combine<<<blocks, 256, 0, st>>>(hp[u]->part, P.nsplit[u], P.K[u], hp[u]->Ng, P.v[u],
                                           P.v_stride[u], P.out[u], P.out_stride[u], out_io, out_is_io);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      if (launches) ++*launches;
    }
  }
  return cudaSuccess;
}

template <int PREC>
cudaError_t gemm2_pair_group(const TcEntry* e, int n, int out_io, int out_is_io, int* status,
                             cudaStream_t st, const TcTune& t, int nR_lim, int* launches, unsigned* sync) {
  using C = G2PCfg<PREC>;
  cudaError_t err = set_smem(k_gemm2_pair<PREC>, C::SMEM, PairKernels<PREC>::g2_attr);
  if (err != cudaSuccess) return err;
  const int kg = t.g2_kgroup == 1 || t.g2_kgroup == 4 ? t.g2_kgroup : 2;
  for (int base = 0; base < n; base += TC_MAX_SLOTS) {
    const int m = n - base < TC_MAX_SLOTS ? n - base : TC_MAX_SLOTS;
    int order[TC_MAX_SLOTS];
    order_slots(e + base, m, 2, order);
    G2Params P;
    memset(&P, 0, sizeof(P));
    const TcProblem* hp[TC_MAX_SLOTS] = {};
    P.out_io = out_io;
    P.out_is_io = out_is_io;
    P.status = status;
    int items = 0, q = 0;
    for (int u = 0; u < m; ++u) {
      const TcEntry& x = e[base + order[u]];
      if (x.K <= 0) continue;
      P.probs = x.dev_base;
      P.pid[q] = x.pid;
      P.K[q] = x.K;
      P.kgroup[q] = x.K < kg ? x.K : kg;
      P.factor[q] = x.factor;
      P.v[q] = x.v;
      P.v_stride[q] = x.v_stride;
      P.out[q] = x.out;
      P.out_stride[q] = x.out_stride;
      const int nr = nR_lim > 0 && nR_lim < x.host->nR ? nR_lim : x.host->nR;
      P.nR[q] = (nr + 1) / 2;                   // 256-row blocks of the CTA pairs
      P.nsplit[q] = g2_partition(*x.host, x.K, C::BN2, P.jb[q], P.jl[q]);
      hp[q] = x.host;
      P.begin[q] = items;
      items += P.nR[q] * x.K * P.nsplit[q];
      ++q;
    }
    P.nslot = q;
    P.begin[q] = items;
    if (items == 0) continue;
    P.sync = sync && q == 1 && P.nsplit[0] == 1 ? sync : nullptr;
    if (P.sync && (err = cudaMemsetAsync(P.sync, 0, sizeof(unsigned), st)) != cudaSuccess) return err;
    const int clusters = pair_clusters_g2<PREC>();
    const int pairs = items < clusters ? items : clusters;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * pairs, 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if ((err = cudaLaunchKernelEx(&cfg, k_gemm2_pair<PREC>, P)) != cudaSuccess) return err;
    if (launches) ++*launches;
    for (int u = 0; u < q; ++u) {
      if (P.nsplit[u] <= 1) continue;
      const long long nk = (long long)P.K[u] * hp[u]->Ng;
      const int blocks = (int)std::min<long long>((nk + 255) / 256, 4LL * num_sms());
      k_g2_combine<<<blocks, 256, 0, st>>>(hp[u]->part, P.nsplit[u], P.K[u], hp[u]->Ng, P.v[u],
                                           P.v_stride[u], P.out[u], P.out_stride[u], out_io, out_is_io);
      if ((err = cudaGetLastError()) != cudaSuccess) return err;
      if (launches) ++*launches;
    }
  }
  return cudaSuccess;
}

}  // namespace

bool tc_supported() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

int tc_pair_units(int prec) {
  return prec == LRDM_BF16X3 ? pair_clusters<LRDM_BF16X3>() : pair_clusters<LRDM_TF32>();
}

bool build_tc_problem(int prec, const Channel& c, const SysState& S, int ch, TcProblem& pr) {
  if (prec == LRDM_BF16X3) return build_problem<LRDM_BF16X3>(c, S, ch, pr);
  return build_problem<LRDM_TF32>(c, S, ch, pr);
}

cudaError_t launch_gemm1_tc_group(int prec, const TcEntry* e, int n, int* status, cudaStream_t st,
                                  const TcTune& t, int nch_lim, int stall, unsigned* sync) {
  if (t.g1_nb == G1_PAIR)
    return prec == LRDM_BF16X3 ? gemm1_pair_group<LRDM_BF16X3>(e, n, status, st, nch_lim, stall, sync)
                               : gemm1_pair_group<LRDM_TF32>(e, n, status, st, nch_lim, stall, sync);
  const bool wide = t.g1_nb == 256;
  if (prec == LRDM_BF16X3)
    return wide ? gemm1_group<LRDM_BF16X3, 256>(e, n, status, st, t, nch_lim, stall)
                : gemm1_group<LRDM_BF16X3, 128>(e, n, status, st, t, nch_lim, stall);
  return wide ? gemm1_group<LRDM_TF32, 256>(e, n, status, st, t, nch_lim, stall)
              : gemm1_group<LRDM_TF32, 128>(e, n, status, st, t, nch_lim, stall);
}

cudaError_t launch_gemm2_tc_group(int prec, const TcEntry* e, int n, int out_io, int out_is_io,
                                  int* status, cudaStream_t st, const TcTune& t, int nR_lim,
                                  int* launches, unsigned* sync) {
  if (t.g2_bn == G2_PAIR)
    return prec == LRDM_BF16X3
               ? gemm2_pair_group<LRDM_BF16X3>(e, n, out_io, out_is_io, status, st, t, nR_lim, launches, sync)
               : gemm2_pair_group<LRDM_TF32>(e, n, out_io, out_is_io, status, st, t, nR_lim, launches, sync);
  const bool narrow = t.g2_bn == 128;
  if (prec == LRDM_BF16X3)
    return narrow ? gemm2_group<LRDM_BF16X3, 128>(e, n, out_io, out_is_io, status, st, t, nR_lim, launches, sync)
                  : gemm2_group<LRDM_BF16X3, 256>(e, n, out_io, out_is_io, status, st, t, nR_lim, launches, sync);
  return narrow ? gemm2_group<LRDM_TF32, 128>(e, n, out_io, out_is_io, status, st, t, nR_lim, launches, sync)
                : gemm2_group<LRDM_TF32, 256>(e, n, out_io, out_is_io, status, st, t, nR_lim, launches, sync);
}

}  // namespace lrdm
