// Fused split-precision H_eff*psi on tcgen05 (sm_103a) for large sigma blocks.
//
// A work item is a 128 x ntile tile of one sigma block and a range of units
// (term k of a class entry, up to 128 psi columns b).  Per unit:
//   MMA1   S[a', b]  = A_k[a', a] . psi^T[b, a]          A, psi^T from shared memory
//   convert          X = alpha * S split into TF32 (hi, lo), written to TMEM
//   MMA2   acc      += X[a', b] . B_k[b', b]^T           X from TMEM, B from shared memory
// so the intermediate never leaves the SM.  Operands are TF32 (hi, lo)
// pairs; a product is lo.hi + hi.lo + hi.hi with FP32 accumulation.
//
// Operand chunks (32 K-columns each: A_k and psi^T for MMA1, B_k for MMA2)
// stream through one byte ring in shared memory, in the order the MMA warp
// consumes them (MMA1(u), MMA2(u-1), MMA1(u+1), ...).  A chunk takes only
// the rows its tensor-map boxes hold, so small blocks keep more chunks in
// flight; up to NSLOT chunks are outstanding.
// Roles (320 threads): warp 0 lane 0 loads by TMA; warp 1 lane 0 issues the
// MMAs; warps 2-9 convert S (each thread one row, half of the columns: it
// loads S, releases it so that MMA1(u+1) can start, then writes X once
// MMA2(u-1) has read the previous X) and finally store the accumulator as
// an FP32 partial tile by TMA.
// TMEM (512 columns): acc [0,128) | S [128,256) | X_hi [256,384) | X_lo [384,512).
// Every mbarrier wait is bounded; on time-out the kernel records an error code
// and winds down (waits for its stores, frees TMEM) instead of hanging.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "heff_fused.h"

namespace dmrg {

namespace {

constexpr int BM = 128;
constexpr int BK = 32;                  // floats per 128-byte swizzle row
constexpr int NTHREADS = 320;
constexpr int NCONV = 256;              // converter / epilogue threads (warps 2..9)
constexpr int MAX_SMEM = 232448;
constexpr long long WAIT_LIMIT = 1LL << 22;
constexpr int NSLOT = 16;               // operand chunks in flight at most
constexpr int STAGE_OUT = 8 * 4096;     // 8 warps x one 32 x 32 FP32 box
// ring bytes; an MMA with M = 128 reads 16 KB from a chunk's A tile even when
// the box holds fewer rows, so the staging area (32 KB) after the ring
// absorbs reads past its end
constexpr int RING = (MAX_SMEM - 1024 - 512 - STAGE_OUT) / 1024 * 1024;
constexpr int SMEM_BYTES = RING + STAGE_OUT + 512 + 1024;
static_assert(SMEM_BYTES <= MAX_SMEM, "smem");
static_assert(STAGE_OUT >= 16384, "A-tile over-read guard");
constexpr uint32_t COL_ACC = 0, COL_S = 128, COL_XH = 256, COL_XL = 384;

struct FShared {
  uint64_t full[NSLOT], empty[NSLOT];
  uint32_t off[NSLOT];                  // ring offset of the chunk in each slot
  uint64_t s_full, s_free, x_full, x_free, acc_full, acc_empty;
  uint32_t tmem;
  int abort;
};
static_assert(sizeof(FShared) <= 512, "barrier area");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait_or_abort(uint32_t a, uint32_t parity, int *err, int code,
                                              volatile int *abort) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try(a, parity)) return true;
    if (*abort) return false;
    if (i > 64) __nanosleep(64);
  }
  atomicCAS(err, 0, code);
  *abort = 1;
  return false;
}
__device__ __forceinline__ void tma2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                      uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                      uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store3d(const CUtensorMap *map, int x, int y, int z,
                                            uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          (uint64_t)map),
      "r"(x), "r"(y), "r"(z), "r"(src)
      : "memory");
}
// K-major operand descriptor, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                       uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t id,
                                       uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(id), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t a, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w)
               : "memory");
}
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(NTHREADS, 1)
k_heff_fused(const FWork *__restrict__ works, int nwork, const FUnit *__restrict__ units,
             const CUtensorMap *__restrict__ maps, int *__restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *ring = smem;
  uint8_t *stage_out = smem + RING;                       // 1024-byte aligned
  FShared *sh = (FShared *)(stage_out + STAGE_OUT);
  volatile int *abort_flag = &sh->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ring_u32 = smem_u32(ring);

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(smem_u32(&sh->full[i]), 1);
      mbar_init(smem_u32(&sh->empty[i]), 1);
    }
    mbar_init(smem_u32(&sh->s_full), 1);
    mbar_init(smem_u32(&sh->s_free), NCONV);
    mbar_init(smem_u32(&sh->x_full), NCONV);
    mbar_init(smem_u32(&sh->x_free), 1);
    mbar_init(smem_u32(&sh->acc_full), 1);
    mbar_init(smem_u32(&sh->acc_empty), NCONV);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh->tmem)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh->tmem;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      // Chunk c goes to slot c % NSLOT at a ring offset chosen first-in
      // first-out; before reusing bytes (or a slot) the producer waits for
      // the chunks that held them to be released by the MMA warp.  Loads
      // follow the MMA warp's consumption order: MMA1(u), then MMA2(u-1).
      int it = 0, oldest = 0;
      uint32_t head = 0;
      uint32_t q_lo[NSLOT], q_hi[NSLOT];
      bool ok = true;
      auto retire = [&]() -> bool {   // wait until chunk `oldest` is released
        if (!wait_or_abort(smem_u32(&sh->empty[oldest % NSLOT]), (oldest / NSLOT) & 1, err, 21,
                           abort_flag))
          return false;
        ++oldest;
        return true;
      };
      auto reserve = [&](uint32_t bytes, uint32_t &pos) -> bool {
        while (oldest <= it - NSLOT)
          if (!retire()) return false;
        for (;;) {
          pos = head + bytes <= (uint32_t)RING ? head : 0u;
          bool clash = false;
          for (int c = oldest; c < it && !clash; ++c)
            clash = q_lo[c % NSLOT] < pos + bytes && pos < q_hi[c % NSLOT];
          if (!clash) break;
          if (!retire()) return false;
        }
        q_lo[it % NSLOT] = pos;
        q_hi[it % NSLOT] = pos + bytes;
        head = pos + bytes;
        return true;
      };
      auto load_r1 = [&](const FWork &w, const FUnit &un) {
        const uint32_t ta = (uint32_t)un.ra * BK * 4, tp = (uint32_t)un.pbox * BK * 4;
        for (int kc = 0; kc < un.nk1 && ok; ++kc, ++it) {
          uint32_t pos;
          if (!reserve(2 * ta + 2 * tp, pos)) {
            ok = false;
            break;
          }
          const int st = it % NSLOT;
          sh->off[st] = pos;
          const uint32_t fb = smem_u32(&sh->full[st]), d = ring_u32 + pos;
          mbar_expect_tx(fb, 2 * ta + 2 * tp);
          tma3d(d, &maps[un.mA_hi], kc * BK, un.k, w.m0, fb);
          tma3d(d + ta, &maps[un.mA_lo], kc * BK, un.k, w.m0, fb);
          tma2d(d + 2 * ta, &maps[un.mP_hi], kc * BK, un.b0, fb);
          tma2d(d + 2 * ta + tp, &maps[un.mP_lo], kc * BK, un.b0, fb);
        }
      };
      auto load_r2 = [&](const FWork &w, const FUnit &un) {
        const uint32_t tb = (uint32_t)w.ntile * BK * 4;
        const int nk2 = (un.nb + BK - 1) / BK;
        for (int kc = 0; kc < nk2 && ok; ++kc, ++it) {
          uint32_t pos;
          if (!reserve(2 * tb, pos)) {
            ok = false;
            break;
          }
          const int st = it % NSLOT;
          sh->off[st] = pos;
          const uint32_t fb = smem_u32(&sh->full[st]), d = ring_u32 + pos;
          mbar_expect_tx(fb, 2 * tb);
          tma3d(d, &maps[un.mB_hi], un.b0 + kc * BK, un.k, w.n0, fb);
          tma3d(d + tb, &maps[un.mB_lo], un.b0 + kc * BK, un.k, w.n0, fb);
        }
      };
      for (int t = blockIdx.x; t < nwork && ok; t += gridDim.x) {
        const FWork w = works[t];
        FUnit prev;
        for (int u = 0; u < w.nu && ok; ++u) {
          const FUnit un = units[w.u0 + u];
          load_r1(w, un);
          if (u > 0) load_r2(w, prev);
          prev = un;
        }
        if (w.nu > 0) load_r2(w, prev);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int ic = 0, j = 0, tt = 0;   // chunk, unit and work-item counters
      bool ok = true;
      // next chunk in consumption order: wait for its data, return its ring address
      auto next_chunk = [&](int code, uint32_t &addr) -> bool {
        const int st = ic % NSLOT;
        if (!wait_or_abort(smem_u32(&sh->full[st]), (ic / NSLOT) & 1, err, code, abort_flag))
          return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        addr = ring_u32 + *(volatile uint32_t *)&sh->off[st];
        return true;
      };
      auto release_chunk = [&]() {
        mma_commit(smem_u32(&sh->empty[ic % NSLOT]));
        ++ic;
      };
      for (int t = blockIdx.x; t < nwork && ok; t += gridDim.x, ++tt) {
        const FWork w = works[t];
        const uint32_t id2 = idesc_tf32(w.ntile);
        const uint32_t tb = (uint32_t)w.ntile * BK * 4;
        bool acc_ready = false;
        uint32_t accum2 = 0;
        // MMA2 of the unit with global index jj: acc += X . B^T over its nb columns
        auto mma2 = [&](int jj, int nb) -> bool {
          if (!acc_ready) {
            if (!wait_or_abort(smem_u32(&sh->acc_empty), (tt & 1) ^ 1, err, 23, abort_flag))
              return false;
            acc_ready = true;
          }
          if (!wait_or_abort(smem_u32(&sh->x_full), jj & 1, err, 24, abort_flag)) return false;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int nk2 = (nb + BK - 1) / BK;
          for (int kc = 0; kc < nk2; ++kc) {
            uint32_t b_hi;
            if (!next_chunk(25, b_hi)) return false;
            const uint32_t b_lo = b_hi + tb;
            const int rem = nb - kc * BK;
            const int nk8 = rem >= BK ? BK / 8 : (rem + 7) / 8;
            for (int k = 0; k < nk8; ++k) {
              const uint32_t kcol = kc * BK + k * 8;   // X columns (K) in TMEM
              const uint32_t ko = k * 32;              // bytes along the swizzled row of B
              mma_ts(tmem + COL_ACC, tmem + COL_XL + kcol, sdesc(b_hi + ko), id2, accum2);
              accum2 = 1;
              mma_ts(tmem + COL_ACC, tmem + COL_XH + kcol, sdesc(b_lo + ko), id2, 1);
              mma_ts(tmem + COL_ACC, tmem + COL_XH + kcol, sdesc(b_hi + ko), id2, 1);
            }
            release_chunk();
          }
          mma_commit(smem_u32(&sh->x_free));
          return true;
        };
        int prev_nb = 0;
        for (int u = 0; u < w.nu; ++u, ++j) {
          const FUnit un = units[w.u0 + u];
          if (!wait_or_abort(smem_u32(&sh->s_free), (j & 1) ^ 1, err, 26, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t id1 = idesc_tf32(un.n1);
          const uint32_t ta = (uint32_t)un.ra * BK * 4, tp = (uint32_t)un.pbox * BK * 4;
          uint32_t accum1 = 0;
          for (int kc = 0; kc < un.nk1; ++kc) {
            uint32_t a_hi;
            if (!next_chunk(27, a_hi)) {
              ok = false;
              break;
            }
            const uint32_t a_lo = a_hi + ta, p_hi = a_hi + 2 * ta, p_lo = p_hi + tp;
            const int rem = un.ka - kc * BK;
            const int nk8 = rem >= BK ? BK / 8 : (rem + 7) / 8;
            for (int k = 0; k < nk8; ++k) {
              const uint32_t ko = k * 32;
              mma_ss(tmem + COL_S, sdesc(a_lo + ko), sdesc(p_hi + ko), id1, accum1);
              accum1 = 1;
              mma_ss(tmem + COL_S, sdesc(a_hi + ko), sdesc(p_lo + ko), id1, 1);
              mma_ss(tmem + COL_S, sdesc(a_hi + ko), sdesc(p_hi + ko), id1, 1);
            }
            release_chunk();
          }
          if (!ok) break;
          mma_commit(smem_u32(&sh->s_full));
          if (u > 0 && !mma2(j - 1, prev_nb)) {
            ok = false;
            break;
          }
          prev_nb = un.nb;
        }
        if (!ok) break;
        if (w.nu > 0 && !mma2(j - 1, prev_nb)) break;
        mma_commit(smem_u32(&sh->acc_full));
      }
    }
  } else {
    // ---------------- converter + epilogue (warps 2..9) ----------------
    const int quarter = warp & 3;                 // TMEM lanes 32*quarter .. +31
    const int half = (warp - 2) >> 2;             // columns [64*half, 64*half + 64)
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t stg = smem_u32(stage_out + (warp - 2) * 4096);
    const uint32_t rowoff = (uint32_t)lane * 128;
    int j = 0, tt = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < nwork && ok; t += gridDim.x, ++tt) {
      const FWork w = works[t];
      for (int u = 0; u < w.nu; ++u, ++j) {
        const FUnit un = units[w.u0 + u];
        if (!wait_or_abort(smem_u32(&sh->s_full), j & 1, err, 28, abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float sv[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int col = half * 64 + c * 16;
          if (col < un.n1) tmem_ld16(tmem + COL_S + lane_off + col, sv + 16 * c);
        }
        tmem_ld_wait();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&sh->s_free));
        // X may be rewritten once MMA2 of the previous unit has completed
        if (!wait_or_abort(smem_u32(&sh->x_free), (j & 1) ^ 1, err, 29, abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int col = half * 64 + c * 16;
          if (col < un.n1) {
            float h[16], l[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float x = un.alpha * sv[16 * c + i];
              h[i] = tf32_round(x);
              l[i] = tf32_round(x - h[i]);
            }
            tmem_st16(tmem + COL_XH + lane_off + col, h);
            tmem_st16(tmem + COL_XL + lane_off + col, l);
          }
        }
        tmem_st_wait();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&sh->x_full));
      }
      if (!ok) break;
      // accumulator -> FP32 partial tile: 32 x 32 boxes staged in shared
      // memory (128-byte swizzle) and stored by TMA (the map clips the edges)
      if (!wait_or_abort(smem_u32(&sh->acc_full), tt & 1, err, 30, abort_flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row0 = w.m0 + quarter * 32;
      if (row0 < w.M) {
        for (int c0 = half * 64; c0 < half * 64 + 64 && c0 < w.ntile && w.n0 + c0 < w.N;
             c0 += 32) {
          float v[32];
          tmem_ld16(tmem + COL_ACC + lane_off + c0, v);
          if (c0 + 16 < w.ntile) {
            tmem_ld16(tmem + COL_ACC + lane_off + c0 + 16, v + 16);
            tmem_ld_wait();
          } else {
            tmem_ld_wait();
#pragma unroll
            for (int i = 16; i < 32; ++i) v[i] = 0.f;
          }
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q)
            st_shared_v4(stg + rowoff + ((uint32_t)(q ^ (lane & 7)) << 4), v[4 * q], v[4 * q + 1],
                         v[4 * q + 2], v[4 * q + 3]);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            tma_store3d(&maps[w.mOut], w.n0 + c0, row0, w.zout, stg);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&sh->acc_empty));
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

int nsm_f() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
  }();
  return n;
}

}  // namespace

cudaError_t fused_prepare() {
  return cudaFuncSetAttribute(k_heff_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t fused_gemm(const FWork *works, int nwork, const FUnit *units, const CUtensorMap *maps,
                       int *err, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  const int grid = nwork < nsm_f() ? nwork : nsm_f();
  k_heff_fused<<<grid, NTHREADS, SMEM_BYTES, s>>>(works, nwork, units, maps, err);
  return cudaGetLastError();
}

}  // namespace dmrg
