// Split-precision grouped GEMM on tcgen05 (sm_103a) for the two H_eff*psi stages.
// (persistent, warp-specialised; see k_split_gemm)
//
// Stage 1:  T[(a',k), b]  = sign * A_stack[(a',k), a] . psi[a, b]
// Stage 2:  sigma[a', b'] = sum_segments T[a', (k,b)] . B_stack[b', (k,b)]^T
// Both are C = A . B^T with K-major operands.  Every operand block is held in
// device memory as x * s = hi + lo (FP16 each, s a power of two per block, so
// the pair takes the 4 bytes of an FP32 value); a product is lo.hi + hi.lo +
// hi.hi (lo.lo, of relative size 2^-22, is below the FP32 accumulation error)
// with FP32 accumulation in tensor memory, and the epilogue takes the scales
// out exactly.  Stage 1 writes T already rescaled and split for stage 2.
// A work item is one 128 x ntile output tile; per 64-wide K chunk the
// producer loads A_hi, A_lo, B_hi, B_lo by TMA and the MMA warp issues
// 4 k-steps x 3 tcgen05.mma of kind::f16 (K = 16 each).
// Every mbarrier wait is bounded; on timeout the kernel records an error
// code, skips the remaining work, waits for its stores, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "heff_split.h"

namespace dmrg {

namespace {

constexpr int BM = 128;           // UMMA M
constexpr int BK = 64;            // halves per 128-byte swizzle row (one K chunk)
constexpr int TILE_A = BM * 128;  // 16 KB
constexpr int MAX_SMEM = 232448;  // 227 KB per CTA
constexpr int NACC = 4;           // TMEM accumulators (4 x 128 columns)
constexpr int WARP_OUT = 8192;    // epilogue staging per warp: (hi, lo) 32 x 64 halves
constexpr long long WAIT_LIMIT = 1LL << 22;      // polls (drain after an abort)
constexpr long long WAIT_CYCLES = 1LL << 31;     // ~1 s at 2 GHz: a pipeline wait gives up
constexpr uint32_t SUSPEND_NS = 100000;          // try_wait suspend-time hint
constexpr int ND = 8;             // work-item descriptor slots in shared memory
constexpr int DESC_BYTES = ND * (int)sizeof(TWork);

// Pipeline geometry for tiles at most NT columns wide (the kernel is built
// for NT = 128 and takes any narrower tile): a stage holds A_hi, A_lo
// (128 x 64 halves each) and B_hi, B_lo (NT x 64).
template <int NT>
struct Geo {
  static constexpr int NTHREADS = 96 + 128;   // producer, MMA, loader + 4 epilogue warps
  static constexpr int STAGE_OUT = 4 * WARP_OUT;
  static constexpr int TILE_B = NT * 128;
  static constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
  static constexpr int STAGES_RAW =
      (MAX_SMEM - 1024 - 512 - STAGE_OUT - DESC_BYTES) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 6 ? 6 : STAGES_RAW;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512 + STAGE_OUT + DESC_BYTES;
};
static_assert(Geo<128>::STAGES >= 3, "pipeline too shallow");
static_assert(Geo<128>::SMEM_BYTES <= MAX_SMEM, "shared memory");

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

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, int x, int y,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle,
// 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);            // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused)
  d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset
  d |= (uint64_t)1 << 46;                            // descriptor version
  d |= (uint64_t)2 << 61;                            // swizzle 128B
  return d;
}

// instruction descriptor: D f32, A/B f16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                        uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(accum)
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st_shared_v4(uint32_t a, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w)
               : "memory");
}

// shared -> global tile store through a 3-D tensor map (bulk async group)
__device__ __forceinline__ void tma_store3d(const CUtensorMap *map, int x, int y, int z,
                                            uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          (uint64_t)map),
      "r"(x), "r"(y), "r"(z), "r"(src)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the staging buffer may be rewritten once the stores issued so far read it
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

// tcgen05.ld of 16 columns without the wait (issue several, then one wait)
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void st_shared_v4u(uint32_t a, uint32_t x, uint32_t y, uint32_t z,
                                              uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w)
               : "memory");
}

// Power of two s with |m| * s <= 2^14 (m = f 2^e, f in [0.5, 1): s = 2^(14-e));
// 1 for m <= 0.  The exponent is clamped so that s stays finite.
__device__ __forceinline__ float pow2_scale(float m) {
  if (!(m > 0.f) || !(m < 3.0e38f)) return 1.f;
  int e;
  frexpf(m, &e);
  int x = 14 - e;
  x = x > 100 ? 100 : (x < -100 ? -100 : x);
  return ldexpf(1.f, x);
}

// Persistent, warp-specialised split GEMM.  The CTAs claim the items of the
// work list in order from a device counter (the host orders the list):
//   warp 0, lane 0   TMA producer over all K chunks of all its tiles
//   warp 1, lane 0   MMA issuer, rotating over four TMEM accumulators
//   warps 2..5       epilogue: drain an accumulator while the next tile runs
//   last warp        claims items and copies their descriptors with plain
//                    loads into a ring of ND shared-memory slots, as far
//                    ahead as the ring allows, so no role waits on a global
//                    load at a tile boundary (and the copies do not queue
//                    behind tile loads in the TMA unit)
// A descriptor slot is refilled after its six readers (producer, MMA issuer,
// four epilogue warps) have released it.
constexpr int ACC_COLS = 128;

struct Shared {
  uint64_t full[8], empty[8], acc_full[NACC], acc_empty[NACC], dfull[ND], dempty[ND];
  uint32_t tmem;
  int abort;
};
static_assert(sizeof(Shared) <= 512, "barrier area");

// try_wait with a suspend-time hint: a waiting thread sleeps in hardware and
// wakes when the phase completes (no polling delay at hand-offs)
__device__ __forceinline__ bool mbar_try_suspend(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity), "r"(SUSPEND_NS)
      : "memory");
  return ok != 0;
}

// Bounded pipeline wait: gives up after WAIT_CYCLES (or when another role
// has given up), records `code` and raises the CTA's abort flag.
__device__ __forceinline__ bool wait_or_abort(uint32_t a, uint32_t parity, int *err, int code,
                                              volatile int *abort) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_suspend(a, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > WAIT_CYCLES) break;
  }
  atomicCAS(err, 0, code);
  *abort = 1;
  return false;
}

template <int NT>
__global__ void __launch_bounds__(Geo<NT>::NTHREADS, 1)
k_split_gemm(const TWork *__restrict__ works, int nwork, const TSeg *__restrict__ segs,
             const CUtensorMap *__restrict__ maps, const PsiStat *__restrict__ pstat,
             int *__restrict__ err, int *__restrict__ next_item) {
  using G = Geo<NT>;
  constexpr int STAGES = G::STAGES;
  constexpr int STAGE_BYTES = G::STAGE_BYTES;
  constexpr int TILE_B = G::TILE_B;
  constexpr int STAGE_OUT = G::STAGE_OUT;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *stage_out = smem + STAGES * STAGE_BYTES;      // 1024-byte aligned
  TWork *desc = (TWork *)(stage_out + STAGE_OUT);         // ND slots, 16-byte aligned
  Shared *sh = (Shared *)(stage_out + STAGE_OUT + DESC_BYTES);
  volatile int *abort_flag = &sh->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(smem_u32(&sh->full[i]), 1);
      mbar_init(smem_u32(&sh->empty[i]), 1);
    }
    for (int i = 0; i < NACC; ++i) {
      mbar_init(smem_u32(&sh->acc_full[i]), 1);
      mbar_init(smem_u32(&sh->acc_empty[i]), 128);
    }
    for (int i = 0; i < ND; ++i) {
      mbar_init(smem_u32(&sh->dfull[i]), 1);
      mbar_init(smem_u32(&sh->dempty[i]), 6);
    }
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh->tmem)),
                 "r"(NACC * ACC_COLS)
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
      int it = 0;
      for (int i = 0; !*abort_flag; ++i) {
        const int sl = i % ND;
        if (!wait_or_abort(smem_u32(&sh->dfull[sl]), (i / ND) & 1, err, 6, abort_flag)) break;
        // read in place; the slot is released once this item's loads are issued
        const TWork &w = desc[sl];
        if (w.mode < 0) break;   // no more items
        const uint32_t stage_tx = 2 * TILE_A + 2 * (uint32_t)w.ntile * 128;
        if (w.R > 1) {
          // packed tile: per chunk, group r's rows of A and B from its own
          // segment (a chunk past the segment's end loads zeros)
          const uint32_t ga = (BM / w.R) * 128, gb = (uint32_t)(w.ntile / w.R) * 128;
          uint32_t tx = 0;
          for (int r = 0; r < w.R; ++r)
            if (w.pseg[r] >= 0) tx += 2 * ga + 2 * gb;
          for (int kc = 0; kc < w.nchunk; ++kc, ++it) {
            const int st = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!wait_or_abort(smem_u32(&sh->empty[st]), ph ^ 1, err, 1, abort_flag)) break;
            uint8_t *base = smem + st * STAGE_BYTES;
            const uint32_t fb = smem_u32(&sh->full[st]);
            mbar_expect_tx(fb, tx);
            for (int r = 0; r < w.R; ++r) {
              if (w.pseg[r] < 0) continue;
              const TSeg sg = segs[w.pseg[r]];
              const int kx = kc * BK < sg.K ? sg.k0 + kc * BK : sg.xoob;
              tma_load(smem_u32(base + r * ga), &maps[sg.mA_hi], kx, 0, fb);
              tma_load(smem_u32(base + TILE_A + r * ga), &maps[sg.mA_lo], kx, 0, fb);
              tma_load(smem_u32(base + 2 * TILE_A + r * gb), &maps[sg.mB_hi], kx, 0, fb);
              tma_load(smem_u32(base + 2 * TILE_A + TILE_B + r * gb), &maps[sg.mB_lo], kx, 0, fb);
            }
          }
          mbar_arrive(smem_u32(&sh->dempty[sl]));
          continue;
        }
        const TSeg sg = w.s;
        const int m0 = w.m0, n0 = w.n0;
        mbar_arrive(smem_u32(&sh->dempty[sl]));
        const int nk = (sg.K + BK - 1) / BK;
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int st = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!wait_or_abort(smem_u32(&sh->empty[st]), ph ^ 1, err, 1, abort_flag)) break;
          uint8_t *base = smem + st * STAGE_BYTES;
          const uint32_t fb = smem_u32(&sh->full[st]);
          mbar_expect_tx(fb, stage_tx);
          const int kx = sg.k0 + kc * BK;
          tma_load(smem_u32(base), &maps[sg.mA_hi], kx, m0, fb);
          tma_load(smem_u32(base + TILE_A), &maps[sg.mA_lo], kx, m0, fb);
          tma_load(smem_u32(base + 2 * TILE_A), &maps[sg.mB_hi], kx, n0, fb);
          tma_load(smem_u32(base + 2 * TILE_A + TILE_B), &maps[sg.mB_lo], kx, n0, fb);
        }
      }
      if (*abort_flag) {
        // a wait gave up somewhere: let this CTA's copies in flight land
        // before it exits (bounded; a completed phase returns at once)
        for (int c = it > STAGES ? it - STAGES : 0; c < it; ++c)
          for (long long k = 0; k < WAIT_LIMIT && !mbar_try(smem_u32(&sh->full[c % STAGES]),
                                                           (c / STAGES) & 1); ++k)
            __nanosleep(64);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int it = 0;
      for (int j = 0; !*abort_flag; ++j) {
        const int sl = j % ND;
        if (!wait_or_abort(smem_u32(&sh->dfull[sl]), (j / ND) & 1, err, 6, abort_flag)) break;
        if (desc[sl].mode < 0) break;
        const int ntile = desc[sl].ntile;
        // packed tiles run all their chunks without trimming (the groups'
        // segments end at different K)
        const int K = desc[sl].R > 1 ? desc[sl].nchunk * BK : desc[sl].s.K;
        mbar_arrive(smem_u32(&sh->dempty[sl]));
        const uint32_t id = idesc_f16(ntile);
        const int acc = j % NACC;
        const uint32_t aph = (j / NACC) & 1;
        if (!wait_or_abort(smem_u32(&sh->acc_empty[acc]), aph ^ 1, err, 2, abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + acc * ACC_COLS;
        uint32_t accum = 0;
        {
          const int nk = (K + BK - 1) / BK;
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int st = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!wait_or_abort(smem_u32(&sh->full[st]), ph, err, 3, abort_flag)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t a_lo = a_hi + TILE_A;
            const uint32_t b_hi = a_hi + 2 * TILE_A;
            const uint32_t b_lo = b_hi + TILE_B;
            // k-steps of 16 that hold data (the rest of a ragged chunk is zero fill)
            const int rem = K - kc * BK;
            const int nk16 = rem >= BK ? BK / 16 : (rem + 15) / 16;
            // a k-step of 16 halves (32 bytes along the swizzled row) adds 2
            // to the encoded start address
            const uint64_t dah = sdesc(a_hi), dal = sdesc(a_lo), dbh = sdesc(b_hi),
                           dbl = sdesc(b_lo);
            auto kstep = [&](int k) {
              const uint64_t ko = 2 * k;
              // small terms first: lo.hi, hi.lo, then hi.hi (lo.lo is below
              // the FP32 accumulation error and is left out)
              mma_f16(d, dal + ko, dbh + ko, id, accum);
              accum = 1;
              mma_f16(d, dah + ko, dbl + ko, id, 1);
              mma_f16(d, dah + ko, dbh + ko, id, 1);
            };
            if (nk16 == BK / 16) {
              // a full chunk: straight-line issue
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) kstep(k);
            } else {
              for (int k = 0; k < nk16; ++k) kstep(k);
            }
            mma_commit(smem_u32(&sh->empty[st]));
          }
        }
        // every work item has K >= 1, so the accumulator always holds data
        mma_commit(smem_u32(&sh->acc_full[acc]));
      }
    }
  } else if (warp == 6) {
    // ---------------- descriptor loader ----------------
    // Items are claimed from the launch's counter (list order: the CTAs
    // share the work dynamically); 12 lanes copy a 192-byte item (16 bytes
    // each), lane 0 then arrives on the slot's barrier (release: the warp's
    // stores are ordered before it by the fence and __syncwarp).  When the
    // list is exhausted, the next slot gets an end mark (mode < 0).
    int i = 0;
    bool ok = true;
    for (;; ++i) {
      const int sl = i % ND;
      if (!wait_or_abort(smem_u32(&sh->dempty[sl]), ((i / ND) & 1) ^ 1, err, 5, abort_flag)) {
        ok = false;
        break;
      }
      int idx = 0;
      if (lane == 0) idx = atomicAdd(next_item, 1);
      idx = __shfl_sync(0xffffffffu, idx, 0);
      if (idx >= nwork) break;
      const uint4 *src = reinterpret_cast<const uint4 *>(works + idx);
      if (lane < (int)(sizeof(TWork) / 16)) reinterpret_cast<uint4 *>(desc + sl)[lane] = src[lane];
      __threadfence_block();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh->dfull[sl]));
    }
    if (ok) {
      if (lane == 0) {
        desc[i % ND].mode = -1;
        __threadfence_block();
        mbar_arrive(smem_u32(&sh->dfull[i % ND]));
      }
      __syncwarp();
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    // Each lane holds one accumulator row.  The warp stages its 32-row
    // sub-tile in shared memory in the 128-byte-swizzled box layout (16-byte
    // chunk q of row r at position q ^ (r & 7)) and one lane stores it by
    // TMA; the tensor maps clip rows and columns outside the destination.
    //   stage 1: T = alpha * C / (sA sP), times T's own power of two, split
    //            into FP16 (hi, lo), 64 columns per box;
    //   stage 2: C / (sT sB) as FP32, 32 columns per box.
    const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
    const uint32_t stg = smem_u32(stage_out + (warp - 2) * WARP_OUT), stg2 = stg + WARP_OUT / 2;
    const uint32_t rowoff = (uint32_t)lane * 128;
    for (int j = 0;; ++j) {
      const int sl = j % ND;
      if (!wait_or_abort(smem_u32(&sh->dfull[sl]), (j / ND) & 1, err, 6, abort_flag)) break;
      // this warp's share of the item, read from the slot, then the slot is released
      const TWork &d = desc[sl];
      if (d.mode < 0) break;
      const int R = d.R, mode = d.mode, ntile = d.ntile, M = d.M, N = d.N, n0 = d.n0;
      const int mOut_lo = d.mOut_lo;
      int row0 = d.m0 + quarter * 32, cbeg = 0, cend = ntile, xoff = n0, mo = d.mOut_hi,
          zo = d.zout;
      bool live = row0 < M;
      float fa = d.fa, rn = d.rn, alpha = d.alpha;
      int pb = d.pblk;
      if (R > 1) {
        // destination of this warp's rows: the diagonal block of its group
        const int per = 4 / R, r = quarter / per, gw = ntile / R;
        row0 = (quarter % per) * 32;
        cbeg = r * gw;
        cend = cbeg + gw;
        xoff = -cbeg;
        mo = d.pout[r];
        zo = d.pz[r];
        live = d.pseg[r] >= 0;
        fa = d.pfa[r];
        rn = d.prn[r];
        pb = live ? d.ppb[r] : 0;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh->dempty[sl]));
      // scale statistics of the psi block: loaded before the accumulator wait
      const PsiStat ps = pstat[pb];
      const int acc = j % NACC;
      const uint32_t aph = (j / NACC) & 1;
      if (!wait_or_abort(smem_u32(&sh->acc_full[acc]), aph, err, 4, abort_flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tbase = tmem + acc * ACC_COLS + ((uint32_t)(quarter * 32) << 16);
      float fac;
      if (R > 1) {
        fac = live ? fa / pow2_scale(rn * ps.cn) : 0.f;
      } else if (mode == TW_SPLIT) {
        fac = alpha * fa * pow2_scale(rn * ps.cn) / pow2_scale(ps.mx);
      } else {
        fac = fa / pow2_scale(rn * ps.cn);
      }
      // the accumulator is handed back to the MMA issuer as soon as its last
      // columns are in registers
      bool released = false;
      auto release = [&]() {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&sh->acc_empty[acc]));
        released = true;
      };
      if (live && mode == TW_SPLIT) {
        for (int c0 = 0; c0 < ntile && n0 + c0 < N; c0 += 64) {
          uint32_t v[64];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (c0 + 16 * q < ntile) {
              tmem_ld16_nw(tbase + c0 + 16 * q, v + 16 * q);
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i) v[16 * q + i] = 0u;
            }
          }
          tmem_ld_wait();
          if (!(c0 + 64 < ntile && n0 + c0 + 64 < N)) release();
          // split pairs of columns with packed conversions, then store once
          // the previous box has left the staging buffer
          uint32_t h[32], l[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float2 t = make_float2(fac * __uint_as_float(v[2 * i]),
                                         fac * __uint_as_float(v[2 * i + 1]));
            const __half2 h2 = __float22half2_rn(t);
            const float2 hb = __half22float2(h2);
            const __half2 l2 = __float22half2_rn(make_float2(t.x - hb.x, t.y - hb.y));
            h[i] = *reinterpret_cast<const uint32_t *>(&h2);
            l[i] = *reinterpret_cast<const uint32_t *>(&l2);
          }
          if (lane == 0) bulk_wait_read();
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint32_t o = rowoff + ((uint32_t)(q ^ (lane & 7)) << 4);
            st_shared_v4u(stg + o, h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
            st_shared_v4u(stg2 + o, l[4 * q], l[4 * q + 1], l[4 * q + 2], l[4 * q + 3]);
          }
          fence_async_shared();
          __syncwarp();
          if (lane == 0) {
            tma_store3d(&maps[mo], n0 + c0, row0, 0, stg);
            tma_store3d(&maps[mOut_lo], n0 + c0, row0, 0, stg2);
            bulk_commit();
          }
        }
      } else if (live) {
        for (int c0 = cbeg; c0 < cend && (R > 1 || n0 + c0 < N); c0 += 32) {
          float v[32];
          tmem_ld16(tbase + c0, v);
          if (c0 + 16 < ntile) {
            tmem_ld16(tbase + c0 + 16, v + 16);
          } else {
#pragma unroll
            for (int i = 16; i < 32; ++i) v[i] = 0.f;
          }
          if (!(c0 + 32 < cend && (R > 1 || n0 + c0 + 32 < N))) release();
          if (lane == 0) bulk_wait_read();
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q)
            st_shared_v4(stg + rowoff + ((uint32_t)(q ^ (lane & 7)) << 4), fac * v[4 * q],
                         fac * v[4 * q + 1], fac * v[4 * q + 2], fac * v[4 * q + 3]);
          fence_async_shared();
          __syncwarp();
          if (lane == 0) {
            tma_store3d(&maps[mo], xoff + c0, row0, zo, stg);
            bulk_commit();
          }
        }
      }
      if (!released) release();
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(NACC * ACC_COLS)
                 : "memory");
  }
}

// Self-test of the bounded waits: one thread waits on a shared-memory barrier
// that nothing completes; wait_or_abort must give up after WAIT_CYCLES and
// record its code.  No memory operation is left in flight.
__global__ void k_wait_selftest(int *err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  mbar_init(smem_u32(&bar), 1);
  abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (wait_or_abort(smem_u32(&bar), 0, err, 7, &abort_flag)) atomicExch(err, -1);
}

// ---------------------------------------------------------------------------
// scaled FP16 (hi, lo) copies and their statistics
// ---------------------------------------------------------------------------

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// one CTA per class entry: max |A|, max row 2-norm of A, max |B| (FP64 stacks)
__global__ void __launch_bounds__(256) k_entry_stats(const StatDesc *__restrict__ ds,
                                                     EntryStat *__restrict__ out) {
  const StatDesc d = ds[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float mA = 0.f, rA = 0.f, mB = 0.f;
  for (long long r = warp; r < d.rowsA; r += 8) {
    const double *row = d.a + r * d.colsA;
    double ss = 0.0;
    float m = 0.f;
    for (int c = lane; c < d.colsA; c += 32) {
      const double x = row[c];
      ss += x * x;
      m = fmaxf(m, (float)fabs(x));
    }
    // row sums of squares in FP32 (only a bound is needed)
    const float s = warp_sum((float)ss);
    mA = fmaxf(mA, warp_max(m));
    rA = fmaxf(rA, sqrtf(s));
  }
  for (long long r = warp; r < d.rowsB; r += 8) {
    const double *row = d.b + r * d.colsB;
    float m = 0.f;
    for (int c = lane; c < d.colsB; c += 32) m = fmaxf(m, (float)fabs(row[c]));
    mB = fmaxf(mB, warp_max(m));
  }
  __shared__ float red[3][8];
  if (lane == 0) {
    red[0][warp] = mA;
    red[1][warp] = rA;
    red[2][warp] = mB;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f, c = 0.f;
    for (int i = 0; i < 8; ++i) {
      a = fmaxf(a, red[0][i]);
      b = fmaxf(b, red[1][i]);
      c = fmaxf(c, red[2][i]);
    }
    // the bound on T uses the row norm rounded up a little (FP32 sums)
    out[blockIdx.x] = {a, b * 1.0001f, c, 0.f};
  }
}

// one CTA per psi block (rows x cols, row-major at psi + off): max |psi| and
// the largest column 2-norm
__global__ void __launch_bounds__(256) k_psi_stats(const PsiDesc *__restrict__ ds,
                                                   const double *__restrict__ psi,
                                                   PsiStat *__restrict__ out) {
  const PsiDesc d = ds[blockIdx.x];
  const double *p = psi + d.off;
  float m = 0.f, cn = 0.f;
  for (int c = threadIdx.x; c < d.cols; c += blockDim.x) {
    double ss = 0.0;
    float mc = 0.f;
    int r = 0;
    // eight loads in flight, then added in row order
    for (; r + 8 <= d.rows; r += 8) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = p[(long long)(r + u) * d.cols + c];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        ss += x[u] * x[u];
        mc = fmaxf(mc, (float)fabs(x[u]));
      }
    }
    for (; r < d.rows; ++r) {
      const double x = p[(long long)r * d.cols + c];
      ss += x * x;
      mc = fmaxf(mc, (float)fabs(x));
    }
    m = fmaxf(m, mc);
    cn = fmaxf(cn, (float)sqrt(ss));
  }
  __shared__ float red[2][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  m = warp_max(m);
  cn = warp_max(cn);
  if (lane == 0) {
    red[0][warp] = m;
    red[1][warp] = cn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a = fmaxf(a, red[0][i]);
      b = fmaxf(b, red[1][i]);
    }
    out[blockIdx.x] = {a, b * 1.0001f};
  }
}

// FP64 -> scaled FP16 (hi, lo), 32 x 32 tiles through shared memory
__global__ void k_f16_split(const F16Split *__restrict__ ds, const PsiStat *__restrict__ pstat,
                            const double *__restrict__ bind) {
  __shared__ double tile[32][33];
  const F16Split d = ds[blockIdx.z];
  const double *src = d.src ? d.src : bind + d.src_off;
  const double s = d.scale > 0.f ? (double)d.scale : (double)pow2_scale(pstat[d.pblk].mx);
  // the destination's padding (columns up to dst_ld) is written with zeros:
  // the tensor maps of the tcgen05 stages read K up to the padded width
  const int prow = d.trans ? d.dst_ld : d.rows, pcol = d.trans ? d.cols : d.dst_ld;
  const int tr = (prow + 31) / 32, tc = (pcol + 31) / 32;
  for (int t = blockIdx.x; t < tr * tc; t += gridDim.x) {
    const int r0 = (t / tc) * 32, c0 = (t % tc) * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      const int r = r0 + j, c = c0 + threadIdx.x;
      tile[j][threadIdx.x] = (r < d.rows && c < d.cols) ? src[(long long)r * d.src_ld + c] : 0.0;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
      int r, c;
      double x;
      if (d.trans) {
        c = c0 + j;
        r = r0 + threadIdx.x;
        x = tile[threadIdx.x][j];
      } else {
        r = r0 + j;
        c = c0 + threadIdx.x;
        x = tile[j][threadIdx.x];
      }
      if (c < pcol && r < prow) {
        const double y = x * s;
        const __half h = __double2half(y);
        const __half l = __double2half(y - (double)__half2float(h));
        const long long o = d.trans ? (long long)c * d.dst_ld + r : (long long)r * d.dst_ld + c;
        d.hi[o] = h;
        d.lo[o] = l;
      }
    }
    __syncthreads();
  }
}

// s + c += x with the rounding error of the add kept in c (Knuth's
// branch-free two-sum): the sum of a few hundred FP32 partials stays accurate
// to about 2^-24 of the total while using only FP32 arithmetic (FP64 units
// are scarce on this part).
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x) {
  const float t = s + x;
  const float z = t - s;
  c += (s - (t - z)) + (x - z);
  s = t;
}

// One thread per four consecutive elements of a sigma row (partial rows are
// 16-byte aligned: ld is a multiple of 4 floats); the partials are added in
// slot order, eight float4 loads in flight per step, so the result does not
// depend on the launch.
__global__ void k_sum_partials(const PartialSum *__restrict__ ps, double *__restrict__ sigma) {
  const PartialSum p = ps[blockIdx.y];
  const int c4n = (p.cols + 3) / 4, rows = p.cols > 0 ? p.n / p.cols : 0;
  const int n4 = rows * c4n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += gridDim.x * blockDim.x) {
    const int r = i / c4n, c = (i - r * c4n) * 4;
    const float4 *src = (const float4 *)(p.ws + (long long)r * p.ld + c);
    const long long st4 = p.stride / 4;
    float s0 = 0, s1 = 0, s2 = 0, s3 = 0, e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    int k = 0;
    for (; k + 8 <= p.nparts; k += 8) {
      float4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __ldg(src + (long long)(k + j) * st4);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        two_sum_add(s0, e0, v[j].x);
        two_sum_add(s1, e1, v[j].y);
        two_sum_add(s2, e2, v[j].z);
        two_sum_add(s3, e3, v[j].w);
      }
    }
    for (; k < p.nparts; ++k) {
      const float4 v = __ldg(src + (long long)k * st4);
      two_sum_add(s0, e0, v.x);
      two_sum_add(s1, e1, v.y);
      two_sum_add(s2, e2, v.z);
      two_sum_add(s3, e3, v.w);
    }
    double *out = sigma + p.off + (long long)r * p.cols + c;
    out[0] = (double)s0 + (double)e0;
    if (c + 1 < p.cols) out[1] = (double)s1 + (double)e1;
    if (c + 2 < p.cols) out[2] = (double)s2 + (double)e2;
    if (c + 3 < p.cols) out[3] = (double)s3 + (double)e3;
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                             const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                             const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static const EncodeFn fn = [] {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeFn) nullptr;
    return (EncodeFn)p;
  }();
  return fn;
}

int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
  }();
  return n;
}

template <int NT>
cudaError_t prepare_nt() {
  return cudaFuncSetAttribute(k_split_gemm<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Geo<NT>::SMEM_BYTES);
}

// (the shared-memory attributes are set by split_prepare, outside any capture)
template <int NT>
cudaError_t launch_nt(const TWork *work, int nwork, int *next_item, const TSeg *seg,
                      const CUtensorMap *maps,
                      const PsiStat *pstat, int *err, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  const int nsm = sm_count();
  const int grid = nwork < nsm ? nwork : nsm;
  k_split_gemm<NT><<<grid, Geo<NT>::NTHREADS, Geo<NT>::SMEM_BYTES, s>>>(work, nwork, seg, maps,
                                                                        pstat, err, next_item);
  return cudaGetLastError();
}

}  // namespace

float pow2_scale_host(float m) {
  if (!(m > 0.f) || !(m < 3.0e38f)) return 1.f;
  int e;
  std::frexp(m, &e);
  int x = 14 - e;
  x = x > 100 ? 100 : (x < -100 ? -100 : x);
  return std::ldexp(1.f, x);
}

int encode_map_h(CUtensorMap *out, const __half *base, long long rows, long long cols,
                 long long ld, int box_rows) {
  const EncodeFn fn = encoder();
  if (!fn) return -1;
  if (((uintptr_t)base & 15) || (ld & 7) || rows <= 0 || cols <= 0) return -2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void *)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int encode_map3_h(CUtensorMap *out, const __half *base, long long d0, long long d1,
                  long long d2, long long s1, long long s2, int box1, int box2) {
  const EncodeFn fn = encoder();
  if (!fn) return -1;
  if (((uintptr_t)base & 15) || (s1 & 7) || (s2 & 7) || d0 <= 0 || d1 <= 0 || d2 <= 0) return -2;
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)s1 * 2, (cuuint64_t)s2 * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box1, (cuuint32_t)box2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void *)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int encode_map3(CUtensorMap *out, const float *base, long long d0, long long d1, long long d2,
                long long s1, long long s2, int box0, int box1, int box2) {
  const EncodeFn fn = encoder();
  if (!fn) return -1;
  if (((uintptr_t)base & 15) || (s1 & 3) || (s2 & 3) || d0 <= 0 || d1 <= 0 || d2 <= 0 ||
      box0 * 4 > 128)
    return -2;
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)s1 * 4, (cuuint64_t)s2 * 4};
  cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, (cuuint32_t)box2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

cudaError_t sum_partials(const PartialSum *p, int n, double *sigma, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(32, n);   // blocks beyond a block's elements exit at once
  k_sum_partials<<<grid, 256, 0, s>>>(p, sigma);
  return cudaGetLastError();
}

cudaError_t entry_stats(const StatDesc *d, int n, EntryStat *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_entry_stats<<<n, 256, 0, s>>>(d, out);
  return cudaGetLastError();
}

cudaError_t psi_stats(const PsiDesc *d, int n, const double *psi, PsiStat *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_psi_stats<<<n, 256, 0, s>>>(d, psi, out);
  return cudaGetLastError();
}

cudaError_t f16_split(const F16Split *d, int n, const PsiStat *pstat, const double *bind,
                      cudaStream_t s, int grid_tiles) {
  const unsigned gx = grid_tiles < 1 ? 1u : (grid_tiles > 128 ? 128u : (unsigned)grid_tiles);
  // grid.z is limited to 65535: launch in chunks of descriptors
  for (int i0 = 0; i0 < n; i0 += 65535) {
    dim3 grid(gx, 1, n - i0 < 65535 ? n - i0 : 65535), block(32, 8);
    k_f16_split<<<grid, block, 0, s>>>(d + i0, pstat, bind);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t split_prepare() { return prepare_nt<128>(); }

cudaError_t wait_selftest(int *err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err);
  return cudaGetLastError();
}

cudaError_t split_gemm(const TWork *work, int nwork, int *next, const TSeg *seg,
                       const CUtensorMap *maps, const PsiStat *pstat, int *err, cudaStream_t s) {
  // the CTAs claim items from *next, which starts at zero
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  return launch_nt<128>(work, nwork, next, seg, maps, pstat, err, s);
}

}  // namespace dmrg
