// 3 x TF32 grouped GEMM on tcgen05 (sm_103a) for the two H_eff*psi stages.
// (persistent, warp-specialised; see k_tf32_gemm)
//
// Stage 1:  T[(a',k), b]  = sign * A_stack[(a',k), a] . psi[a, b]
// Stage 2:  sigma[a', b'] = sum_segments T[a', (k,b)] . B_stack[b', (k,b)]^T
// Both are C = A . B^T with K-major operands.  The operator stacks and T are
// FP32 in device memory; psi^T comes split as TF32 (hi, lo).  Each FP32
// operand chunk is split on chip: the tensor core reads the FP32 tile as the
// high part (top 19 bits) and converter warps write the low part next to it.
// A product is lo.hi + hi.lo + hi.hi (lo.lo, of relative size 2^-22, is
// below the FP32 accumulation error) with FP32 accumulation in tensor
// memory.  A work item is one 128 x ntile output tile; per 32-wide K chunk
// the producer loads A and B (and psi^T's low part) by TMA, the converters
// add the low parts and the MMA warp issues 4 k-steps x 3 tcgen05.mma.
// Every mbarrier wait is bounded; on timeout the kernel records an error
// code, skips the remaining work, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "heff_tf32.h"

namespace dmrg {

namespace {

constexpr int BM = 128;           // UMMA M
constexpr int BK = 32;            // floats per 128-byte swizzle row
constexpr int TILE_A = BM * BK * 4;          // 16 KB
constexpr int MAX_SMEM = 232448;             // 227 KB per CTA
constexpr int NACC = 4;                      // TMEM accumulators (4 x 128 columns)
constexpr int STAGE_OUT = 4 * 4096;          // epilogue staging: 4 warps x one 32 x 32 box

// Pipeline geometry for a launch whose tiles are at most NT columns wide:
// a TMA stage holds the FP32 chunks A (128 x 32) and B (NT x 32); a low-part
// slot holds A_lo and B_lo.  The FP32 chunks stay until the MMAs that read
// them as high parts complete; the low parts need only LO slots.
constexpr int LO = 2;
template <int NT>
struct Geo {
  static constexpr int TILE_B = NT * BK * 4;
  static constexpr int STAGE_BYTES = TILE_A + TILE_B;
  static constexpr int STAGES_RAW =
      (MAX_SMEM - 1024 - 512 - STAGE_OUT - LO * STAGE_BYTES) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr int SMEM_BYTES = (STAGES + LO) * STAGE_BYTES + 1024 + 512 + STAGE_OUT;
};
static_assert(Geo<128>::STAGES >= 4, "pipeline too shallow");
constexpr long long WAIT_LIMIT = 1LL << 22;

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

// instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
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

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

// four FP32 values at src -> their low TF32 parts at dst
__device__ __forceinline__ void lo_split4(uint32_t src, uint32_t dst) {
  float x[4];
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
               : "r"(src)
               : "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float hi = __uint_as_float(__float_as_uint(x[i]) & 0xffffe000u);
    x[i] = tf32_round(x[i] - hi);
  }
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "f"(x[0]), "f"(x[1]),
               "f"(x[2]), "f"(x[3])
               : "memory");
}

// Persistent, warp-specialised 3xTF32 GEMM.  Each CTA walks the work list
// with stride gridDim.x (the list is sorted by cost, largest first):
//   warp 0, lane 0   TMA producer over all K chunks of all its tiles
//   warp 1, lane 0   MMA issuer, rotating over four TMEM accumulators
//   warps 2..5       epilogue: drain an accumulator while the next tile runs
//   warps 6..13      converters: split each FP32 operand chunk on chip
constexpr int NTHREADS = 448;
constexpr int NCONV = 256;
constexpr int ACC_COLS = 128;

struct Shared {
  uint64_t full[8], empty[8], lo_full[LO], lo_empty[LO], acc_full[NACC], acc_empty[NACC];
  uint32_t tmem;
  int abort;
};
static_assert(sizeof(Shared) <= 512, "barrier area");

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

template <int NT>
__global__ void __launch_bounds__(NTHREADS, 1)
k_tf32_gemm(const TWork *__restrict__ works, int nwork, const TSeg *__restrict__ segs,
            const CUtensorMap *__restrict__ maps, int *__restrict__ err) {
  using G = Geo<NT>;
  constexpr int STAGES = G::STAGES;
  constexpr int STAGE_BYTES = G::STAGE_BYTES;
  constexpr int TILE_B = G::TILE_B;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *lo_ring = smem + STAGES * STAGE_BYTES;        // low parts
  uint8_t *stage_out = lo_ring + LO * STAGE_BYTES;       // 1024-byte aligned
  Shared *sh = (Shared *)(stage_out + STAGE_OUT);
  volatile int *abort_flag = &sh->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(smem_u32(&sh->full[i]), 1);
      mbar_init(smem_u32(&sh->empty[i]), 1);
    }
    for (int i = 0; i < LO; ++i) {
      mbar_init(smem_u32(&sh->lo_full[i]), NCONV);
      mbar_init(smem_u32(&sh->lo_empty[i]), 1);
    }
    for (int i = 0; i < NACC; ++i) {
      mbar_init(smem_u32(&sh->acc_full[i]), 1);
      mbar_init(smem_u32(&sh->acc_empty[i]), 128);
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
      for (int t = blockIdx.x; t < nwork && !*abort_flag; t += gridDim.x) {
        const TWork w = works[t];
        const uint32_t stage_tx = TILE_A + (uint32_t)w.ntile * BK * 4;
        if (w.R > 1) {
          // packed tile: per chunk, group r's rows of A and B from its own
          // segment (a chunk past the segment's end loads zeros)
          const uint32_t ga = (BM / w.R) * BK * 4, gb = (uint32_t)(w.ntile / w.R) * BK * 4;
          uint32_t tx = 0;
          for (int r = 0; r < w.R; ++r)
            if (w.pseg[r] >= 0) tx += ga + gb;
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
              tma_load(smem_u32(base + TILE_A + r * gb), &maps[sg.mB_hi], kx, 0, fb);
            }
          }
          continue;
        }
        for (int s = 0; s < w.nseg && !*abort_flag; ++s) {
          const TSeg sg = segs[w.seg0 + s];
          const int nk = (sg.K + BK - 1) / BK;
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int st = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!wait_or_abort(smem_u32(&sh->empty[st]), ph ^ 1, err, 1, abort_flag)) break;
            uint8_t *base = smem + st * STAGE_BYTES;
            const uint32_t fb = smem_u32(&sh->full[st]);
            mbar_expect_tx(fb, stage_tx);
            const int kx = sg.k0 + kc * BK;
            tma_load(smem_u32(base), &maps[sg.mA_hi], kx, w.m0, fb);
            tma_load(smem_u32(base + TILE_A), &maps[sg.mB_hi], kx, w.n0, fb);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int it = 0, j = 0;
      for (int t = blockIdx.x; t < nwork && !*abort_flag; t += gridDim.x, ++j) {
        const TWork w = works[t];
        const uint32_t id = idesc_tf32(w.ntile);
        const int acc = j % NACC;
        const uint32_t aph = (j / NACC) & 1;
        if (!wait_or_abort(smem_u32(&sh->acc_empty[acc]), aph ^ 1, err, 2, abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + acc * ACC_COLS;
        uint32_t accum = 0;
        const int nseg = w.R > 1 ? 1 : w.nseg;
        for (int s = 0; s < nseg; ++s) {
          // packed tiles run all their chunks without trimming (the groups'
          // segments end at different K)
          const int K = w.R > 1 ? w.nchunk * BK : segs[w.seg0 + s].K;
          const int nk = (K + BK - 1) / BK;
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int st = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            // the low parts of chunk `it` are ready (its FP32 chunk too)
            const int ls = it % LO;
            if (!wait_or_abort(smem_u32(&sh->lo_full[ls]), (it / LO) & 1, err, 3, abort_flag))
              break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t b_hi = a_hi + TILE_A;
            const uint32_t a_lo = smem_u32(lo_ring + ls * STAGE_BYTES);
            const uint32_t b_lo = a_lo + TILE_A;
            // k-steps of 8 that hold data (the rest of a ragged chunk is zero fill)
            const int rem = K - kc * BK;
            const int nk8 = rem >= BK ? BK / 8 : (rem + 7) / 8;
            // descriptors of the chunk's tiles; a k-step of 8 tf32 (32 bytes
            // along the swizzled row) adds 2 to the encoded start address
            const uint64_t dah = sdesc(a_hi), dal = sdesc(a_lo), dbh = sdesc(b_hi),
                           dbl = sdesc(b_lo);
            for (int k = 0; k < nk8; ++k) {
              const uint64_t ko = 2 * k;
              // small terms first: lo.hi, hi.lo, then hi.hi (lo.lo is below
              // the FP32 accumulation error and is left out)
              mma_tf32(d, dal + ko, dbh + ko, id, accum);
              accum = 1;
              mma_tf32(d, dah + ko, dbl + ko, id, 1);
              mma_tf32(d, dah + ko, dbh + ko, id, 1);
            }
            mma_commit(smem_u32(&sh->empty[st]));
            mma_commit(smem_u32(&sh->lo_empty[ls]));
          }
        }
        // every work item has K >= 1, so the accumulator always holds data
        mma_commit(smem_u32(&sh->acc_full[acc]));
      }
    }
  } else if (warp >= 6) {
    // ---------------- converters (warps 6..13) ----------------
    // For every chunk (same order as the producer) write the low parts
    // lo = rna_tf32(x - trunc_tf32(x)) of the FP32 operand tiles next to
    // them; the tensor core reads the FP32 tile itself as the high part (it
    // uses the top 19 bits), so hi + lo carries x to ~2^-22.  The layout is
    // elementwise, so the swizzled tile maps to the same swizzled offsets.
    const int tid = threadIdx.x - 6 * 32;
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < nwork && ok; t += gridDim.x) {
      const TWork w = works[t];
      int nk = 0;
      if (w.R > 1) {
        nk = w.nchunk;
      } else {
        for (int s = 0; s < w.nseg; ++s) nk += (segs[w.seg0 + s].K + BK - 1) / BK;
      }
      const int n4 = (TILE_A + w.ntile * BK * 4) / 16;   // float4s of the A and B chunks
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int st = it % STAGES, ls = it % LO;
        if (!wait_or_abort(smem_u32(&sh->full[st]), (it / STAGES) & 1, err, 5, abort_flag) ||
            !wait_or_abort(smem_u32(&sh->lo_empty[ls]), ((it / LO) & 1) ^ 1, err, 6, abort_flag)) {
          ok = false;
          break;
        }
        // A (16 KB) and B (ntile rows) are contiguous in both slots
        const uint32_t src = smem_u32(smem + st * STAGE_BYTES);
        const uint32_t dst = smem_u32(lo_ring + ls * STAGE_BYTES);
#pragma unroll 4
        for (int i = tid; i < n4; i += NCONV) lo_split4(src + 16 * i, dst + 16 * i);
        fence_async_shared();
        mbar_arrive(smem_u32(&sh->lo_full[ls]));
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    // Each lane holds one accumulator row.  Per 32-column block the warp
    // stages its 32 x 32 sub-tile in shared memory in the 128-byte-swizzled
    // box layout (16-byte chunk q of row r at position q ^ (r & 7)) and one
    // lane stores it by TMA; the tensor map clips rows and columns outside
    // the destination.
    const int quarter = warp & 3;            // TMEM lanes 32*quarter .. +31
    const uint32_t stg = smem_u32(stage_out + (warp - 2) * 4096);
    const uint32_t rowoff = (uint32_t)lane * 128;
    int j = 0;
    for (int t = blockIdx.x; t < nwork; t += gridDim.x, ++j) {
      const TWork w = works[t];
      const int acc = j % NACC;
      const uint32_t aph = (j / NACC) & 1;
      if (!wait_or_abort(smem_u32(&sh->acc_full[acc]), aph, err, 4, abort_flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tbase = tmem + acc * ACC_COLS + ((uint32_t)(quarter * 32) << 16);
      // destination of this warp's rows: a plain tile, or the diagonal block
      // of its group in a packed tile
      int row0 = w.m0 + quarter * 32, cbeg = 0, cend = w.ntile, xoff = w.n0, mo = w.mOut_hi,
          zo = w.zout;
      bool live = row0 < w.M;
      if (w.R > 1) {
        const int per = 4 / w.R, r = quarter / per, gw = w.ntile / w.R;
        row0 = (quarter % per) * 32;
        cbeg = r * gw;
        cend = cbeg + gw;
        xoff = -cbeg;
        mo = w.pout[r];
        zo = w.pz[r];
        live = w.pseg[r] >= 0;
      }
      if (live) {
        for (int c0 = cbeg; c0 < cend && (w.R > 1 || w.n0 + c0 < w.N); c0 += 32) {
          float v[32];
          tmem_ld16(tbase + c0, v);
          if (c0 + 16 < w.ntile) {
            tmem_ld16(tbase + c0 + 16, v + 16);
          } else {
#pragma unroll
            for (int i = 16; i < 32; ++i) v[i] = 0.f;
          }
          if (lane == 0) bulk_wait_read();
          __syncwarp();
          const float al = w.mode == TW_SPLIT ? w.alpha : 1.f;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            st_shared_v4(stg + rowoff + ((uint32_t)(q ^ (lane & 7)) << 4), al * v[4 * q],
                         al * v[4 * q + 1], al * v[4 * q + 2], al * v[4 * q + 3]);
          fence_async_shared();
          __syncwarp();
          if (lane == 0) {
            tma_store3d(&maps[mo], xoff + c0, row0, zo, stg);
            bulk_commit();
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&sh->acc_empty[acc]))
                   : "memory");
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

}  // namespace

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

int encode_map(CUtensorMap *out, const float *base, int rows, int cols, long long ld,
               int box_rows) {
  static const EncodeFn fn = [] {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeFn) nullptr;
    return (EncodeFn)p;
  }();
  if (!fn) return -1;
  if (((uintptr_t)base & 15) || (ld & 3) || rows <= 0 || cols <= 0) return -2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -3;
}

int encode_map3(CUtensorMap *out, const float *base, long long d0, long long d1, long long d2,
                long long s1, long long s2, int box0, int box1, int box2) {
  static const EncodeFn fn = [] {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeFn) nullptr;
    return (EncodeFn)p;
  }();
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

template <int NT>
cudaError_t prepare_nt() {
  return cudaFuncSetAttribute(k_tf32_gemm<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Geo<NT>::SMEM_BYTES);
}

cudaError_t tf32_prepare() {
  cudaError_t e = prepare_nt<32>();
  if (e == cudaSuccess) e = prepare_nt<64>();
  if (e == cudaSuccess) e = prepare_nt<128>();
  return e;
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

// (the shared-memory attributes are set by tf32_prepare, outside any capture)
template <int NT>
cudaError_t launch_nt(const TWork *work, int nwork, const TSeg *seg, const CUtensorMap *maps,
                      int *err, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  const int nsm = sm_count();
  const int grid = nwork < nsm ? nwork : nsm;
  k_tf32_gemm<NT><<<grid, NTHREADS, Geo<NT>::SMEM_BYTES, s>>>(work, nwork, seg, maps, err);
  return cudaGetLastError();
}

cudaError_t tf32_gemm(const TWork *work, const int *nwork3, const TSeg *seg,
                      const CUtensorMap *maps, int *err, cudaStream_t s) {
  // work items are grouped by tile width: [<= 32 | <= 64 | <= 128]
  cudaError_t e = launch_nt<32>(work, nwork3[0], seg, maps, err, s);
  if (e != cudaSuccess) return e;
  e = launch_nt<64>(work + nwork3[0], nwork3[1], seg, maps, err, s);
  if (e != cudaSuccess) return e;
  return launch_nt<128>(work + nwork3[0] + nwork3[1], nwork3[2], seg, maps, err, s);
}

}  // namespace dmrg
