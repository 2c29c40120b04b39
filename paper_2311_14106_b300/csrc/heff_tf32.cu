// 3 x TF32 grouped GEMM on tcgen05 (sm_103a) for the two H_eff*psi stages.
//
// Stage 1:  T[(a',k), b]  = sign * A_stack[(a',k), a] . psi[a, b]
// Stage 2:  sigma[a', b'] = sum_segments T[a', (k,b)] . B_stack[b', (k,b)]^T
// Both are C = A . B^T with K-major operands.  Each FP64 operand x is held as
// x_hi + x_lo (TF32 each); the product uses hi.hi + hi.lo + lo.hi with FP32
// accumulation in tensor memory.  One CTA computes one 128 x ntile tile:
//   warp 0 (one lane)  TMA producer: A_hi, A_lo, B_hi, B_lo per 32-wide K chunk
//   warp 1 (one lane)  MMA issuer: 4 k-steps x 3 tcgen05.mma per chunk
//   warps 0-3          epilogue: tcgen05.ld of the accumulator rows
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
constexpr int STAGES = 3;
constexpr int TILE_A = BM * BK * 4;          // 16 KB
constexpr int TILE_B = 128 * BK * 4;         // up to 16 KB
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
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

// bounded wait: false (and error recorded) if the phase never completes
__device__ bool mbar_wait(uint32_t a, uint32_t parity, int *err, int code) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try(a, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  atomicCAS(err, 0, code);
  return false;
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

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(128, 1)
k_tf32_gemm(const TWork *__restrict__ works, const TSeg *__restrict__ segs,
            const CUtensorMap *__restrict__ maps, double *__restrict__ out64,
            int *__restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES);
  uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TWork w = works[blockIdx.x];
  const uint32_t full0 = smem_u32(&bars[0]);
  const uint32_t empty0 = smem_u32(&bars[STAGES]);
  const uint32_t done = smem_u32(&bars[2 * STAGES]);

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // number of K chunks over all segments
  int nchunks = 0;
  for (int s = 0; s < w.nseg; ++s) nchunks += (segs[w.seg0 + s].K + BK - 1) / BK;
  const uint32_t tile_b_bytes = (uint32_t)w.ntile * BK * 4;
  const uint32_t stage_tx = 2 * TILE_A + 2 * tile_b_bytes;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int it = 0;
    for (int s = 0; s < w.nseg && !*abort_flag; ++s) {
      const TSeg sg = segs[w.seg0 + s];
      const int nk = (sg.K + BK - 1) / BK;
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int st = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        if (!mbar_wait(empty0 + 8 * st, ph ^ 1, err, 1)) {
          *abort_flag = 1;
          break;
        }
        uint8_t *base = smem + st * STAGE_BYTES;
        const uint32_t fb = full0 + 8 * st;
        mbar_expect_tx(fb, stage_tx);
        const int kx = sg.k0 + kc * BK;
        tma_load(smem_u32(base), &maps[sg.mA_hi], kx, w.m0, fb);
        tma_load(smem_u32(base + TILE_A), &maps[sg.mA_lo], kx, w.m0, fb);
        tma_load(smem_u32(base + 2 * TILE_A), &maps[sg.mB_hi], kx, w.n0, fb);
        tma_load(smem_u32(base + 2 * TILE_A + TILE_B), &maps[sg.mB_lo], kx, w.n0, fb);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t id = idesc_tf32(w.ntile);
    uint32_t accum = 0;
    for (int it = 0; it < nchunks; ++it) {
      const int st = it % STAGES;
      const uint32_t ph = (it / STAGES) & 1;
      if (*abort_flag || !mbar_wait(full0 + 8 * st, ph, err, 2)) {
        *abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(smem + st * STAGE_BYTES);
      const uint32_t a_lo = a_hi + TILE_A;
      const uint32_t b_hi = a_hi + 2 * TILE_A;
      const uint32_t b_lo = b_hi + TILE_B;
#pragma unroll
      for (int k = 0; k < BK / 8; ++k) {
        const uint32_t ko = k * 32;   // 8 tf32 = 32 bytes along the swizzled row
        mma_tf32(tmem, sdesc(a_lo + ko), sdesc(b_hi + ko), id, accum);
        accum = 1;
        mma_tf32(tmem, sdesc(a_hi + ko), sdesc(b_lo + ko), id, 1);
        mma_tf32(tmem, sdesc(a_hi + ko), sdesc(b_hi + ko), id, 1);
      }
      mma_commit(empty0 + 8 * st);
    }
    if (nchunks == 0 || *abort_flag) {
      // nothing accumulated: signal completion without MMA
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(done) : "memory");
    } else {
      mma_commit(done);
    }
    if (nchunks == 0) accum = 0;
    // remember whether the accumulator holds data
    if (accum == 0) *abort_flag = *abort_flag ? 1 : 2;
  }
  __syncwarp();

  // ---------------- epilogue ----------------
  const bool ok = mbar_wait(done, 0, err, 3);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const int flag = *abort_flag;
  if (ok && flag != 1) {
    const int row = w.m0 + warp * 32 + lane;
    const bool zero = (flag == 2);
    for (int c0 = 0; c0 < w.ntile; c0 += 16) {
      float v[16];
      if (!zero) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (row >= w.M) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = w.n0 + c0 + i;
        if (col >= w.N) break;
        const float x = w.alpha * v[i];
        if (w.mode == 0) {
          const long long o = (long long)(row / w.nrep) * w.ld + (long long)(row % w.nrep) * w.rep + col;
          const float h = tf32_round(x);
          w.out_hi[o] = h;
          w.out_lo[o] = tf32_round(x - h);
        } else if (w.mode == 1) {
          out64[w.off64 + (long long)row * w.ld + col] = (double)x;
        } else {
          w.out32[(long long)row * w.ld + col] = x;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128)
                 : "memory");
  }
}

}  // namespace

__global__ void k_sum_partials(const PartialSum *__restrict__ ps, double *__restrict__ sigma) {
  const PartialSum p = ps[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < p.nparts; ++k) acc += (double)p.ws[k * p.stride + i];
    sigma[p.off + i] = acc;
  }
}

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                             const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                             const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_map(CUtensorMap *out, const float *base, int rows, int cols, long long ld,
               int box_rows) {
  static EncodeFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return -1;
    fn = (EncodeFn)p;
  }
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

cudaError_t sum_partials(const PartialSum *p, int n, double *sigma, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(8, n);
  k_sum_partials<<<grid, 256, 0, s>>>(p, sigma);
  return cudaGetLastError();
}

cudaError_t tf32_gemm(const TWork *work, int nwork, const TSeg *seg, const CUtensorMap *maps,
                      double *out64, int *err, cudaStream_t s) {
  if (nwork <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tf32_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_tf32_gemm<<<nwork, 128, SMEM_BYTES, s>>>(work, seg, maps, out64, err);
  return cudaGetLastError();
}

}  // namespace dmrg
