// Split-precision H_eff*psi on the 5th-generation tensor cores.
//
// Operands are FP64 numbers held as x * s = hi + lo with hi, lo FP16 and s a
// power of two chosen per operator block (per psi block, per stage-1 output
// block) so that |x * s| <= 2^14: a product is lo.hi + hi.lo + hi.hi with FP32
// accumulation in tensor memory (TMEM), and the power-of-two factors are taken
// out exactly in the epilogue.  Elements within 2^17 of their block's scale
// keep ~22 significant bits; smaller ones keep an absolute accuracy of about
// 2^-39 of the block's largest element.  All operand matrices are K-major,
// row strides a multiple of 8 halves (16 bytes); tiles are fetched by TMA
// with 128-byte swizzle (64 halves per row).
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace dmrg {

// One K-segment: A (M x K) and B (N x K), each as (hi, lo) tensor maps.
struct TSeg {
  int mA_hi, mA_lo, mB_hi, mB_lo;   // indices into the tensor-map table
  int K;             // length of this K range
  int k0;            // first K index (multiple of 64)
  int xoob;          // a K coordinate past the maps' extent (loads read zeros)
  int pad;
};

// Epilogue of a work item.
enum { TW_SPLIT = 0,      // stage 1: T = alpha * C, rescaled and split (hi, lo) into T
       TW_PARTIAL = 1 };  // stage 2: C unscaled into an FP32 partial tile (split-K slot)

// One 128 x ntile output tile.  The epilogue stores it by TMA through 3-D
// tensor maps (x column, y row, z slot); the maps clip rows and columns
// outside the destination.  Each CTA copies its work items into shared
// memory with bulk copies a few items ahead, so the size is a multiple of
// 16 bytes.
struct TWork {
  TSeg s;            // the item's K range (packed tiles: that of group 0)
  int M, N;          // full problem extent (rows, columns)
  int m0, n0;        // tile origin
  int ntile;         // UMMA N of this tile (multiple of 16, <= 128)
  int mode;          // TW_SPLIT or TW_PARTIAL
  float alpha;       // fermion sign (stage 1)
  float fa;          // 1 / scale of the entry's operator block (A stack in stage 1, B in stage 2)
  float rn;          // largest row 2-norm of the entry's A stack (sets the scale of T)
  int pblk;          // psi block the entry reads
  int mOut_hi, mOut_lo;   // store maps (T hi, lo; or the partial slots)
  int zout;               // z coordinate of the destination (partial slot)
  // Packed partial tiles (R = 2 or 4; R <= 1 otherwise): R independent
  // segments, each with at most 128/R rows and columns, share one MMA
  // tile: group r occupies rows and columns [r*128/R, (r+1)*128/R) and the
  // diagonal block r of the product is its partial tile (the off-diagonal
  // blocks are discarded).  One tensor instruction then advances R
  // segments.  pseg[r] < 0 marks an unused group.
  int R, nchunk;
  int pseg[4], pout[4], pz[4], ppb[4];
  float pfa[4], prn[4];
  int pad;
};
static_assert(sizeof(TWork) == 192, "TWork is copied in 16-byte units");

// Sum of the split-K partial tiles of one sigma block (rows x cols, partial
// rows ld floats apart, ld and stride multiples of 4, ws 16-byte aligned):
// sigma[off + r*cols + c] = sum_p ws[p*stride + r*ld + c], in a fixed order.
struct PartialSum {
  const float *ws;
  long long stride;
  long long off;
  long long ld;
  int n;             // rows * cols
  int cols;
  int nparts;
  int pad;
};

// Per class entry of the window: largest |element| of its A and B stacks and
// the largest 2-norm of an A-stack row (a row (a', k) has the psi-row length).
struct EntryStat {
  float maxA, rnA, maxB, pad;
};
struct StatDesc {
  const double *a;
  long long rowsA;
  int colsA;
  int pad0;
  const double *b;
  long long rowsB;
  int colsB;
  int pad1;
};

// Per psi block, per apply: largest |element| and largest column 2-norm.
struct PsiStat {
  float mx, cn;
};
struct PsiDesc {
  long long off;     // offset of the block in psi
  int rows, cols;    // da x db, row-major
};

// FP64 matrix -> scaled FP16 (hi, lo), optionally transposed (trans = 1
// writes cols x rows).  scale > 0 is the power of two to apply; scale == 0
// takes the power of two of psi block pblk's statistics (psi^T operands).
// src == NULL reads the bound vector at src_off.
struct F16Split {
  const double *src;
  long long src_ld;
  __half *hi, *lo;
  long long dst_ld;
  int rows, cols;
  int trans;
  int pblk;
  float scale;
  int pad;
  long long src_off;
};

struct SplitPlan {
  // operand storage (FP16 hi, lo; A rows zero-padded to 16 halves, B rows to 8)
  __half *Ah = nullptr, *Al = nullptr;   // [a'][k][a]
  __half *Bh = nullptr, *Bl = nullptr;   // [b'][k][b_pad]
  __half *Th = nullptr, *Tl = nullptr;   // [a'][k][b_pad], per apply
  __half *Ph = nullptr, *Pl = nullptr;   // psi^T per block [b][a], per apply
  PsiStat *pstat = nullptr;              // per psi block, per apply
  CUtensorMap *maps = nullptr;      // device copy of the tensor maps
  TSeg *seg = nullptr;
  TWork *work1 = nullptr, *work2 = nullptr;
  int nwork1 = 0, nwork2 = 0;
  float *ws = nullptr;              // split-K partial tiles of stage 2
  PartialSum *psum = nullptr;
  int npsum = 0;
  void *psi_split = nullptr;        // F16Split descriptors (device), one per psi block
  int npsi = 0;
  int psi_tiles = 1;                // most 32 x 32 tiles of one psi block
  PsiDesc *psi_desc = nullptr;      // psi block extents (device)
  int *err = nullptr;               // device error flag (bounded waits)
  int *next = nullptr;              // device item counters: stage 1, stage 2
};

// Power of two s with |m| * s <= 2^14 (1 for m <= 0); host and device agree.
float pow2_scale_host(float m);

// 2-D tensor map over a row-major FP16 matrix (rows x cols, row stride ld
// halves, ld % 8 == 0, base 16-byte aligned), box 64 x box_rows, 128-byte
// swizzle.  Returns 0 on success.
int encode_map_h(CUtensorMap *out, const __half *base, long long rows, long long cols,
                 long long ld, int box_rows);
// 3-D FP16 map (d0 innermost; strides in halves, multiples of 8), box
// 64 x box1 x box2, 128-byte swizzle.
int encode_map3_h(CUtensorMap *out, const __half *base, long long d0, long long d1,
                  long long d2, long long s1, long long s2, int box1, int box2);
// 3-D FP32 map (strides in floats, multiples of 4), box box0 x box1 x box2
// (box0 * 4 <= 128), 128-byte swizzle.
int encode_map3(CUtensorMap *out, const float *base, long long d0, long long d1, long long d2,
                long long s1, long long s2, int box0, int box1, int box2);

// Device address and size of the fixed scratch array (heff_static.cu); the
// first call on a device looks the address up.
cudaError_t static_scratch(void **ptr, size_t *bytes);

cudaError_t sum_partials(const PartialSum *p, int n, double *sigma, cudaStream_t s);
cudaError_t entry_stats(const StatDesc *d, int n, EntryStat *out, cudaStream_t s);
cudaError_t psi_stats(const PsiDesc *d, int n, const double *psi, PsiStat *out, cudaStream_t s);
// grid_tiles: CTAs per descriptor (each walks the descriptor's 32 x 32 tiles
// with that stride); no more than its tile count is useful.
cudaError_t f16_split(const F16Split *d, int n, const PsiStat *pstat, const double *bind,
                      cudaStream_t s, int grid_tiles = 128);

// One thread waits on a barrier nothing completes; *err (zeroed by the
// caller) receives 7 when the bounded wait gave up as designed, -1 if the
// wait returned success.
cudaError_t wait_selftest(int *err, cudaStream_t s);

// Sets the kernels' shared-memory attributes (call before any stream capture).
cudaError_t split_prepare();

// One launch over nwork items of any tile width (at most 128): persistent
// CTAs claim them in list order from the device counter *next, which is
// zeroed here first.
cudaError_t split_gemm(const TWork *work, int nwork, int *next, const TSeg *seg,
                       const CUtensorMap *maps, const PsiStat *pstat, int *err, cudaStream_t s);

}  // namespace dmrg
