// Split-precision (3 x TF32) H_eff*psi on the 5th-generation tensor cores.
//
// Operands are FP64 numbers split as x = hi + lo (both TF32); a product is
// hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory (TMEM).  All
// operands are K-major row-major float matrices whose row stride is a
// multiple of 4 floats; tiles are fetched by TMA with 128-byte swizzle.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace dmrg {

// One K-segment: A (M x K) and B (N x K), each as (hi, lo) tensor maps.
struct TSeg {
  int mA_hi, mA_lo, mB_hi, mB_lo;   // indices into the tensor-map table (FP32
                                    // operands use the _hi map only)
  int K;             // length of this K range
  int k0;            // first K index (multiple of 32)
  int xoob;          // a K coordinate past the maps' extent (loads read zeros)
  int pad;
};

// Epilogue of a work item.
enum { TW_SPLIT = 0,      // stage 1: alpha * C stored to T (FP32)
       TW_PARTIAL = 1 };  // stage 2: C stored as an FP32 partial tile (split-K slot)

// One 128 x ntile output tile.  The epilogue stores it by TMA through 3-D
// tensor maps (x column, y row, z slot) with 32 x 32 boxes; the maps clip
// rows and columns outside the destination.
struct TWork {
  int seg0, nseg;
  int M, N;          // full problem extent (rows, columns)
  int m0, n0;        // tile origin
  int ntile;         // UMMA N of this tile (multiple of 16, <= 128)
  int mode;          // TW_SPLIT or TW_PARTIAL
  float alpha;
  int mOut_hi, mOut_lo;   // store map (mOut_lo unused)
  int zout;               // z coordinate of the destination (partial slot)
  // Packed partial tiles (R = 2 or 4; R = 1 otherwise): R independent
  // segments, each with at most 128/R rows and columns, share one MMA
  // tile: group r occupies rows and columns [r*128/R, (r+1)*128/R) and the
  // diagonal block r of the product is its partial tile (the off-diagonal
  // blocks are discarded).  One tensor instruction then advances R
  // segments.  pseg[r] < 0 marks an unused group.
  int R, nchunk;
  int pseg[4], pout[4], pz[4];
};

// FP64 sum of the split-K partial tiles of one sigma block (rows x cols,
// partial rows ld floats apart, ld and stride multiples of 4, ws 16-byte
// aligned): sigma[off + r*cols + c] = sum_p ws[p*stride + r*ld + c],
// summed in a fixed order.
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

struct Tf32Plan {
  // operand storage (FP32, padded rows; the kernels split it on chip)
  float *A32 = nullptr;                // [a'][k][a], rows 16-byte aligned
  float *B32 = nullptr;                // [b'][k][b], b padded to 4 floats
  float *T32 = nullptr;                // [a'][k][b], b padded to 4 floats
  float *P32 = nullptr;                // psi^T per block, [b][a]
  CUtensorMap *maps = nullptr;      // device copy of the tensor maps
  TSeg *seg = nullptr;
  TWork *work1 = nullptr, *work2 = nullptr;
  int nwork1 = 0, nwork2 = 0;
  int n1[3] = {0, 0, 0}, n2[3] = {0, 0, 0};   // per tile-width bucket
  float *ws = nullptr;              // split-K partial tiles of stage 2
  PartialSum *psum = nullptr;
  int npsum = 0;
  void *psi_split = nullptr;        // SplitT descriptors (device), one per psi block
  int npsi = 0;
  int *err = nullptr;               // device error flag (bounded waits)
};

// Encode a 2-D tensor map over a row-major float matrix (rows x cols,
// row stride ld floats, ld % 4 == 0, base 16-byte aligned) with a
// (32 x box_rows) box and 128-byte swizzle.  Returns 0 on success.
int encode_map(CUtensorMap *out, const float *base, int rows, int cols, long long ld,
               int box_rows);

// Encode a 3-D tensor map (d0 innermost; strides s1, s2 in floats, multiples
// of 4) with a (box0 x box1 x box2) box and 128-byte swizzle (box0 = 32).
int encode_map3(CUtensorMap *out, const float *base, long long d0, long long d1, long long d2,
                long long s1, long long s2, int box0, int box1, int box2);

// Device address and size of the fixed scratch array (heff_static.cu); the
// first call on a device looks the address up.
cudaError_t static_scratch(void **ptr, size_t *bytes);

cudaError_t sum_partials(const PartialSum *p, int n, double *sigma, cudaStream_t s);

// Sets the kernels' shared-memory attributes (call before any stream capture).
cudaError_t tf32_prepare();

// work holds nwork3[0] items with ntile <= 32, then nwork3[1] with ntile <= 64,
// then nwork3[2] with ntile <= 128 (one launch each, pipeline sized to the width).
cudaError_t tf32_gemm(const TWork *work, const int *nwork3, const TSeg *seg,
                      const CUtensorMap *maps, int *err, cudaStream_t s);

}  // namespace dmrg
