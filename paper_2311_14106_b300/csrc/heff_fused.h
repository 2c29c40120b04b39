// Fused split-precision H_eff*psi for large sigma blocks: both contractions
// of a term in one kernel, the intermediate S = A_k psi kept in tensor memory.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace dmrg {

// One unit of work: term k of one class entry, psi columns [b0, b0 + nb).
//   S[a', b]   = A_k[a', :] . psi[:, b]                  (MMA1, K = psi rows a)
//   sigma_tile += alpha * S[a', b] . B_k[b', b]^T         (MMA2, K = b)
struct FUnit {
  int mA_hi, mA_lo;   // 3-D maps over the A stack [a'][k][a]  (x a, y k, z a')
  int mP_hi, mP_lo;   // 2-D maps over psi^T [b][a]              (x a, y b)
  int mB_hi, mB_lo;   // 3-D maps over the padded B stack [b'][k][b] (x b, y k, z b')
  int k;              // term index (y coordinate of the 3-D maps)
  int b0, nb;         // psi columns of this unit (nb <= 128)
  int n1;             // MMA1 N: nb rounded up to 16
  int ra;             // rows of the A maps' box (a' rows loaded per chunk)
  int pbox;           // rows of the psi^T map's box (bytes expected per load)
  int ka, nk1;        // K of MMA1 (psi rows a) and its 32-wide chunks
  float alpha;        // fermionic sign of the class
};

// One 128 x ntile tile of a sigma block over a range of units; the result is
// an FP32 partial tile (slot zout of the block's 3-D partial map mOut).
struct FWork {
  int u0, nu;
  int M, N;           // sigma block rows (a') and columns (b')
  int m0, n0, ntile;  // tile origin and UMMA N of MMA2 (multiple of 16, <= 128)
  int mOut, zout;
};

// Sets the fused kernels' shared-memory attributes (call outside any capture).
cudaError_t fused_prepare();

// One persistent launch over all tiles (largest first).
cudaError_t fused_gemm(const FWork *works, int nwork, const FUnit *units, const CUtensorMap *maps,
                       int *err, cudaStream_t s);

}  // namespace dmrg
