// Internal kernel interfaces of libdmrgb300 (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmrg {

// One K-segment of a grouped GEMM: C += A_seg * B_seg, with arbitrary
// element strides so that transposed and interleaved operands need no copy.
// A(m,k) = A[m*a_rs + k*a_cs + b*a_bs], B(k,n) = B[k*b_rs + n*b_cs + b*b_bs].
struct GemmSeg {
  const double *A;
  const double *B;
  long long a_rs, a_cs, a_bs;
  long long b_rs, b_cs, b_bs;
  int K;
  int pad;
};

// C(m,n) = alpha * sum_seg A_seg B_seg + beta * C, for `batch` independent
// problems; C(m,n) = C[m*c_rs + n*c_cs + b*c_bs].
struct GemmDesc {
  double *C;
  long long c_rs, c_cs, c_bs;
  int M, N, batch;
  int seg0, nseg;
  int tiles_m, tiles_n;
  double alpha, beta;
  long long tile0;   // prefix sum of tiles over descriptors
  // 0: `batch` separate problems; 1: the batch folded into the rows (one
  // problem of batch*M rows, row b*M + m; every segment's B shared, b_bs = 0);
  // 2: folded into the columns (batch*N columns; every segment's A shared)
  int fold;
  int pad;
};

// Source operator class for the Kronecker gather (op-major storage: op k of
// the class starts at d + k*nnz; block b starts at blk_off[b]).
struct GSrc {
  const double *d;
  long long nnz;
  const int *in2blk;     // input sector -> block index or -1
  const int *blk_out;    // block -> output sector
  const long long *blk_off;
};

// One term of an enlarged-block operator: coef * (X-op or identity) x site.
struct GTerm {
  int src;     // index into GSrc table, -1 = identity on the block
  int idx;     // operator index inside the source class
  int trans;   // use the transpose of the block operator
  int p2;      // parity of the second factor of the product
  int ctype;   // spin-adapted parts: index into the sub-block's coefficient table
  int pad;
  double m[16];  // site factor, 4x4 frame m[so*4+si], coefficient folded in
};

// One sub-block (piece pair) of an output block of an enlarged operator
// class.  All operators of the class are written for this rectangle.
struct GSub {
  double *out;           // class base (op-major)
  long long nnz_out;     // elements per operator of the class
  long long out_off;     // offset of the rectangle's (0,0) inside an op
  int out_ld;            // row length of the output block
  int rows, cols;
  int so, si;            // site state index: output row piece, input col piece
  int a_out, a_in;       // block sector indices of the pieces
  int n_in;              // particle number used by the fermion sign
  int nops;
  const int *term_ptr;   // per op CSR into the term array (device)
  // spin-adapted parts: recoupling coefficient of each term type (GTerm::ctype)
  // for this sub-block's spins; NULL: all 1
  const double *ctab;
};

// Copy (optionally transposed, scaled) operator blocks into a stack.
struct SCopy {
  const double *src;     // NULL: identity if ident, else zero
  double *dst;
  long long dst_ld;
  int src_ld;
  int rows, cols;
  int trans, ident;
  double coef;
};


// A segment with B == NULL reads bindB + b_bs; a descriptor with C == NULL
// writes bindC + c_bs (psi / sigma supplied per call, batch must be 1).
cudaError_t launch_gemm_f64(const GemmDesc *d_desc, int ndesc,
                            const GemmSeg *d_seg, long long total_tiles,
                            cudaStream_t s, const double *bindB = nullptr,
                            double *bindC = nullptr, int tm = 64, int tn = 64);
cudaError_t launch_gather(const GSub *d_sub, int nsub, int max_ops,
                          const GTerm *d_terms, const GSrc *d_src, int d,
                          cudaStream_t s);
// FP64 sum of split-K partial blocks: out[off + i] = sum_p ws[p*stride + i].
struct PartialSum64 {
  const double *ws;
  long long stride;
  long long off;
  int n;
  int nparts;
};
cudaError_t launch_sum_partials64(const PartialSum64 *p, int n, double *out, cudaStream_t s);

cudaError_t launch_stack_copy(const SCopy *d_cp, int n, cudaStream_t s);

// Davidson helpers (FP64).  V holds k vectors with leading dimension ld.
// dots: out[i] = <V_i, x>, two-pass deterministic reduction (work >= 64*k).
cudaError_t launch_dots(const double *V, int k, long long ld,
                        const double *x, long long n, double *work,
                        double *out, cudaStream_t s);
// out = a * out + sum_i c[i] V_i   (a, c on the device)
cudaError_t launch_lincomb(double *out, const double *V, int k, long long ld,
                           const double *coef, const double *a, long long n,
                           cudaStream_t s);
// The same with the coefficients passed by value (k <= kLincombMax): no copy
// to the device and nothing for the host to wait on.
constexpr int kLincombMax = 64;
struct LincombCoef {
  double c[kLincombMax];
};
cudaError_t launch_lincomb_v(double *out, const double *V, int k, long long ld,
                             const LincombCoef &c, double a, long long n, cudaStream_t s);
// out = a * out + cs * sum_i c[i] V_i with c on the device (e.g. the result of
// launch_dots, cs = -1 for a projection step)
cudaError_t launch_lincomb_d(double *out, const double *V, int k, long long ld,
                             const double *c, double cs, double a, long long n, cudaStream_t s);
// r = (r) / (diag - theta) with clamping; diag may be NULL (no-op scale 1)
cudaError_t launch_precond(double *r, const double *diag, const double *theta,
                           long long n, cudaStream_t s);
cudaError_t launch_random(double *x, long long n, uint64_t seed,
                          cudaStream_t s);
cudaError_t launch_scale(double *x, const double *c, int invert_sqrt,
                         long long n, cudaStream_t s);
// Copy selected columns (ascending order list) of a column-major matrix
// (eigenvectors, ld) into a row-major (rows x ncols) matrix, reversed order
// handled by the caller's column list.
cudaError_t launch_select_cols(const double *evec, int ld, int rows,
                               const int *cols, int ncols, double *out,
                               cudaStream_t s);

}  // namespace dmrg
