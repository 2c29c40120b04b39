// FP64 kernels of the DMRG hot path and its helpers (sm_103a).
//
//  * k_gemm_f64   grouped, batched, segmented FP64 GEMM with arbitrary element
//                 strides: block-operator renormalisation (A' = T^T A T), the
//                 FP64 H_eff*psi stages and small helper products.
//  * k_gather     builds enlarged-block operators L. = L x site and
//                 .R = site x R as sums of (block op) x (site matrix) products
//                 with the fermionic sign of the operator ordering.
//  * k_stack_copy copies (transposed, scaled) operator blocks into the
//                 interleaved H_eff term stacks.
//  * Davidson BLAS-1: dots, linear combinations, preconditioner, start vector.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace dmrg {

// ----------------------------------------------------------------------------
// grouped FP64 GEMM: TM x TN tiles (16, 32 or 64 each), K chunk 16, 256
// threads, (TM/16) x (TN/16) outputs per thread.  The host picks the tile
// shape per descriptor, and may fold a batch of problems that share one
// operand into the rows or columns of a single problem (small operator blocks
// would otherwise waste most of a tile).
// ----------------------------------------------------------------------------
constexpr int GK = 16;

template <int TM, int TN>
__global__ void __launch_bounds__(256)
k_gemm_f64(const GemmDesc *__restrict__ descs, int nd,
           const GemmSeg *__restrict__ segs, long long total,
           const double *__restrict__ bindB, double *__restrict__ bindC) {
  constexpr int RM = TM / 16, RN = TN / 16;
  __shared__ double As[GK][TM + 1];
  __shared__ double Bs[GK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    // locate descriptor: last d with tile0 <= t
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (descs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const GemmDesc d = descs[lo];
    long long lt = t - d.tile0;
    const int per_b = d.tiles_m * d.tiles_n;
    const int b = d.fold ? 0 : (int)(lt / per_b);
    const int rem = (int)(lt % per_b);
    const int m0 = (rem / d.tiles_n) * TM;
    const int n0 = (rem % d.tiles_n) * TN;
    const int Mt = d.fold == 1 ? d.batch * d.M : d.M;
    const int Nt = d.fold == 2 ? d.batch * d.N : d.N;
    double acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = 0.0;
    for (int sgi = 0; sgi < d.nseg; ++sgi) {
      const GemmSeg sg = segs[d.seg0 + sgi];
      const double *A = sg.A + (long long)b * sg.a_bs;
      // a NULL operand pointer means "bound vector + offset" (psi at apply time)
      const double *B = sg.B ? sg.B + (long long)b * sg.b_bs : bindB + sg.b_bs;
      for (int k0 = 0; k0 < sg.K; k0 += GK) {
#pragma unroll
        for (int j = 0; j < RM; ++j) {
          int idx = tid + 256 * j;
          int kk = idx & 15, r = idx >> 4;
          int m = m0 + r, k = k0 + kk;
          double v = 0.0;
          if (m < Mt && k < sg.K) {
            if (d.fold == 1) {
              const int bb = m / d.M;
              v = A[(long long)bb * sg.a_bs + (m - bb * d.M) * sg.a_rs + k * sg.a_cs];
            } else {
              v = A[m * sg.a_rs + k * sg.a_cs];
            }
          }
          As[kk][r] = v;
        }
#pragma unroll
        for (int j = 0; j < RN; ++j) {
          int idx = tid + 256 * j;
          int kb = idx / TN, c = idx % TN;
          int n = n0 + c, k2 = k0 + kb;
          double v = 0.0;
          if (n < Nt && k2 < sg.K) {
            if (d.fold == 2) {
              const int bb = n / d.N;
              v = B[(long long)bb * sg.b_bs + k2 * sg.b_rs + (n - bb * d.N) * sg.b_cs];
            } else {
              v = B[k2 * sg.b_rs + n * sg.b_cs];
            }
          }
          Bs[kb][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
          double a[RM], bb[RN];
#pragma unroll
          for (int i = 0; i < RM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < RN; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
      }
    }
    double *C = d.C ? d.C + (long long)b * d.c_bs : bindC + d.c_bs;
#pragma unroll
    for (int i = 0; i < RM; ++i) {
      int m = m0 + ty + 16 * i;
      if (m >= Mt) continue;
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        int n = n0 + tx + 16 * j;
        if (n >= Nt) continue;
        long long o;
        if (d.fold == 1) {
          const int bb = m / d.M;
          o = (long long)bb * d.c_bs + (m - bb * d.M) * d.c_rs + n * d.c_cs;
        } else if (d.fold == 2) {
          const int bb = n / d.N;
          o = (long long)bb * d.c_bs + m * d.c_rs + (n - bb * d.N) * d.c_cs;
        } else {
          o = m * d.c_rs + n * d.c_cs;
        }
        double *p = C + o;
        double v = d.alpha * acc[i][j];
        if (d.beta != 0.0) v += d.beta * *p;
        *p = v;
      }
    }
  }
}

#define GEMM_F64_CASE(a, b)                                                              \
  if (tm == a && tn == b) {                                                              \
    k_gemm_f64<a, b><<<(unsigned)grid, 256, 0, s>>>(d_desc, ndesc, d_seg, total_tiles,   \
                                                    bindB, bindC);                       \
    return cudaGetLastError();                                                           \
  }

cudaError_t launch_gemm_f64(const GemmDesc *d_desc, int ndesc,
                            const GemmSeg *d_seg, long long total_tiles,
                            cudaStream_t s, const double *bindB, double *bindC, int tm,
                            int tn) {
  if (ndesc <= 0 || total_tiles <= 0) return cudaSuccess;
  long long grid = total_tiles < (1LL << 20) ? total_tiles : (1LL << 20);
  GEMM_F64_CASE(16, 16)
  GEMM_F64_CASE(32, 32)
  GEMM_F64_CASE(64, 64)
  GEMM_F64_CASE(64, 16)
  GEMM_F64_CASE(16, 64)
  return cudaErrorInvalidValue;
}
#undef GEMM_F64_CASE

// ----------------------------------------------------------------------------
// Kronecker gather for enlarged-block operators
// ----------------------------------------------------------------------------
constexpr int GOPS = 8;   // operators per CTA

__global__ void __launch_bounds__(256)
k_gather(const GSub *__restrict__ subs, const GTerm *__restrict__ terms,
         const GSrc *__restrict__ srcs, int dsite) {
  const GSub s = subs[blockIdx.x];
  const int k0 = blockIdx.y * GOPS;
  if (k0 >= s.nops) return;
  const int k1 = min(k0 + GOPS, s.nops);
  const int nel = s.rows * s.cols;
  const int sidx = s.so * dsite + s.si;   // dsite = 4 (frame width)
  const bool odd_in = (s.n_in & 1) != 0;
  for (int k = k0; k < k1; ++k) {
    const int t0 = s.term_ptr[k], t1 = s.term_ptr[k + 1];
    double *out = s.out + (long long)k * s.nnz_out + s.out_off;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int r = e / s.cols, c = e - r * s.cols;
      double acc = 0.0;
      for (int ti = t0; ti < t1; ++ti) {
        const GTerm &T = terms[ti];
        double w = T.m[sidx];
        if (w == 0.0) continue;
        if (s.ctab) w *= s.ctab[T.ctype];
        if (T.p2 && odd_in) w = -w;
        double v;
        if (T.src < 0) {
          v = (s.a_out == s.a_in && r == c) ? 1.0 : 0.0;
        } else {
          const GSrc src = srcs[T.src];
          if (!T.trans) {
            int bi = src.in2blk[s.a_in];
            if (bi < 0 || src.blk_out[bi] != s.a_out) continue;
            v = src.d[(long long)T.idx * src.nnz + src.blk_off[bi] + (long long)r * s.cols + c];
          } else {
            int bi = src.in2blk[s.a_out];
            if (bi < 0 || src.blk_out[bi] != s.a_in) continue;
            v = src.d[(long long)T.idx * src.nnz + src.blk_off[bi] + (long long)c * s.rows + r];
          }
        }
        acc = fma(w, v, acc);
      }
      out[(long long)r * s.out_ld + c] = acc;
    }
  }
}

cudaError_t launch_gather(const GSub *d_sub, int nsub, int max_ops,
                          const GTerm *d_terms, const GSrc *d_src, int d,
                          cudaStream_t s) {
  if (nsub <= 0 || max_ops <= 0) return cudaSuccess;
  dim3 grid(nsub, (max_ops + GOPS - 1) / GOPS);
  k_gather<<<grid, 256, 0, s>>>(d_sub, d_terms, d_src, d);
  return cudaGetLastError();
}

__global__ void k_sum_partials64(const PartialSum64 *__restrict__ ps, double *__restrict__ out) {
  const PartialSum64 p = ps[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < p.nparts; ++k) acc += p.ws[k * p.stride + i];
    out[p.off + i] = acc;
  }
}

cudaError_t launch_sum_partials64(const PartialSum64 *p, int n, double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(8, n);
  k_sum_partials64<<<grid, 256, 0, s>>>(p, out);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// stack copy
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_stack_copy(const SCopy *__restrict__ cps) {
  const SCopy c = cps[blockIdx.x];
  const int nel = c.rows * c.cols;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < nel; e += gridDim.y * blockDim.x) {
    const int r = e / c.cols, q = e - r * c.cols;
    double v;
    if (c.src == nullptr) {
      v = (c.ident && r == q) ? c.coef : 0.0;
    } else {
      v = c.coef * (c.trans ? c.src[(long long)q * c.src_ld + r]
                            : c.src[(long long)r * c.src_ld + q]);
    }
    c.dst[(long long)r * c.dst_ld + q] = v;
  }
}

cudaError_t launch_stack_copy(const SCopy *d_cp, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(n, 4);
  k_stack_copy<<<grid, 256, 0, s>>>(d_cp);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Davidson BLAS-1
// ----------------------------------------------------------------------------
constexpr int DOT_BLOCKS = 296;   // 2 x 148 SMs

__global__ void __launch_bounds__(256)
k_dots_partial(const double *__restrict__ V, int k, long long ld,
               const double *__restrict__ x, long long n, double *__restrict__ work) {
  __shared__ double red[256];
  for (int i = 0; i < k; ++i) {
    double acc = 0.0;
    const double *v = V + i * ld;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
      acc = fma(v[j], x[j], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) work[i * gridDim.x + blockIdx.x] = red[0];
    __syncthreads();
  }
}

__global__ void k_dots_final(const double *__restrict__ work, int nb, int k,
                             double *__restrict__ out) {
  __shared__ double red[256];
  for (int i = 0; i < k; ++i) {
    double acc = 0.0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) acc += work[i * nb + j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = red[0];
    __syncthreads();
  }
}

cudaError_t launch_dots(const double *V, int k, long long ld, const double *x,
                        long long n, double *work, double *out, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  k_dots_partial<<<DOT_BLOCKS, 256, 0, s>>>(V, k, ld, x, n, work);
  k_dots_final<<<1, 256, 0, s>>>(work, DOT_BLOCKS, k, out);
  return cudaGetLastError();
}

__global__ void k_lincomb(double *__restrict__ out, const double *__restrict__ V,
                          int k, long long ld, const double *__restrict__ coef,
                          const double *__restrict__ a, long long n) {
  const double a0 = a ? *a : 0.0;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double v = (a0 != 0.0) ? a0 * out[j] : 0.0;
    for (int i = 0; i < k; ++i) v = fma(coef[i], V[i * ld + j], v);
    out[j] = v;
  }
}

cudaError_t launch_lincomb(double *out, const double *V, int k, long long ld,
                           const double *coef, const double *a, long long n,
                           cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_lincomb<<<(unsigned)blocks, 256, 0, s>>>(out, V, k, ld, coef, a, n);
  return cudaGetLastError();
}

__global__ void k_lincomb_v(double *__restrict__ out, const double *__restrict__ V, int k,
                            long long ld, const __grid_constant__ LincombCoef c, double a,
                            long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double v = (a != 0.0) ? a * out[j] : 0.0;
    for (int i = 0; i < k; ++i) v = fma(c.c[i], V[i * ld + j], v);
    out[j] = v;
  }
}

cudaError_t launch_lincomb_v(double *out, const double *V, int k, long long ld,
                             const LincombCoef &c, double a, long long n, cudaStream_t s) {
  if (k < 0 || k > kLincombMax) return cudaErrorInvalidValue;
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_lincomb_v<<<(unsigned)blocks, 256, 0, s>>>(out, V, k, ld, c, a, n);
  return cudaGetLastError();
}

__global__ void k_lincomb_d(double *__restrict__ out, const double *__restrict__ V, int k,
                            long long ld, const double *__restrict__ c, double cs, double a,
                            long long n) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double v = (a != 0.0) ? a * out[j] : 0.0;
    for (int i = 0; i < k; ++i) v = fma(cs * c[i], V[i * ld + j], v);
    out[j] = v;
  }
}

cudaError_t launch_lincomb_d(double *out, const double *V, int k, long long ld,
                             const double *c, double cs, double a, long long n, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_lincomb_d<<<(unsigned)blocks, 256, 0, s>>>(out, V, k, ld, c, cs, a, n);
  return cudaGetLastError();
}

__global__ void k_precond(double *__restrict__ r, const double *__restrict__ diag,
                          const double *__restrict__ theta, long long n) {
  const double th = *theta;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    double den = diag[j] - th;
    if (fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
    r[j] = r[j] / den;
  }
}

cudaError_t launch_precond(double *r, const double *diag, const double *theta,
                           long long n, cudaStream_t s) {
  if (!diag) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_precond<<<(unsigned)blocks, 256, 0, s>>>(r, diag, theta, n);
  return cudaGetLastError();
}

// splitmix64 -> uniform in [-1, 1)
__global__ void k_random(double *x, long long n, uint64_t seed) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(j + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    x[j] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

cudaError_t launch_random(double *x, long long n, uint64_t seed, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_random<<<(unsigned)blocks, 256, 0, s>>>(x, n, seed);
  return cudaGetLastError();
}

__global__ void k_scale(double *x, const double *c, int invert_sqrt, long long n) {
  double f = *c;
  if (invert_sqrt) f = 1.0 / sqrt(f);
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x)
    x[j] *= f;
}

cudaError_t launch_scale(double *x, const double *c, int invert_sqrt, long long n,
                         cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_scale<<<(unsigned)blocks, 256, 0, s>>>(x, c, invert_sqrt, n);
  return cudaGetLastError();
}

__global__ void k_select_cols(const double *__restrict__ evec, int ld, int rows,
                              const int *__restrict__ cols, int ncols,
                              double *__restrict__ out) {
  const long long n = (long long)rows * ncols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / ncols), j = (int)(e % ncols);
    out[e] = evec[(long long)cols[j] * ld + r];
  }
}

cudaError_t launch_select_cols(const double *evec, int ld, int rows,
                               const int *cols, int ncols, double *out,
                               cudaStream_t s) {
  long long n = (long long)rows * ncols;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_select_cols<<<(unsigned)blocks, 256, 0, s>>>(evec, ld, rows, cols, ncols, out);
  return cudaGetLastError();
}

}  // namespace dmrg
