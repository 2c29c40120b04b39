// Host runtime of libdmrgb300: Hamiltonian set-up (Eq. 1, Sec. II.B
// rotation), sector tables ("Tables", Sec. III.B), block operators
// (normal and complementary), the two-site window, H_eff*psi, Davidson,
// truncation and sweeps.  All bulk arithmetic runs in the CUDA kernels of
// kernels.cu / heff_split.cu; this file builds their work lists.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <shared_mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dmrg_b300.h"
#include "formulas.h"
#include "heff_split.h"
#include "kernels.h"
#include "model.h"
#include "su2.h"

using namespace dmrg;

namespace {

struct Err {
  int code;
  std::string msg;
};

#define CK(call)                                                            \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess)                                                  \
      throw Err{DMRG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

[[noreturn]] void fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  throw Err{code, buf};
}

double now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Iso {
  std::vector<QN> qn;
  std::vector<int> rows, cols;
  std::vector<double> host;        // concatenated row-major
  std::vector<long long> off;
  double *d = nullptr;
};

// cudaMalloc / cudaFree synchronise the device, which would invalidate a CUDA
// graph capture running in another thread (several contexts are served
// concurrently).  Allocation and release take this lock shared; a capture
// takes it exclusively for the few microseconds it lasts.
std::shared_mutex &capture_lock() {
  static std::shared_mutex mu;
  return mu;
}

// Device buffers that live together (one H_eff window, one block, one
// call's work lists) and are released together.  Requests of up to 64 KB
// (descriptor tables, small work lists: hundreds per window) are carved from
// 1 MB chunks, so they cost no cudaMalloc / cudaFree of their own (cudaFree
// synchronises the whole device, which stalls concurrent solves).  Every
// returned pointer is 256-byte aligned, as cudaMalloc's are.
//
// A buffer set bound to a stream (the temporaries of one call, all used on
// that stream) allocates and frees stream-ordered from the device's memory
// pool instead: no device-wide synchronisation, and the pool reuses the
// memory once the stream has passed the free.
void keep_pool_memory() {
  // the pool keeps up to 8 GB of freed memory for reuse (a property of this
  // process's pool object only)
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(mu);
  if (!done.insert(dev).second) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = 8ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
}

// Stream on which long-lived buffers are taken from and returned to the pool
// (one per device, non-blocking).  An allocation is synchronised before use,
// and the buffers' last users have finished when they are released (the
// calls that use them end with a stream synchronisation), so neither needs
// ordering against the callers' streams.
// (Never throws: it also runs in destructors; the legacy stream stands in if
// no stream can be made.)
cudaStream_t release_stream() {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  cudaStream_t &r = streams[dev];
  if (!r && cudaStreamCreateWithFlags(&r, cudaStreamNonBlocking) != cudaSuccess) r = nullptr;
  return r;
}

struct WinBuf {
  static constexpr size_t kChunk = 1 << 20, kSmall = 64 << 10;
  std::vector<void *> ptrs;
  char *cur = nullptr;   // free part of the current small-request chunk
  size_t left = 0;
  cudaStream_t st = nullptr;
  bool ordered = false;  // stream-ordered (pool) allocation on st
  bool lasting = false;  // pool allocation on release_stream() (long-lived buffers)
  WinBuf() = default;
  explicit WinBuf(cudaStream_t s) : st(s), ordered(true) {}
  // owns its allocations: movable, not copyable
  WinBuf(const WinBuf &) = delete;
  WinBuf &operator=(const WinBuf &) = delete;
  WinBuf(WinBuf &&o) noexcept { take(o); }
  WinBuf &operator=(WinBuf &&o) noexcept {
    if (this != &o) {
      clear();
      take(o);
    }
    return *this;
  }
  void take(WinBuf &o) {
    ptrs.swap(o.ptrs);
    cur = o.cur;
    left = o.left;
    st = o.st;
    ordered = o.ordered;
    lasting = o.lasting;
    o.ptrs.clear();
    o.cur = nullptr;
    o.left = 0;
  }
  // long-lived buffers, released without a device synchronisation
  static WinBuf lasting_buf() {
    WinBuf b;
    b.ordered = true;
    b.lasting = true;
    return b;
  }
  void *raw(size_t bytes) {
    void *p = nullptr;
    std::shared_lock<std::shared_mutex> lk(capture_lock());
    if (ordered) keep_pool_memory();
    const cudaStream_t as = lasting ? release_stream() : st;
    if ((ordered ? cudaMallocAsync(&p, bytes, as) : cudaMalloc(&p, bytes)) != cudaSuccess) {
      cudaGetLastError();
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      fail(DMRG_ERR_OOM, "cudaMalloc(%zu) failed (%.1f GB of %.1f GB free)", bytes, fr / 1e9,
           tot / 1e9);
    }
    if (lasting) CK(cudaStreamSynchronize(as));   // usable on any stream from here
    ptrs.push_back(p);
    return p;
  }
  void *alloc(size_t bytes) {
    bytes = (std::max<size_t>(bytes, 8) + 255) & ~(size_t)255;
    if (bytes > kSmall) return raw(bytes);
    if (bytes > left) {
      cur = (char *)raw(kChunk);
      left = kChunk;
    }
    void *p = cur;
    cur += bytes;
    left -= bytes;
    return p;
  }
  void clear() {
    cur = nullptr;
    left = 0;
    if (ptrs.empty()) return;
    std::shared_lock<std::shared_mutex> lk(capture_lock());
    const cudaStream_t fs = lasting ? release_stream() : st;
    for (void *p : ptrs) {
      if (ordered)
        cudaFreeAsync(p, fs);
      else
        cudaFree(p);
    }
    ptrs.clear();
  }
  ~WinBuf() { clear(); }
};

// Device memory at a fixed virtual address whose physical memory can be
// given back and taken again (CUDA virtual memory management): the work
// descriptors that point into it stay valid while it is unmapped.  Used for
// the FP64 operator stacks and the FP64 intermediate of a window, which the
// split-precision path needs only while it builds its FP16 copies.
struct VmmFns {
  CUresult (*reserve)(CUdeviceptr *, size_t, size_t, CUdeviceptr, unsigned long long);
  CUresult (*addr_free)(CUdeviceptr, size_t);
  CUresult (*create)(CUmemGenericAllocationHandle *, size_t, const CUmemAllocationProp *,
                     unsigned long long);
  CUresult (*release)(CUmemGenericAllocationHandle);
  CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long);
  CUresult (*unmap)(CUdeviceptr, size_t);
  CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc *, size_t);
  CUresult (*granularity)(size_t *, const CUmemAllocationProp *, CUmemAllocationGranularity_flags);
};

const VmmFns &vmm() {
  static const VmmFns f = [] {
    VmmFns v;
    memset(&v, 0, sizeof v);
    auto get = [](const char *name, void **p) {
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion(name, p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess)
        *p = nullptr;
    };
    get("cuMemAddressReserve", (void **)&v.reserve);
    get("cuMemAddressFree", (void **)&v.addr_free);
    get("cuMemCreate", (void **)&v.create);
    get("cuMemRelease", (void **)&v.release);
    get("cuMemMap", (void **)&v.map);
    get("cuMemUnmap", (void **)&v.unmap);
    get("cuMemSetAccess", (void **)&v.set_access);
    get("cuMemGetAllocationGranularity", (void **)&v.granularity);
    return v;
  }();
  return f;
}

struct VmmBuf {
  CUdeviceptr va = 0;
  size_t size = 0;
  CUmemGenericAllocationHandle h = 0;
  bool mapped = false;
  int dev = 0;
  VmmBuf() = default;
  VmmBuf(const VmmBuf &) = delete;
  VmmBuf &operator=(const VmmBuf &) = delete;
  CUmemAllocationProp prop() const {
    CUmemAllocationProp p;
    memset(&p, 0, sizeof p);
    p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    p.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    p.location.id = dev;
    return p;
  }
  // address range only
  void reserve(size_t bytes) {
    free_all();
    const VmmFns &f = vmm();
    if (!f.reserve || !f.create || !f.map || !f.set_access || !f.granularity)
      fail(DMRG_ERR_CUDA, "CUDA virtual memory management entry points unavailable");
    CK(cudaGetDevice(&dev));
    const CUmemAllocationProp p = prop();
    size_t g = 0;
    if (f.granularity(&g, &p, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED) != CUDA_SUCCESS || g == 0)
      g = 2 << 20;
    size = (std::max<size_t>(bytes, 1) + g - 1) / g * g;
    if (f.reserve(&va, size, 0, 0, 0) != CUDA_SUCCESS) {
      va = 0;
      fail(DMRG_ERR_OOM, "cuMemAddressReserve(%zu) failed", size);
    }
  }
  // physical memory behind the range
  void map() {
    if (mapped || !va) return;
    const VmmFns &f = vmm();
    std::shared_lock<std::shared_mutex> lk(capture_lock());
    const CUmemAllocationProp p = prop();
    if (f.create(&h, size, &p, 0) != CUDA_SUCCESS) {
      h = 0;
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      fail(DMRG_ERR_OOM, "cuMemCreate(%zu) failed (%.1f GB of %.1f GB free)", size, fr / 1e9,
           tot / 1e9);
    }
    if (f.map(va, size, 0, h, 0) != CUDA_SUCCESS) {
      f.release(h);
      h = 0;
      fail(DMRG_ERR_OOM, "cuMemMap(%zu) failed", size);
    }
    CUmemAccessDesc a;
    memset(&a, 0, sizeof a);
    a.location = p.location;
    a.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    if (f.set_access(va, size, &a, 1) != CUDA_SUCCESS) {
      f.unmap(va, size);
      f.release(h);
      h = 0;
      fail(DMRG_ERR_CUDA, "cuMemSetAccess failed");
    }
    mapped = true;
  }
  // give the physical memory back (the caller has finished all work on it)
  void unmap() {
    if (!mapped) return;
    const VmmFns &f = vmm();
    std::shared_lock<std::shared_mutex> lk(capture_lock());
    f.unmap(va, size);
    f.release(h);
    h = 0;
    mapped = false;
  }
  void free_all() {
    unmap();
    if (va) vmm().addr_free(va, size);
    va = 0;
    size = 0;
  }
  double *ptr() const { return (double *)va; }
  ~VmmBuf() { free_all(); }
};

template <class T>
T *upload(WinBuf &wb, const std::vector<T> &v, cudaStream_t s) {
  T *d = (T *)wb.alloc(sizeof(T) * std::max<size_t>(v.size(), 1));
  if (!v.empty()) CK(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  return d;
}

struct TermF {
  Fac A, B;
  double coef;
  // spin-adapted terms [A^k (x) B^k]^0: twice the rank, adjoint factors
  int tk = -1;
  int adjA = 0, adjB = 0;
};

struct HClass {
  QN dA;
  int pB = 0;
  std::vector<TermF> terms;
  std::map<int, long long> a_off, b_off, t_off;   // keyed by input psi block
};

struct S1 {
  int ci, pi, po;   // H_eff class, input psi block, output psi block
};

struct PsiBlk {
  int a, b;          // sector indices in L. and .R
  long long off;
  int da, db;
};

// Host tables of the split path (psi split descriptors, tensor maps, K
// ranges, tile lists, partial sums) for given scratch pointers.
struct SplitTables {
  std::vector<F16Split> psi_split;
  std::vector<CUtensorMap> maps;
  std::vector<TSeg> segs;
  std::vector<TWork> w1, w2;      // stage-1 and stage-2 items, in launch order
  std::vector<PartialSum> psums;
};

// Split-precision plan for nv vectors applied together (dmrg_heff_apply_batch):
// its own per-apply scratch and device tables, built from the window's FP16
// operator copies and the autotuner's choices.
struct BatchPlan {
  int nv = 0;
  SplitTables tb;
  __half *Ph = nullptr, *Pl = nullptr, *Th = nullptr, *Tl = nullptr;
  float *ws = nullptr;
  PsiStat *pstat = nullptr;
  PsiDesc *pdesc = nullptr;
  int *next = nullptr;
  void *dsplit = nullptr, *dmaps = nullptr, *dseg = nullptr, *dw1 = nullptr, *dw2 = nullptr,
       *dps = nullptr;
  int psi_tiles = 1;
  std::map<std::pair<const void *, const void *>, cudaGraphExec_t> graphs;
};

// One launch of the grouped FP64 GEMM: descriptors of one tile size.
struct F64Launch {
  GemmDesc *d;
  int nd;
  long long tiles;
  int tm, tn;
};

struct Window {
  bool valid = false;
  int l = -1;
  BlockPart Ld, Rd;
  // window buffers are released without a device synchronisation: after the
  // last H_eff*psi enqueued through the public entry points (use_ev)
  WinBuf ldbuf = WinBuf::lasting_buf(), rdbuf = WinBuf::lasting_buf();
  cudaEvent_t use_ev = nullptr;
  bool used = false;
  std::vector<PsiBlk> psi;
  long long psi_len = 0;
  std::vector<int> a2psi;
  std::vector<HClass> hc;
  WinBuf buf = WinBuf::lasting_buf();   // descriptors, split-path copies and scratch
  // FP64 stacks and T at fixed addresses; T is backed on the first FP64
  // apply, and under an HBM budget A and B are given back once the split
  // path has its FP16 copies (and gathered again by the next FP64 apply)
  VmmBuf vA, vB, vT;
  std::vector<SCopy> stack_copies;   // the gather that fills A and B
  bool fp64_stacks = false;          // A and B hold the window's operators
  double *Astack = nullptr, *Bstack = nullptr, *T = nullptr;
  long long nA = 0, nB = 0, nT = 0;
  GemmSeg *s1 = nullptr, *s2 = nullptr;
  std::vector<F64Launch> f64_1, f64_2;   // the FP64 stages by tile size
  double flops = 0, flops1 = 0, flops2 = 0;
  double *diag = nullptr;
  std::vector<S1> s1info;                 // stage-1 regions (class, psi in, psi out)
  double *ws64 = nullptr;                 // FP64 split-K partial blocks of stage 2
  std::vector<PartialSum64> ps64;
  PartialSum64 *d_ps64 = nullptr;
  std::vector<GemmDesc> stage1, stage2;   // host copies (split-path planning)
  std::vector<GemmSeg> seg1, seg2;
  SplitPlan tf;          // split-precision plan (heff_split)
  bool tf_ready = false;
  bool tf_copies = false;            // FP16 (hi, lo) copies of the operator stacks exist
  int ksub = 0;                      // split-K range in use
  int cap1 = 128, order1 = 0;        // stage-1 schedule in use (tile-width cap, item order)
  void *tbl_ptr[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t tbl_cap[6] = {0, 0, 0, 0, 0, 0};
  std::map<std::pair<const void *, const void *>, cudaGraphExec_t> graphs;
  std::vector<long long> offA, ldA, offBp, bpad;   // split copies (halves)
  std::vector<float> sA, sB, rnA;                   // per entry: scales, largest A row norm
  long long gen = 0;                 // build counter of this window
  std::map<int, BatchPlan> batch;    // multi-vector split plans by vector count
};

}  // namespace

// spin-adapted formula of one target tensor: (factor, adjoint, factor,
// adjoint) -> coefficient
using SU2Terms = std::map<std::tuple<TKey, int, TKey, int>, double>;

struct dmrg_ctx {
  dmrg_config cfg;
  std::string err;
  bool spinful = false;
  bool su2 = false;   // U(1)xSU(2): sectors are multiplets, QN = highest-weight (N_up, N_dn)
  int N = 0, M = 0;
  QN target{0, 0};
  std::vector<double> h, W;
  bool ham = false;
  std::map<int, Iso> liso, riso;
  std::map<int, Iso> Lmap, Rmap;   // device isometries of the current blocks L_n, R_n
  std::vector<std::unique_ptr<BlockPart>> L;        // L[n], n sites
  std::map<int, std::unique_ptr<BlockPart>> R;      // R[n], sites n..N-1
  std::map<BlockPart *, std::unique_ptr<WinBuf>> partbuf;    // index tables, isometries
  std::map<BlockPart *, std::unique_ptr<WinBuf>> partdata;   // operator data (stageable)
  // staging of renormalized block operators under cfg.hbm_budget_bytes
  cudaStream_t stage_stream = nullptr;
  cudaEvent_t stage_ev = nullptr;
  std::vector<std::array<cudaEvent_t, 2>> h2d_events;   // timed host-to-device copies
  double st_h2d_bytes = 0, st_h2d_ms = 0, st_d2h_bytes = 0, st_peak = 0;
  long long st_offloads = 0, st_reloads = 0, st_releases = 0;
  Window win;
  SplitTables tables;    // host copy of the split-path tables of the window
  cudaStream_t stream = nullptr;
  cusolverDnHandle_t solver = nullptr;
  cusolverDnParams_t solver_params = nullptr;
  int precision = DMRG_FP64;
  double prof[7] = {0};
  double mem_max[6] = {0};   // dmrg_memory_stats
  // spin-adapted formulas already derived for this Hamiltonian, by (modes of
  // the first part, modes of the second, target tensor)
  std::map<std::pair<std::vector<int>, std::vector<int>>, std::map<TKey, SU2Terms>> derive_cache;
  long long derive_cache_terms = 0;
  // optional per-stage event timing of H_eff*psi
  bool timing = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double tacc[5] = {0, 0, 0, 0, 0};
  bool pending = false;
  // Davidson scratch
  WinBuf dav;
  long long dav_n = 0;
  double *V = nullptr, *AV = nullptr, *work = nullptr, *small = nullptr, *r = nullptr;
  double *rs = nullptr;   // thick-restart scratch (3 vectors)
  double *jd = nullptr;   // correction-equation scratch (4 vectors)
  // refinement of split solves: split-precision CG steps per correction,
  // on windows of at least this many algorithmic flops per apply
  int refine_steps = 20;
  double refine_min_flops = 1e8;
  // split contexts solve windows below this many flops per product with the
  // FP64 product alone (dmrg_set_split_min_flops)
  double split_min_flops = 0;
  uint64_t start_count = 0;
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;            // private stream for graph capture
  int ksub_choice = 0;                          // autotuned split-K range (0: not yet)
  int cap1_choice = 0, order1_choice = 0;       // autotuned stage-1 schedule (0: not yet)
  std::vector<std::array<double, 2>> tune_log;  // (candidate, ms per apply)
  // Bounded-wait status of the tcgen05 kernels for stream-ordered callers:
  // after each public split apply the device error word is copied (stream
  // ordered) into pinned host memory; the next call (or dmrg_sync) reads it
  // once the copy's event has completed.  [0] window path, [1] static path.
  int *hflag = nullptr;
  cudaEvent_t flag_ev[2] = {nullptr, nullptr};
  bool flag_pending[2] = {false, false};
  int sticky = DMRG_OK;                         // error owed to the next call
  std::string sticky_msg;
  int unconverged = 0;                          // window solves of the last sweep
  bool swept = false;                           // Lmap/Rmap hold the sweep's isometries
  int center_l = -1;                            // final window of the last sweep
  std::vector<double> center_psi;               // its psi (host copy)
};

namespace {

// ---------------------------------------------------------------------------
// Hamiltonian
// ---------------------------------------------------------------------------
void torus_bonds(int Lx, int Ly, bool nnn, std::vector<std::pair<int, int>> &out) {
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      int r = y * Lx + x;
      if (!nnn) {
        out.push_back({r, y * Lx + (x + 1) % Lx});
        out.push_back({r, ((y + 1) % Ly) * Lx + x});
      } else {
        out.push_back({r, ((y + 1) % Ly) * Lx + (x + 1) % Lx});
        out.push_back({r, ((y - 1 + Ly) % Ly) * Lx + (x + 1) % Lx});
      }
    }
}

// quarter transform along one index of a 4-index tensor: out[..a..] =
// sum_i in[..i..] U[i,a]
void quarter(const std::vector<double> &in, std::vector<double> &out, const double *U,
             int N, int axis) {
  out.assign(in.size(), 0.0);
  size_t st[4] = {(size_t)N * N * N, (size_t)N * N, (size_t)N, 1};
  for (size_t e = 0; e < in.size(); ++e) {
    double v = in[e];
    if (v == 0.0) continue;
    int i = (int)((e / st[axis]) % N);
    size_t base = e - (size_t)i * st[axis];
    const double *u = U + (size_t)i * N;
    for (int a = 0; a < N; ++a) out[base + (size_t)a * st[axis]] += v * u[a];
  }
}

// ---------------------------------------------------------------------------
// site operators (exact)
// ---------------------------------------------------------------------------
struct Mat4 {
  double m[16] = {0};
};
Mat4 mm(const Mat4 &a, const Mat4 &b) {
  Mat4 c;
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      double v = a.m[i * 4 + k];
      if (v == 0.0) continue;
      for (int j = 0; j < 4; ++j) c.m[i * 4 + j] += v * b.m[k * 4 + j];
    }
  return c;
}
Mat4 tr(const Mat4 &a) {
  Mat4 c;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) c.m[i * 4 + j] = a.m[j * 4 + i];
  return c;
}
void axpy(Mat4 &y, double a, const Mat4 &x) {
  for (int i = 0; i < 16; ++i) y.m[i] += a * x.m[i];
}

QN shift_c(const dmrg_ctx *C, int p) {
  if (!C->spinful) return {-1, 0};
  return (p % 2 == 0) ? QN{-1, 0} : QN{0, -1};
}

SiteOp mkop(const Mat4 &m, QN shift) {
  SiteOp o;
  o.shift = shift;
  o.parity = qparity(shift);
  memcpy(o.m, m.m, sizeof o.m);
  return o;
}

SitePart make_site(const dmrg_ctx *C, int i) {
  SitePart s;
  s.site = i;
  const int M = C->M;
  if (C->spinful) {
    s.modes = {2 * i, 2 * i + 1};
    s.d = 4;
    s.sq = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};
  } else {
    s.modes = {i};
    s.d = 2;
    s.sq = {{0, 0}, {1, 0}};
  }
  // local state index -> occupation bits (bit j = mode j of the site)
  std::vector<int> bits = C->spinful ? std::vector<int>{0, 2, 1, 3} : std::vector<int>{0, 1};
  std::vector<int> pos(4, -1);
  for (int k = 0; k < s.d; ++k) pos[bits[k]] = k;
  std::map<int, Mat4> cl;
  for (size_t j = 0; j < s.modes.size(); ++j) {
    Mat4 c;
    for (int k = 0; k < s.d; ++k) {
      int b = bits[k];
      if (!((b >> j) & 1)) continue;
      int below = __builtin_popcount(b & ((1 << j) - 1));
      c.m[pos[b & ~(1 << j)] * 4 + k] = (below & 1) ? -1.0 : 1.0;
    }
    cl[s.modes[j]] = c;
  }
  Mat4 I;
  for (int k = 0; k < s.d; ++k) I.m[k * 4 + k] = 1.0;
  s.I = mkop(I, {0, 0});
  auto hh = [&](int p, int q) { return C->h[(size_t)p * M + q]; };
  auto WW = [&](int p, int q, int r, int t) {
    return C->W[(((size_t)p * M + q) * M + r) * M + t];
  };
  Mat4 H;
  for (int p : s.modes)
    for (int q : s.modes) axpy(H, hh(p, q), mm(tr(cl[p]), cl[q]));
  for (int p : s.modes)
    for (int q : s.modes)
      for (int r : s.modes)
        for (int t : s.modes) {
          double w = WW(p, q, r, t);
          if (w != 0.0) axpy(H, w, mm(mm(tr(cl[p]), tr(cl[q])), mm(cl[r], cl[t])));
        }
  s.H = mkop(H, {0, 0});
  for (int p : s.modes) s.c[p] = mkop(cl[p], shift_c(C, p));
  for (size_t a = 0; a < s.modes.size(); ++a)
    for (size_t b = a + 1; b < s.modes.size(); ++b) {
      int p = s.modes[a], q = s.modes[b];
      s.cc[{p, q}] = mkop(mm(cl[p], cl[q]), qadd(shift_c(C, p), shift_c(C, q)));
    }
  for (int p : s.modes)
    for (int r : s.modes) s.cdc[{p, r}] = mkop(mm(tr(cl[p]), cl[r]), qsub(shift_c(C, r), shift_c(C, p)));
  std::vector<int> others;
  for (int y = 0; y < M; ++y)
    if (!has(s.modes, y)) others.push_back(y);
  for (int y : others) {
    Mat4 S;
    for (int q : s.modes) axpy(S, 0.5 * hh(y, q), cl[q]);
    for (int q : s.modes)
      for (int r : s.modes)
        for (int t : s.modes) {
          double w = WW(y, q, r, t);
          if (w != 0.0) axpy(S, 2.0 * w, mm(tr(cl[q]), mm(cl[r], cl[t])));
        }
    s.S[y] = mkop(S, shift_c(C, y));
  }
  for (size_t a = 0; a < others.size(); ++a)
    for (size_t b = a + 1; b < others.size(); ++b) {
      int x = others[a], z = others[b];
      Mat4 P;
      for (int p : s.modes)
        for (int q : s.modes) {
          double w = WW(x, z, p, q);
          if (w != 0.0) axpy(P, w, mm(cl[p], cl[q]));
        }
      s.P[{x, z}] = mkop(P, qadd(shift_c(C, x), shift_c(C, z)));
    }
  for (int x : others)
    for (int z : others) {
      Mat4 Qm;
      for (int p : s.modes)
        for (int q : s.modes) {
          double w = WW(x, p, z, q);
          if (w != 0.0) axpy(Qm, w, mm(tr(cl[p]), cl[q]));
        }
      s.Q[{x, z}] = mkop(Qm, qsub(shift_c(C, x), shift_c(C, z)));
    }
  return s;
}

// Spin-adapted site: the three multiplets {0} (N=0), {up, dn} (N=1, J=1/2;
// |1/2,+1/2> = |up>, |1/2,-1/2> = |dn>), {updn} (N=2, J=0), and the reduced
// matrices of every site tensor.  The tensor components are the couplings of
// the spin-orbital site operators (make_site, S_z basis {0, dn, up, updn})
// given in su2.h; the reduced element R(s' <- s) is read off at the highest
// weight of s', and every component must obey the Wigner-Eckart form.
SitePart make_site_su2(const dmrg_ctx *C, int i) {
  const SitePart z = make_site(C, i);
  SitePart s;
  s.site = i;
  s.modes = z.modes;
  s.d = 3;
  s.sq = {su2::label(0, 0), su2::label(1, 1), su2::label(2, 0)};
  s.tj = {0, 1, 0};
  auto szi = [](int mult, int tm) { return mult == 0 ? 0 : (mult == 2 ? 3 : (tm > 0 ? 2 : 1)); };
  auto so = [](int x, int tm) { return 2 * x + (tm > 0 ? 0 : 1); };
  auto sg = [](int tm) { return tm > 0 ? 1.0 : -1.0; };
  auto mat = [](const SiteOp &o) {
    Mat4 m;
    memcpy(m.m, o.m, sizeof m.m);
    return m;
  };
  auto get = [&](const std::map<int, SiteOp> &m, int k) {
    auto it = m.find(k);
    return it == m.end() ? Mat4() : mat(it->second);
  };
  auto getp = [&](const std::map<PairKey, SiteOp> &m, int a, int b) {
    auto it = m.find({a, b});
    return it == m.end() ? Mat4() : mat(it->second);
  };
  // P_ab with a, b spin-orbitals in any order (stored for a < b)
  auto Pso = [&](int a, int b) {
    if (a == b) return Mat4();
    if (a < b) return getp(z.P, a, b);
    Mat4 m = getp(z.P, b, a);
    for (double &x : m.m) x = -x;
    return m;
  };
  auto reduce = [&](const TKey &key, const std::map<int, Mat4> &comp) {
    SiteTen t;
    t.tk = key.tk;
    t.parity = key.parity();
    bool nz = false;
    for (int so_ = 0; so_ < 3; ++so_)
      for (int si = 0; si < 3; ++si) {
        const int tjo = s.tj[so_], tji = s.tj[si];
        double R = 0.0;
        for (int tmi = -tji; tmi <= tji; tmi += 2) {
          const int tq = tjo - tmi;
          auto it = comp.find(tq);
          if (it == comp.end()) continue;
          R += su2::cg(tji, tmi, key.tk, tq, tjo, tjo) * it->second.m[szi(so_, tjo) * 4 + szi(si, tmi)];
        }
        t.m[so_ * 4 + si] = R;
        nz |= R != 0.0;
        // Wigner-Eckart check of every component
        for (auto &kv : comp)
          for (int tmi = -tji; tmi <= tji; tmi += 2) {
            const int tmo = tmi + kv.first;
            if (std::abs(tmo) > tjo) continue;
            const double want = su2::cg(tji, tmi, key.tk, kv.first, tjo, tmo) * R;
            const double got = kv.second.m[szi(so_, tmo) * 4 + szi(si, tmi)];
            if (std::fabs(want - got) > 1e-12 * (1.0 + std::fabs(got)))
              fail(DMRG_ERR_STATE, "internal: site tensor (%d,%d,%d,%d) is not a spin tensor",
                   key.kind, key.i, key.j, key.tk);
          }
      }
    if (nz) s.ten[key] = t;
  };
  reduce({0, 0, 0, 0}, {{0, mat(z.H)}});
  {
    Mat4 cm = get(z.c, so(i, 1));
    for (double &x : cm.m) x = -x;
    reduce({1, i, 0, 1}, {{1, get(z.c, so(i, -1))}, {-1, cm}});
  }
  for (int y = 0; y < C->N; ++y) {
    if (y == i) continue;
    Mat4 sm = get(z.S, so(y, 1));
    for (double &x : sm.m) x = -x;
    reduce({2, y, 0, 1}, {{1, get(z.S, so(y, -1))}, {-1, sm}});
  }
  // A~^0_ii = [c~_i x c~_i]^0; B^k_ii = [c+_i x c~_i]^k
  for (int tk = 0; tk <= 2; tk += 2) {
    std::map<int, Mat4> ca, cb;
    for (int m1 = -1; m1 <= 1; m1 += 2)
      for (int m2 = -1; m2 <= 1; m2 += 2) {
        const int tq = m1 + m2;
        if (std::abs(tq) > tk) continue;
        const double w = su2::cg(1, m1, 1, m2, tk, tq);
        if (w == 0.0) continue;
        const Mat4 cc = mm(get(z.c, so(i, -m1)), get(z.c, so(i, -m2)));
        axpy(ca[tq], w * sg(m1) * sg(m2), cc);
        const Mat4 cd = mm(tr(get(z.c, so(i, m1))), get(z.c, so(i, -m2)));
        axpy(cb[tq], w * sg(m2), cd);
      }
    if (tk == 0) reduce({3, i, i, 0}, ca);
    reduce({4, i, i, tk}, cb);
  }
  // complementary pair tensors for every pair of spatial modes off the site
  for (int x = 0; x < C->N; ++x)
    for (int y = 0; y < C->N; ++y) {
      if (x == i || y == i) continue;
      for (int tk = 0; tk <= 2; tk += 2) {
        std::map<int, Mat4> cp, cq;
        for (int m1 = -1; m1 <= 1; m1 += 2)
          for (int m2 = -1; m2 <= 1; m2 += 2) {
            const int tq = m1 + m2;
            if (std::abs(tq) > tk) continue;
            const double w = su2::cg(1, m1, 1, m2, tk, tq);
            if (w == 0.0) continue;
            if (x <= y) axpy(cp[tq], w * sg(m1) * sg(m2), Pso(so(x, -m1), so(y, -m2)));
            axpy(cq[tq], w * sg(m2), getp(z.Q, so(x, -m2), so(y, m1)));
          }
        if (x <= y && !(x == y && tk == 2)) reduce({5, x, y, tk}, cp);
        reduce({6, x, y, tk}, cq);
      }
    }
  return s;
}

SitePart site_of(const dmrg_ctx *C, int i) { return C->su2 ? make_site_su2(C, i) : make_site(C, i); }

// The .R sector paired with L. sector qa in psi: the complement of qa in the
// target (spin-adapted, total S = 0: the same spin, the other particles).
QN partner(const dmrg_ctx *C, const QN &qa) {
  if (C->su2) return su2::label(su2::n_of(C->target) - su2::n_of(qa), su2::tj_of(qa));
  return qsub(C->target, qa);
}

// ---------------------------------------------------------------------------
// operator classes
// ---------------------------------------------------------------------------
struct OpSpec {
  int kind;   // 0 H, 1 c, 2 S, 3 cc, 4 cdc, 5 P, 6 Q
  int i, j;
  QN shift;
  int tk = -1;   // spin-adapted: twice the tensor rank (-1: spin-orbital operator)
  int g = 0;     // spin-adapted: this component's 2(J' - J)
};

QN spec_shift(const dmrg_ctx *C, int kind, int i, int j) {
  switch (kind) {
    case 0: return {0, 0};
    case 1: case 2: return shift_c(C, i);
    case 3: case 5: return qadd(shift_c(C, i), shift_c(C, j));
    case 4: return qsub(shift_c(C, j), shift_c(C, i));
    default: return qsub(shift_c(C, i), shift_c(C, j));
  }
}

std::vector<OpSpec> block_specs_su2(const dmrg_ctx *C, const std::vector<int> &so_modes);

// All operators a block holds ("both normal and complementary" policy).
std::vector<OpSpec> block_specs(const dmrg_ctx *C, const std::vector<int> &modes) {
  if (C->su2) return block_specs_su2(C, modes);
  std::vector<OpSpec> v;
  v.push_back({0, 0, 0, {0, 0}});
  for (int x : modes) v.push_back({1, x, 0, spec_shift(C, 1, x, 0)});
  std::vector<int> out;
  for (int y = 0; y < C->M; ++y)
    if (!has(modes, y)) out.push_back(y);
  for (int y : out) v.push_back({2, y, 0, spec_shift(C, 2, y, 0)});
  for (size_t a = 0; a < modes.size(); ++a)
    for (size_t b = a + 1; b < modes.size(); ++b)
      v.push_back({3, modes[a], modes[b], spec_shift(C, 3, modes[a], modes[b])});
  for (int p : modes)
    for (int r : modes) v.push_back({4, p, r, spec_shift(C, 4, p, r)});
  for (size_t a = 0; a < out.size(); ++a)
    for (size_t b = a + 1; b < out.size(); ++b)
      v.push_back({5, out[a], out[b], spec_shift(C, 5, out[a], out[b])});
  for (int x : out)
    for (int z : out) v.push_back({6, x, z, spec_shift(C, 6, x, z)});
  return v;
}

// Spin-adapted parts: every tensor of the part (kinds as OpSpec; spatial
// indices), each as its spin-change components.  Annihilation-type tensors
// (c~, S~) lower N by 1, the pair tensors A~ and P by 2; B, Q and H keep N.
std::vector<OpSpec> block_specs_su2(const dmrg_ctx *C, const std::vector<int> &so_modes) {
  std::vector<int> in;
  for (int p : so_modes)
    if (!has(in, p >> 1)) in.push_back(p >> 1);
  std::vector<int> out;
  for (int y = 0; y < C->N; ++y)
    if (!has(in, y)) out.push_back(y);
  std::vector<OpSpec> v;
  auto put = [&](int kind, int i, int j, int tk, int dn) {
    for (int g = -tk; g <= tk; g += 2) {
      OpSpec o;
      o.kind = kind;
      o.i = i;
      o.j = j;
      o.tk = tk;
      o.g = g;
      o.shift = su2::label(dn, g);
      v.push_back(o);
    }
  };
  put(0, 0, 0, 0, 0);
  for (int x : in) put(1, x, 0, 1, -1);
  for (int y : out) put(2, y, 0, 1, -1);
  for (size_t a = 0; a < in.size(); ++a)
    for (size_t b = a; b < in.size(); ++b)
      for (int tk = 0; tk <= (a == b ? 0 : 2); tk += 2) put(3, in[a], in[b], tk, -2);
  for (int p : in)
    for (int r : in)
      for (int tk = 0; tk <= 2; tk += 2) put(4, p, r, tk, 0);
  for (size_t a = 0; a < out.size(); ++a)
    for (size_t b = a; b < out.size(); ++b)
      for (int tk = 0; tk <= (a == b ? 0 : 2); tk += 2) put(5, out[a], out[b], tk, -2);
  for (int x : out)
    for (int z : out)
      for (int tk = 0; tk <= 2; tk += 2) put(6, x, z, tk, 0);
  return v;
}

void set_ref(BlockPart &B, const OpSpec &s, Ref r) {
  if (s.tk >= 0) {
    TRef &t = B.ten[TKey{s.kind, s.i, s.j, s.tk}];
    t.tk = s.tk;
    t.r[(s.g + s.tk) / 2] = r;
    return;
  }
  switch (s.kind) {
    case 0: B.H = r; break;
    case 1: B.c[s.i] = r; break;
    case 2: B.S[s.i] = r; break;
    case 3: B.cc[{s.i, s.j}] = r; break;
    case 4: B.cdc[{s.i, s.j}] = r; break;
    case 5: B.P[{s.i, s.j}] = r; break;
    default: B.Q[{s.i, s.j}] = r; break;
  }
}

// Assign operators to classes by QN shift and lay out the blocks.  Returns
// for every spec its Ref.  Device memory is allocated from wb.
std::vector<Ref> make_classes(BlockPart &B, const std::vector<OpSpec> &specs, WinBuf &wb,
                              cudaStream_t s, WinBuf *data = nullptr) {
  std::map<QN, int> byshift;
  std::vector<Ref> refs(specs.size());
  for (size_t k = 0; k < specs.size(); ++k) {
    auto it = byshift.find(specs[k].shift);
    int ci;
    if (it == byshift.end()) {
      ci = (int)B.cls.size();
      byshift[specs[k].shift] = ci;
      OpClass oc;
      oc.shift = specs[k].shift;
      oc.parity = qparity(oc.shift);
      B.cls.push_back(oc);
    } else {
      ci = it->second;
    }
    refs[k] = {ci, B.cls[ci].nops++};
  }
  const int ns = (int)B.basis.qn.size();
  for (auto &oc : B.cls) {
    oc.in2blk.assign(ns, -1);
    long long off = 0;
    for (int i = 0; i < ns; ++i) {
      int j = B.basis.find(qadd(B.basis.qn[i], oc.shift));
      if (j < 0) continue;
      oc.in2blk[i] = (int)oc.blk_in.size();
      oc.blk_in.push_back(i);
      oc.blk_out.push_back(j);
      oc.blk_off.push_back(off);
      off += (long long)B.basis.dim[j] * B.basis.dim[i];
    }
    oc.nnz = off;
    oc.d = (double *)(data ? data : &wb)->alloc(sizeof(double) * std::max<long long>(1, oc.nnz * oc.nops));
    oc.d_in2blk = upload(wb, oc.in2blk, s);
    oc.d_blk_out = upload(wb, oc.blk_out, s);
    oc.d_blk_off = upload(wb, oc.blk_off, s);
  }
  // drop empty classes' references: an op whose class has no block is zero
  for (size_t k = 0; k < specs.size(); ++k) {
    Ref r = refs[k];
    if (B.cls[r.cls].nnz == 0) r.cls = -1;
    set_ref(B, specs[k], r);
  }
  return refs;
}

bool allowed_q(const dmrg_ctx *C, const QN &q, int cap) {
  if (C->su2) {
    // the other `cap` sites hold N - N_q particles, whose spin (at most
    // min(n, 2 cap - n)/2, of the parity of n) must couple with J_q to S
    const int n_rest = su2::n_of(C->target) - su2::n_of(q);
    if (n_rest < 0 || n_rest > 2 * cap) return false;
    const int jmax2 = std::min(n_rest, 2 * cap - n_rest);
    const int tjq = su2::tj_of(q), tS = su2::tj_of(C->target);
    if (tjq < 0) return false;
    for (int t = std::abs(tjq - tS); t <= tjq + tS; t += 2)
      if (t <= jmax2 && ((t - n_rest) & 1) == 0) return true;
    return false;
  }
  for (int k = 0; k < (C->spinful ? 2 : 1); ++k) {
    int d = C->target[k] - q[k];
    if (d < 0 || d > cap) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------
// enlarged block: X x site (left) or site x X (right)
// ---------------------------------------------------------------------------
void enlarge_su2(dmrg_ctx *C, const BlockPart &X, const SitePart &st, bool site_first, int cap,
                 BlockPart &U, WinBuf &wb);

void enlarge(dmrg_ctx *C, const BlockPart &X, const SitePart &st, bool site_first, int cap,
             BlockPart &U, WinBuf &wb) {
  if (C->su2) {
    enlarge_su2(C, X, st, site_first, cap, U, wb);
    return;
  }
  cudaStream_t s = C->stream;
  // basis with pieces ordered by site state
  std::map<QN, std::vector<Piece>> pm;
  for (int k = 0; k < st.d; ++k)
    for (size_t j = 0; j < X.basis.qn.size(); ++j) {
      QN Q = qadd(X.basis.qn[j], st.sq[k]);
      if (!allowed_q(C, Q, cap)) continue;
      pm[Q].push_back({k, (int)j, 0, X.basis.dim[j]});
    }
  U.basis = Basis();
  U.pieces.clear();
  for (auto &kv : pm) {
    int off = 0;
    for (auto &p : kv.second) {
      p.off = off;
      off += p.dim;
    }
    U.basis.qn.push_back(kv.first);
    U.basis.dim.push_back(off);
    U.pieces.push_back(kv.second);
  }
  U.enlarged = true;
  U.site_first = site_first;
  U.modes.clear();
  if (site_first) {
    U.modes = st.modes;
    U.modes.insert(U.modes.end(), X.modes.begin(), X.modes.end());
  } else {
    U.modes = X.modes;
    U.modes.insert(U.modes.end(), st.modes.begin(), st.modes.end());
  }
  std::vector<OpSpec> specs = block_specs(C, U.modes);
  make_classes(U, specs, wb, s);

  Side sx, ss;
  sx.b = &X;
  ss.s = &st;
  const Side &F = site_first ? ss : sx;
  const Side &G = site_first ? sx : ss;
  const bool block_first = !site_first;

  // per class, per op: terms
  std::vector<std::vector<std::vector<GTerm>>> terms(U.cls.size());
  for (size_t ci = 0; ci < U.cls.size(); ++ci) terms[ci].resize(U.cls[ci].nops);
  // The terms of one enlarged operator are accumulated per source operator
  // of X (class, index, transposed) or X's identity.  A dense slot table over
  // X's operators finds a term in O(1); the terms are emitted in key order.
  std::vector<long long> cls_base(X.cls.size() + 1, 0);
  for (size_t c = 0; c < X.cls.size(); ++c) cls_base[c + 1] = cls_base[c] + X.cls[c].nops;
  std::vector<int> slot(1 + 2 * (size_t)cls_base.back(), -1);
  std::vector<GTerm> accv;
  std::vector<std::pair<std::tuple<int, int, int>, int>> touched;   // (key, slot table index)
  for (size_t k = 0; k < specs.size(); ++k) {
    const OpSpec &sp = specs[k];
    Ref r;
    switch (sp.kind) {
      case 0: r = U.H; break;
      case 1: r = U.c[sp.i]; break;
      case 2: r = U.S[sp.i]; break;
      case 3: r = U.cc[{sp.i, sp.j}]; break;
      case 4: r = U.cdc[{sp.i, sp.j}]; break;
      case 5: r = U.P[{sp.i, sp.j}]; break;
      default: r = U.Q[{sp.i, sp.j}]; break;
    }
    if (r.cls < 0) continue;
    accv.clear();
    touched.clear();
    AddFn add = [&](const Fac &A, const Fac &B, double coef) {
      if (A.kind == 0 || B.kind == 0) return;
      const Fac &Xf = block_first ? A : B;
      const Fac &Sf = block_first ? B : A;
      if (Sf.kind != 3 || Xf.kind == 3) fail(DMRG_ERR_STATE, "internal: bad enlarged term");
      QN tot = qadd(A.shift, B.shift);
      if (tot != sp.shift) fail(DMRG_ERR_STATE, "internal: shift mismatch in enlarged op");
      double c = coef * A.scale * B.scale;
      std::tuple<int, int, int> key = Xf.kind == 2 ? std::make_tuple(-1, 0, 0)
                                                   : std::make_tuple(Xf.ref.cls, Xf.ref.idx, Xf.trans);
      size_t si = 0;
      if (Xf.kind != 2) {
        if (Xf.ref.cls < 0 || Xf.ref.cls >= (int)X.cls.size() || Xf.ref.idx < 0 ||
            Xf.ref.idx >= X.cls[Xf.ref.cls].nops || (Xf.trans != 0 && Xf.trans != 1))
          fail(DMRG_ERR_STATE, "internal: bad source operator in enlarged term");
        si = 1 + 2 * (size_t)(cls_base[Xf.ref.cls] + Xf.ref.idx) + (size_t)Xf.trans;
      }
      if (slot[si] < 0) {
        GTerm t;
        memset(&t, 0, sizeof t);
        t.src = std::get<0>(key);
        t.idx = std::get<1>(key);
        t.trans = std::get<2>(key);
        t.p2 = B.parity;
        slot[si] = (int)accv.size();
        accv.push_back(t);
        touched.push_back({key, (int)si});
      }
      GTerm &g = accv[slot[si]];
      for (int e = 0; e < 16; ++e) g.m[e] += c * Sf.so.m[e];
    };
    switch (sp.kind) {
      case 0: formula_H(F, G, add, true); break;
      case 1: formula_c(F, G, sp.i, add); break;
      case 2: formula_S(F, G, sp.i, add); break;
      case 3: formula_cc(F, G, sp.i, sp.j, add); break;
      case 4: formula_cdc(F, G, sp.i, sp.j, add); break;
      case 5: formula_P(F, G, sp.i, sp.j, C->W.data(), C->M, add); break;
      default: formula_Q(F, G, sp.i, sp.j, C->W.data(), C->M, add); break;
    }
    auto &dst = terms[r.cls][r.idx];
    std::sort(touched.begin(), touched.end());
    for (auto &kv : touched) {
      const GTerm &g = accv[slot[kv.second]];
      slot[kv.second] = -1;
      bool nz = false;
      for (int e = 0; e < 16; ++e) nz |= g.m[e] != 0.0;
      if (nz) dst.push_back(g);
    }
  }
  // flatten terms, CSR per class
  std::vector<GTerm> all;
  std::vector<std::vector<int>> ptr(U.cls.size());
  for (size_t ci = 0; ci < U.cls.size(); ++ci) {
    ptr[ci].push_back((int)all.size());
    for (auto &tl : terms[ci]) {
      all.insert(all.end(), tl.begin(), tl.end());
      ptr[ci].push_back((int)all.size());
    }
  }
  WinBuf tmp(s);   // work lists, released once the gather has run
  GTerm *d_terms = upload(tmp, all, s);
  std::vector<int *> d_ptr(U.cls.size());
  for (size_t ci = 0; ci < U.cls.size(); ++ci) d_ptr[ci] = upload(tmp, ptr[ci], s);
  std::vector<GSrc> srcs;
  for (auto &oc : X.cls) srcs.push_back({oc.d, oc.nnz, oc.d_in2blk, oc.d_blk_out, oc.d_blk_off});
  GSrc *d_srcs = upload(tmp, srcs, s);
  std::vector<GSub> subs;
  int max_ops = 0;
  for (size_t ci = 0; ci < U.cls.size(); ++ci) {
    const OpClass &oc = U.cls[ci];
    if (oc.nnz == 0) continue;
    max_ops = std::max(max_ops, oc.nops);
    for (size_t b = 0; b < oc.blk_in.size(); ++b) {
      int qi = oc.blk_in[b], qo = oc.blk_out[b];
      int ld = U.basis.dim[qi];
      for (const Piece &po : U.pieces[qo])
        for (const Piece &pi : U.pieces[qi]) {
          GSub g;
          memset(&g, 0, sizeof g);
          g.out = oc.d;
          g.nnz_out = oc.nnz;
          g.out_off = oc.blk_off[b] + (long long)po.off * ld + pi.off;
          g.out_ld = ld;
          g.rows = po.dim;
          g.cols = pi.dim;
          g.so = po.site_state;
          g.si = pi.site_state;
          g.a_out = po.blk_sector;
          g.a_in = pi.blk_sector;
          g.n_in = site_first ? qnum(st.sq[pi.site_state]) : qnum(X.basis.qn[pi.blk_sector]);
          g.nops = oc.nops;
          g.term_ptr = d_ptr[ci];
          subs.push_back(g);
        }
    }
  }
  GSub *d_subs = upload(tmp, subs, s);
  CK(launch_gather(d_subs, (int)subs.size(), max_ops, d_terms, d_srcs, 4, s));
  CK(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// spin-adapted formulas
// ---------------------------------------------------------------------------
// Terms [X (x) Y]^k of one tensor T (rank k) of the part F u G, keyed by
// (tensor of F, adjoint?, tensor of G, adjoint?).  The highest component
// [T]_k is a fixed combination of spin-orbital operators (su2.h); each is
// expanded by its spin-orbital formula (formulas.h), every product of tensor
// components a X_qa (x) b Y_qb is projected on the coupled forms,
//   X_qa Y_qb = sum_kappa <ka qa kb qb | kappa k> [X (x) Y]^kappa_k + ...,
// and the kappa = k parts are summed.  The kappa != k parts must cancel
// (T is a rank-k tensor): checked.

SU2Terms derive_su2(const dmrg_ctx *C, const SideS &F, const SideS &G, const TKey &T) {
  const int tk = T.tk, tq = T.tk;
  SU2Terms alpha;
  std::map<std::tuple<TKey, int, TKey, int, int>, double> other;
  double d = 1.0, scale = 0.0;
  auto add = [&](const SFac &A, const SFac &B, double coef) {
    for (const TComp &a : A.c)
      for (const TComp &b : B.c) {
        if (a.tq + b.tq != tq) fail(DMRG_ERR_STATE, "internal: spin projection of a product");
        const int ka = a.key.kind < 0 ? 0 : a.key.tk, kb = b.key.kind < 0 ? 0 : b.key.tk;
        const int aa = a.key.kind < 0 ? 0 : a.adj, ba = b.key.kind < 0 ? 0 : b.adj;
        const double base = d * coef * a.a * b.a;
        scale += std::fabs(base);
        for (int kap = std::abs(ka - kb); kap <= ka + kb; kap += 2) {
          const double w = su2::cg(ka, a.tq, kb, b.tq, kap, tq);
          if (w == 0.0) continue;
          if (kap == tk) alpha[std::make_tuple(a.key, aa, b.key, ba)] += base * w;
          else other[std::make_tuple(a.key, aa, b.key, ba, kap)] += base * w;
        }
      }
  };
  const double *W = C->W.data();
  const int M = C->M;
  auto so = [](int x, int tm) { return 2 * x + (tm > 0 ? 0 : 1); };
  auto sg = [](int tm) { return tm > 0 ? 1.0 : -1.0; };
  switch (T.kind) {
    case 0: formula_H(F, G, add, true); break;
    case 1: formula_c(F, G, so(T.i, -1), add); break;   // [c~]_{+1/2} = c_dn
    case 2: formula_S(F, G, so(T.i, -1), add); break;   // [S~]_{+1/2} = S_dn
    default:
      for (int m1 = -1; m1 <= 1; m1 += 2) {
        const int m2 = tq - m1;
        if (std::abs(m2) != 1) continue;
        const double w = su2::cg(1, m1, 1, m2, tk, tq);
        if (w == 0.0) continue;
        if (T.kind == 3) {          // [A~]_q = sum <..> s s c_{i,-m1} c_{j,-m2}
          const int a = so(T.i, -m1), b = so(T.j, -m2);
          if (a == b) continue;
          d = w * sg(m1) * sg(m2);
          if (a < b) {
            formula_cc(F, G, a, b, add);
          } else {
            d = -d;
            formula_cc(F, G, b, a, add);
          }
        } else if (T.kind == 4) {   // [B]_q = sum <..> s c+_{i,m1} c_{j,-m2}
          d = w * sg(m2);
          formula_cdc(F, G, so(T.i, m1), so(T.j, -m2), add);
        } else if (T.kind == 5) {   // [P]_q = sum <..> s s P_{(i,-m1),(j,-m2)}
          const int a = so(T.i, -m1), b = so(T.j, -m2);
          if (a == b) continue;
          d = w * sg(m1) * sg(m2);
          formula_P(F, G, a, b, W, M, add);
        } else {                    // [Q]_q = sum <..> s Q_{(i,-m2),(j,m1)}
          d = w * sg(m2);
          formula_Q(F, G, so(T.i, -m2), so(T.j, m1), W, M, add);
        }
      }
  }
  double omax = 0.0;
  for (auto &kv : other) omax = std::max(omax, std::fabs(kv.second));
  if (omax > 1e-10 * std::max(scale, 1e-300))
    fail(DMRG_ERR_STATE, "internal: tensor (%d,%d,%d,%d) has a rank-%d part %.3g", T.kind, T.i, T.j,
         T.tk, -1, omax);
  for (auto it = alpha.begin(); it != alpha.end();)
    it = std::fabs(it->second) <= 1e-14 * scale ? alpha.erase(it) : std::next(it);
  return alpha;
}

SideS side_of(const SitePart &st) {
  SideS sd;
  sd.so_modes = st.modes;
  sd.has = [&st](const TKey &k) { return st.ten.count(k) > 0; };
  return sd;
}

// A block's tensors as the formulas see them when derived once for every
// block of the same modes: a tensor counts if the block defines it, even if
// all its classes are empty in the current basis (those terms are zero and
// the users of the derived terms skip factors without data).
SideS side_of_defined(const BlockPart &B) {
  SideS sd;
  sd.so_modes = B.modes;
  sd.has = [&B](const TKey &k) { return B.ten.count(k) > 0; };
  return sd;
}

// derive_su2 memoised per context: the terms depend only on the parts' modes,
// the target tensor and the Hamiltonian (cleared when it changes).  A sweep
// meets every enlargement (block x site) again in its other pass, and every
// later sweep meets them all again.  derive_table returns the table of one
// pair of parts (looked up once per enlargement), derive_in one tensor's terms.
// f(0..n-1) on up to 8 host threads (items claimed 16 at a time); the first
// exception of any thread is rethrown here.  For independent host work only.
template <class Fn>
void parallel_for(size_t n, Fn &&f) {
  const size_t hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(std::min<size_t>(hw, 8), (n + 63) / 64);
  if (nt <= 1) {
    for (size_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<size_t> next{0};
  std::exception_ptr err;
  std::mutex em;
  auto run = [&]() {
    try {
      for (;;) {
        const size_t i = next.fetch_add(16);
        if (i >= n) break;
        for (size_t j = i; j < std::min(n, i + 16); ++j) f(j);
      }
    } catch (...) {
      std::lock_guard<std::mutex> lk(em);
      if (!err) err = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  for (size_t t = 1; t < nt; ++t) th.emplace_back(run);
  run();
  for (auto &t : th) t.join();
  if (err) std::rethrow_exception(err);
}

std::map<TKey, SU2Terms> &derive_table(dmrg_ctx *C, const SideS &F, const SideS &G) {
  // bounded host memory: start over past 2^24 cached terms
  if (C->derive_cache_terms > (1LL << 24)) {
    C->derive_cache.clear();
    C->derive_cache_terms = 0;
  }
  return C->derive_cache[std::make_pair(F.so_modes, G.so_modes)];
}

const SU2Terms &derive_in(dmrg_ctx *C, std::map<TKey, SU2Terms> &tab, const SideS &F,
                          const SideS &G, const TKey &T) {
  auto it = tab.find(T);
  if (it != tab.end()) return it->second;
  SU2Terms al = derive_su2(C, F, G, T);
  C->derive_cache_terms += (long long)al.size() + 1;
  return tab.emplace(T, std::move(al)).first->second;
}

// coefficient-table slot of a term type (2 k of the block factor, of the site
// factor, of the target; block factor adjoint)
inline int ctype_of(int tkX, int tkS, int tk, int adj) { return ((tkX * 3 + tkS) * 3 + tk) * 2 + adj; }
constexpr int kCtypes = 54;

// enlarged spin-adapted block: X x site (left) or site x X (right)
void enlarge_su2(dmrg_ctx *C, const BlockPart &X, const SitePart &st, bool site_first, int cap,
                 BlockPart &U, WinBuf &wb) {
  cudaStream_t s = C->stream;
  std::map<QN, std::vector<Piece>> pm;
  for (int k = 0; k < st.d; ++k)
    for (size_t j = 0; j < X.basis.qn.size(); ++j) {
      const QN &qb = X.basis.qn[j];
      const int n = su2::n_of(qb) + su2::n_of(st.sq[k]);
      const int t1 = su2::tj_of(qb), t2 = st.tj[k];
      for (int tj = std::abs(t1 - t2); tj <= t1 + t2; tj += 2) {
        const QN Q = su2::label(n, tj);
        if (!allowed_q(C, Q, cap)) continue;
        pm[Q].push_back({k, (int)j, 0, X.basis.dim[j]});
      }
    }
  U.basis = Basis();
  U.pieces.clear();
  for (auto &kv : pm) {
    int off = 0;
    for (auto &p : kv.second) {
      p.off = off;
      off += p.dim;
    }
    U.basis.qn.push_back(kv.first);
    U.basis.dim.push_back(off);
    U.pieces.push_back(kv.second);
  }
  U.enlarged = true;
  U.site_first = site_first;
  U.modes.clear();
  if (site_first) {
    U.modes = st.modes;
    U.modes.insert(U.modes.end(), X.modes.begin(), X.modes.end());
  } else {
    U.modes = X.modes;
    U.modes.insert(U.modes.end(), st.modes.begin(), st.modes.end());
  }
  std::vector<OpSpec> specs = block_specs(C, U.modes);
  make_classes(U, specs, wb, s);

  const SideS sx = side_of_defined(X), ss = side_of(st);
  const SideS &F = site_first ? ss : sx;
  const SideS &G = site_first ? sx : ss;
  std::map<TKey, SU2Terms> &dtab = derive_table(C, F, G);
  // per class, per op: terms
  std::vector<std::vector<std::vector<GTerm>>> terms(U.cls.size());
  for (size_t ci = 0; ci < U.cls.size(); ++ci) terms[ci].resize(U.cls[ci].nops);
  // the tensors with data; formulas not derived yet for these parts are
  // derived on several host threads and cached in order, then every tensor's
  // terms are built on several threads (each writes only its own slots)
  std::vector<std::pair<const TKey *, const TRef *>> work;
  for (auto &tv : U.ten) {
    bool any = false;
    for (const Ref &r : tv.second.r) any |= r.cls >= 0;
    if (any) work.push_back({&tv.first, &tv.second});
  }
  std::vector<const SU2Terms *> alp(work.size(), nullptr);
  std::vector<size_t> miss;
  for (size_t i = 0; i < work.size(); ++i) {
    auto it = dtab.find(*work[i].first);
    if (it != dtab.end()) alp[i] = &it->second;
    else miss.push_back(i);
  }
  std::vector<SU2Terms> fresh(miss.size());
  parallel_for(miss.size(), [&](size_t k) { fresh[k] = derive_su2(C, F, G, *work[miss[k]].first); });
  for (size_t k = 0; k < miss.size(); ++k) {
    C->derive_cache_terms += (long long)fresh[k].size() + 1;
    alp[miss[k]] = &dtab.emplace(*work[miss[k]].first, std::move(fresh[k])).first->second;
  }
  parallel_for(work.size(), [&](size_t wi) {
    const TKey &T = *work[wi].first;
    const TRef &tref = *work[wi].second;
    const SU2Terms &al = *alp[wi];
    // merged by (source class, index, transpose, coefficient type); a tensor
    // has a few such terms, so a linear search is the cheapest map
    std::vector<GTerm> acc;
    for (auto &kv : al) {
      const TKey &kf = std::get<0>(kv.first), &kg = std::get<2>(kv.first);
      const int af = std::get<1>(kv.first), ag = std::get<3>(kv.first);
      const TKey &kx = site_first ? kg : kf, &ks = site_first ? kf : kg;
      const int ax = site_first ? ag : af, as = site_first ? af : ag;
      const int tkX = kx.kind < 0 ? 0 : kx.tk, tkS = ks.kind < 0 ? 0 : ks.tk;
      // site factor (reduced, adjoint if asked), with the term's coefficient
      double m[16] = {0};
      if (ks.kind < 0) {
        for (int k = 0; k < st.d; ++k) m[k * 4 + k] = 1.0;
      } else {
        const SiteTen &t = st.ten.at(ks);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            m[a * 4 + b] = as ? su2::adjoint_factor(st.tj[b], st.tj[a], tkS) * t.m[b * 4 + a]
                              : t.m[a * 4 + b];
      }
      const int p2 = site_first ? kx.parity() : (ks.kind < 0 ? 0 : ks.parity());
      const int ct = ctype_of(tkX, tkS, T.tk, kx.kind < 0 ? 0 : ax);
      auto put = [&](int src, int idx, int trans) {
        GTerm *gt = nullptr;
        for (GTerm &x : acc)
          if (x.src == src && x.idx == idx && x.trans == trans && x.ctype == ct) {
            gt = &x;
            break;
          }
        if (!gt) {
          GTerm g;
          memset(&g, 0, sizeof g);
          g.src = src;
          g.idx = idx;
          g.trans = trans;
          g.p2 = p2;
          g.ctype = ct;
          acc.push_back(g);
          gt = &acc.back();
        }
        for (int e = 0; e < 16; ++e) gt->m[e] += kv.second * m[e];
      };
      if (kx.kind < 0) {
        put(-1, 0, 0);
      } else {
        const TRef &tr = X.ten.at(kx);
        for (const Ref &r : tr.r)
          if (r.cls >= 0) put(r.cls, r.idx, ax);
      }
    }
    // (source class, index, transpose, coefficient type) order, as a map would give
    std::sort(acc.begin(), acc.end(), [](const GTerm &a, const GTerm &b) {
      return std::make_tuple(a.src, a.idx, a.trans, a.ctype) <
             std::make_tuple(b.src, b.idx, b.trans, b.ctype);
    });
    for (const Ref &r : tref.r)
      if (r.cls >= 0) terms[r.cls][r.idx] = acc;
  });
  // flatten terms, CSR per class
  std::vector<GTerm> all;
  std::vector<std::vector<int>> ptr(U.cls.size());
  for (size_t ci = 0; ci < U.cls.size(); ++ci) {
    ptr[ci].push_back((int)all.size());
    for (auto &tl : terms[ci]) {
      all.insert(all.end(), tl.begin(), tl.end());
      ptr[ci].push_back((int)all.size());
    }
  }
  WinBuf tmp(s);   // work lists, released once the gather has run
  GTerm *d_terms = upload(tmp, all, s);
  std::vector<int *> d_ptr(U.cls.size());
  for (size_t ci = 0; ci < U.cls.size(); ++ci) d_ptr[ci] = upload(tmp, ptr[ci], s);
  std::vector<GSrc> srcs;
  for (auto &oc : X.cls) srcs.push_back({oc.d, oc.nnz, oc.d_in2blk, oc.d_blk_out, oc.d_blk_off});
  GSrc *d_srcs = upload(tmp, srcs, s);
  std::vector<GSub> subs;
  std::vector<double> ctab;
  int max_ops = 0;
  for (size_t ci = 0; ci < U.cls.size(); ++ci) {
    const OpClass &oc = U.cls[ci];
    if (oc.nnz == 0) continue;
    max_ops = std::max(max_ops, oc.nops);
    for (size_t b = 0; b < oc.blk_in.size(); ++b) {
      const int qi = oc.blk_in[b], qo = oc.blk_out[b];
      const int ld = U.basis.dim[qi];
      const int tJ = su2::tj_of(U.basis.qn[qi]), tJp = su2::tj_of(U.basis.qn[qo]);
      for (const Piece &po : U.pieces[qo])
        for (const Piece &pi : U.pieces[qi]) {
          GSub g;
          memset(&g, 0, sizeof g);
          g.out = oc.d;
          g.nnz_out = oc.nnz;
          g.out_off = oc.blk_off[b] + (long long)po.off * ld + pi.off;
          g.out_ld = ld;
          g.rows = po.dim;
          g.cols = pi.dim;
          g.so = po.site_state;
          g.si = pi.site_state;
          g.a_out = po.blk_sector;
          g.a_in = pi.blk_sector;
          g.n_in = site_first ? qnum(st.sq[pi.site_state]) : qnum(X.basis.qn[pi.blk_sector]);
          g.nops = oc.nops;
          g.term_ptr = d_ptr[ci];
          // recoupling coefficient of every term type for these spins
          const int tjx = su2::tj_of(X.basis.qn[pi.blk_sector]);
          const int tjxp = su2::tj_of(X.basis.qn[po.blk_sector]);
          const int tjs = st.tj[pi.site_state], tjsp = st.tj[po.site_state];
          const size_t base = ctab.size();
          ctab.resize(base + kCtypes, 0.0);
          for (int tkX = 0; tkX <= 2; ++tkX)
            for (int tkS = 0; tkS <= 2; ++tkS)
              for (int tk = 0; tk <= 2; ++tk) {
                if (((tkX + tkS + tk) & 1) || tk > tkX + tkS || tk < std::abs(tkX - tkS)) continue;
                const double K = site_first
                    ? su2::coupling(tjs, tjx, tJ, tjsp, tjxp, tJp, tkS, tkX, tk)
                    : su2::coupling(tjx, tjs, tJ, tjxp, tjsp, tJp, tkX, tkS, tk);
                ctab[base + ctype_of(tkX, tkS, tk, 0)] = K;
                ctab[base + ctype_of(tkX, tkS, tk, 1)] = K * su2::adjoint_factor(tjx, tjxp, tkX);
              }
          g.ctab = reinterpret_cast<const double *>(base);   // offset, made a pointer below
          subs.push_back(g);
        }
    }
  }
  double *d_ctab = upload(tmp, ctab, s);
  for (GSub &g : subs) g.ctab = d_ctab + reinterpret_cast<size_t>(g.ctab);
  GSub *d_subs = upload(tmp, subs, s);
  CK(launch_gather(d_subs, (int)subs.size(), max_ops, d_terms, d_srcs, 4, s));
  CK(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// renormalization: B = T^T U T  (T = isometry on U's sectors)
// ---------------------------------------------------------------------------
WinBuf &data_of(dmrg_ctx *C, BlockPart *B);

// Grouped FP64 GEMM with the tile shape chosen per descriptor: an operator
// block of a few rows or columns would leave most of a 64 x 64 tile idle.  A
// batch of problems that share one operand (the isometry in a
// renormalization) can be folded into the rows or columns of one problem.
// Each descriptor takes the shape and folding that issue the fewest
// multiply-adds, with a small penalty on small tiles; one launch per shape.
// Descriptors' tile fields are recomputed here.
const int kGemmShapes[5][2] = {{16, 16}, {32, 32}, {64, 64}, {64, 16}, {16, 64}};

// Tile shape (index into kGemmShapes) and folding (0 none, 1 rows, 2 columns)
// that issue the fewest multiply-adds for `batch` problems of M x N, folding
// into rows allowed if f1, into columns if f2; a small penalty per tile edge
// favours larger tiles.
void gemm_tile_choice(int M, int N, int batch, bool f1, bool f2, bool square_only, int *shape,
                      int *fold) {
  double bc = -1;
  *shape = 2;
  *fold = 0;
  for (int q = 0; q < (square_only ? 3 : 5); ++q)
    for (int f = 0; f < (square_only ? 1 : 3); ++f) {
      if ((f == 1 && !f1) || (f == 2 && !f2)) continue;
      const int tm = kGemmShapes[q][0], tn = kGemmShapes[q][1];
      const double Mt = f == 1 ? (double)batch * M : M;
      const double Nt = f == 2 ? (double)batch * N : N;
      const double tiles = std::ceil(Mt / tm) * std::ceil(Nt / tn) * (f ? 1 : batch);
      const double c = tiles * tm * tn * (1.0 + 4.0 / tm + 4.0 / tn);
      if (bc < 0 || c < bc) {
        bc = c;
        *shape = q;
        *fold = f;
      }
    }
}

std::vector<F64Launch> plan_gemm_f64(std::vector<GemmDesc> d, const std::vector<GemmSeg> &g,
                                     WinBuf &wb, cudaStream_t s, bool square_only = false) {
  std::vector<F64Launch> out;
  if (d.empty()) return out;
  std::vector<GemmDesc> bucket[5];
  for (GemmDesc &x : d) {
    bool f1 = x.batch > 1, f2 = x.batch > 1;
    for (int q = 0; q < x.nseg; ++q) {
      const GemmSeg &sg = g[x.seg0 + q];
      f1 = f1 && sg.B != nullptr && sg.b_bs == 0;
      f2 = f2 && sg.a_bs == 0;
    }
    int best = 2, bfold = 0;
    gemm_tile_choice(x.M, x.N, x.batch, f1, f2, square_only, &best, &bfold);
    x.fold = bfold;
    bucket[best].push_back(x);
  }
  for (int q = 0; q < 5; ++q) {
    std::vector<GemmDesc> &b = bucket[q];
    if (b.empty()) continue;
    const int tm = kGemmShapes[q][0], tn = kGemmShapes[q][1];
    long long t = 0;
    for (GemmDesc &x : b) {
      const long long Mt = x.fold == 1 ? (long long)x.batch * x.M : x.M;
      const long long Nt = x.fold == 2 ? (long long)x.batch * x.N : x.N;
      x.tiles_m = (int)((Mt + tm - 1) / tm);
      x.tiles_n = (int)((Nt + tn - 1) / tn);
      x.tile0 = t;
      t += (long long)x.tiles_m * x.tiles_n * (x.fold ? 1 : x.batch);
    }
    out.push_back({upload(wb, b, s), (int)b.size(), t, tm, tn});
  }
  return out;
}

void run_gemm_f64(const std::vector<F64Launch> &plan, const GemmSeg *dseg, cudaStream_t s,
                  const double *bindB = nullptr, double *bindC = nullptr) {
  for (const F64Launch &l : plan)
    CK(launch_gemm_f64(l.d, l.nd, dseg, l.tiles, s, bindB, bindC, l.tm, l.tn));
}

void gemm_f64_grouped(const std::vector<GemmDesc> &d, const std::vector<GemmSeg> &g, WinBuf &wb,
                      cudaStream_t s) {
  if (d.empty()) return;
  const GemmSeg *dg = upload(wb, g, s);
  run_gemm_f64(plan_gemm_f64(d, g, wb, s), dg, s);
}

// Temporaries of one renormalization chunk: 2^28 doubles (2 GB).
constexpr long long kRenTmpDoubles = 1LL << 28;

void renormalize(dmrg_ctx *C, const BlockPart &U, const Iso &T, BlockPart &B, WinBuf &wb) {
  cudaStream_t s = C->stream;
  B.basis = Basis();
  std::vector<int> u_of(T.qn.size());
  for (size_t k = 0; k < T.qn.size(); ++k) {
    int j = U.basis.find(T.qn[k]);
    if (j < 0 || U.basis.dim[j] != T.rows[k])
      fail(DMRG_ERR_ARG, "isometry sector %zu (QN %d,%d): rows %d do not match enlarged dim %d",
           k, T.qn[k][0], T.qn[k][1], T.rows[k], j < 0 ? 0 : U.basis.dim[j]);
    u_of[k] = j;
    B.basis.qn.push_back(T.qn[k]);
    B.basis.dim.push_back(T.cols[k]);
  }
  B.modes = U.modes;
  B.enlarged = false;
  // same operators, same shifts
  std::vector<OpSpec> specs = block_specs(C, B.modes);
  make_classes(B, specs, wb, s, &data_of(C, &B));
  // U's class for each shift
  std::map<QN, int> ushift;
  for (size_t ci = 0; ci < U.cls.size(); ++ci) ushift[U.cls[ci].shift] = (int)ci;
  long long tmp_total = 0;
  struct Job {
    int bc, bb, uc, ub;
    long long tmp;
  };
  std::vector<Job> jobs;
  for (size_t bc = 0; bc < B.cls.size(); ++bc) {
    const OpClass &ob = B.cls[bc];
    if (ob.nnz == 0) continue;
    auto it = ushift.find(ob.shift);
    if (it == ushift.end()) fail(DMRG_ERR_STATE, "internal: missing class in renormalize");
    const OpClass &ou = U.cls[it->second];
    if (ou.nops != ob.nops) fail(DMRG_ERR_STATE, "internal: op count mismatch");
    for (size_t b = 0; b < ob.blk_in.size(); ++b) {
      int ki = ob.blk_in[b], ko = ob.blk_out[b];
      int ub = ou.in2blk[u_of[ki]];
      if (ub < 0 || ou.blk_out[ub] != u_of[ko]) fail(DMRG_ERR_STATE, "internal: block mismatch");
      jobs.push_back({(int)bc, (int)b, it->second, ub, 0});
    }
  }
  // The intermediates U_k T_i are computed for chunks of jobs whose
  // temporaries fit kRenTmpDoubles (a job larger than that is a chunk of its
  // own); the chunks run one after the other on the stream, reusing one buffer.
  std::vector<size_t> chunk{0};
  {
    long long cur = 0;
    for (size_t i = 0; i < jobs.size(); ++i) {
      const Job &j = jobs[i];
      const long long t = (long long)B.cls[j.bc].nops *
                          U.basis.dim[u_of[B.cls[j.bc].blk_out[j.bb]]] *
                          T.cols[B.cls[j.bc].blk_in[j.bb]];
      if (cur > 0 && cur + t > kRenTmpDoubles) {
        chunk.push_back(i);
        cur = 0;
      }
      jobs[i].tmp = cur;
      cur += t;
      tmp_total = std::max(tmp_total, cur);
    }
    chunk.push_back(jobs.size());
  }
  C->mem_max[2] = std::max(C->mem_max[2], 8.0 * tmp_total);
  WinBuf work(s);   // intermediate products and work lists of this call
  double *tmp = (double *)work.alloc(sizeof(double) * std::max<long long>(tmp_total, 1));
  for (size_t c = 0; c + 1 < chunk.size(); ++c) {
  std::vector<GemmDesc> d1, d2;
  std::vector<GemmSeg> s1, s2;
  long long t1 = 0, t2 = 0;
  for (size_t ji = chunk[c]; ji < chunk[c + 1]; ++ji) {
    const Job &j = jobs[ji];
    const OpClass &ob = B.cls[j.bc];
    const OpClass &ou = U.cls[j.uc];
    int ki = ob.blk_in[j.bb], ko = ob.blk_out[j.bb];
    int du_o = U.basis.dim[u_of[ko]], du_i = U.basis.dim[u_of[ki]];
    int db_o = T.cols[ko], db_i = T.cols[ki];
    // tmp_k = U_k (du_o x du_i) * T_i (du_i x db_i)
    GemmSeg g;
    memset(&g, 0, sizeof g);
    g.A = ou.d + ou.blk_off[j.ub];
    g.a_rs = du_i; g.a_cs = 1; g.a_bs = ou.nnz;
    g.B = T.d + T.off[ki];
    g.b_rs = db_i; g.b_cs = 1; g.b_bs = 0;
    g.K = du_i;
    GemmDesc d;
    memset(&d, 0, sizeof d);
    d.C = tmp + j.tmp;
    d.c_rs = db_i; d.c_cs = 1; d.c_bs = (long long)du_o * db_i;
    d.M = du_o; d.N = db_i; d.batch = ob.nops;
    d.seg0 = (int)s1.size(); d.nseg = 1;
    d.tiles_m = (du_o + 63) / 64; d.tiles_n = (db_i + 63) / 64;
    d.alpha = 1.0; d.beta = 0.0;
    d.tile0 = t1;
    t1 += (long long)d.tiles_m * d.tiles_n * d.batch;
    s1.push_back(g);
    d1.push_back(d);
    // out_k = T_o^T (db_o x du_o) * tmp_k (du_o x db_i)
    GemmSeg g2;
    memset(&g2, 0, sizeof g2);
    g2.A = T.d + T.off[ko];
    g2.a_rs = 1; g2.a_cs = db_o; g2.a_bs = 0;
    g2.B = tmp + j.tmp;
    g2.b_rs = db_i; g2.b_cs = 1; g2.b_bs = (long long)du_o * db_i;
    g2.K = du_o;
    GemmDesc e;
    memset(&e, 0, sizeof e);
    e.C = ob.d + ob.blk_off[j.bb];
    e.c_rs = db_i; e.c_cs = 1; e.c_bs = ob.nnz;
    e.M = db_o; e.N = db_i; e.batch = ob.nops;
    e.seg0 = (int)s2.size(); e.nseg = 1;
    e.tiles_m = (db_o + 63) / 64; e.tiles_n = (db_i + 63) / 64;
    e.alpha = 1.0; e.beta = 0.0;
    e.tile0 = t2;
    t2 += (long long)e.tiles_m * e.tiles_n * e.batch;
    s2.push_back(g2);
    d2.push_back(e);
  }
  if (!d1.empty()) {
    gemm_f64_grouped(d1, s1, work, s);
    gemm_f64_grouped(d2, s2, work, s);
  }
  }
  CK(cudaStreamSynchronize(s));
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// blocks from isometries
// ---------------------------------------------------------------------------
void drop_host_copy(BlockPart *B) {
  for (double *h : B->host)
    if (h) cudaFreeHost(h);
  B->host.clear();
}

void free_part(dmrg_ctx *C, BlockPart *B) {
  auto it = C->partbuf.find(B);
  if (it != C->partbuf.end()) C->partbuf.erase(it);
  auto jt = C->partdata.find(B);
  if (jt != C->partdata.end()) C->partdata.erase(jt);
  if (B) drop_host_copy(B);
}

WinBuf &buf_of(dmrg_ctx *C, BlockPart *B) {
  auto &p = C->partbuf[B];
  if (!p) p.reset(new WinBuf(WinBuf::lasting_buf()));
  return *p;
}

WinBuf &data_of(dmrg_ctx *C, BlockPart *B) {
  auto &p = C->partdata[B];
  if (!p) p.reset(new WinBuf(WinBuf::lasting_buf()));
  return *p;
}

// all renormalized blocks of the context (their device buffers too)
void clear_blocks(dmrg_ctx *C) {
  for (auto &b : C->L)
    if (b) free_part(C, b.get());
  for (auto &kv : C->R)
    if (kv.second) free_part(C, kv.second.get());
  C->L.clear();
  C->R.clear();
}

// ---------------------------------------------------------------------------
// HBM staging of renormalized block operators (cfg.hbm_budget_bytes > 0)
// ---------------------------------------------------------------------------
// A sweep holds every block L_n, R_n; on large lattices their operators
// exceed HBM.  Blocks are immutable once built, so a block whose next use is
// far away is offloaded: its operator data is copied once into pinned host
// memory and the device copy freed; it is copied back (on a side stream,
// ahead of use) when a window needs it.  A block that the sweep rebuilds
// before its next use is released outright.

long long data_bytes(const BlockPart &B) {
  long long b = 0;
  for (const OpClass &oc : B.cls) b += 8 * std::max<long long>(1, oc.nnz * oc.nops);
  return b;
}

void stage_init(dmrg_ctx *C) {
  if (!C->stage_stream) CK(cudaStreamCreateWithFlags(&C->stage_stream, cudaStreamNonBlocking));
  if (!C->stage_ev) CK(cudaEventCreateWithFlags(&C->stage_ev, cudaEventDisableTiming));
}

long long resident_bytes(dmrg_ctx *C) {
  long long r = 0;
  for (auto &b : C->L)
    if (b && b->state == 0) r += data_bytes(*b);
  for (auto &kv : C->R)
    if (kv.second && kv.second->state == 0) r += data_bytes(*kv.second);
  return r;
}

void offload(dmrg_ctx *C, BlockPart *B) {
  if (!B || B->state != 0 || B->cls.empty()) return;
  stage_init(C);
  if (B->host.empty()) {
    // wait for the work that built the block, then copy it out once
    CK(cudaEventRecord(C->stage_ev, C->stream));
    CK(cudaStreamWaitEvent(C->stage_stream, C->stage_ev, 0));
    B->host.assign(B->cls.size(), nullptr);
    for (size_t c = 0; c < B->cls.size(); ++c) {
      const size_t n = 8 * std::max<long long>(1, B->cls[c].nnz * B->cls[c].nops);
      if (cudaHostAlloc((void **)&B->host[c], n, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        fail(DMRG_ERR_OOM, "pinned host allocation of %zu bytes failed", n);
      }
      CK(cudaMemcpyAsync(B->host[c], B->cls[c].d, n, cudaMemcpyDeviceToHost, C->stage_stream));
      C->st_d2h_bytes += (double)n;
    }
    CK(cudaStreamSynchronize(C->stage_stream));
  }
  auto it = C->partdata.find(B);
  if (it != C->partdata.end()) C->partdata.erase(it);
  for (OpClass &oc : B->cls) oc.d = nullptr;
  B->state = 1;
  ++C->st_offloads;
}

// Copy an offloaded block back on the staging stream; `s` waits for it.
void reload(dmrg_ctx *C, BlockPart *B, cudaStream_t s) {
  if (!B || B->state != 1) return;
  stage_init(C);
  WinBuf &wb = data_of(C, B);
  std::array<cudaEvent_t, 2> ev{};
  CK(cudaEventCreate(&ev[0]));
  CK(cudaEventCreate(&ev[1]));
  CK(cudaEventRecord(ev[0], C->stage_stream));
  for (size_t c = 0; c < B->cls.size(); ++c) {
    const size_t n = 8 * std::max<long long>(1, B->cls[c].nnz * B->cls[c].nops);
    B->cls[c].d = (double *)wb.alloc(n);
    CK(cudaMemcpyAsync(B->cls[c].d, B->host[c], n, cudaMemcpyHostToDevice, C->stage_stream));
    C->st_h2d_bytes += (double)n;
  }
  CK(cudaEventRecord(ev[1], C->stage_stream));
  CK(cudaStreamWaitEvent(s, ev[1], 0));
  C->h2d_events.push_back(ev);
  B->state = 0;
  ++C->st_reloads;
}

void release(dmrg_ctx *C, BlockPart *B) {
  if (!B || B->state == 2) return;
  if (B->state == 0) {
    // the device data may still be read by queued work on the context stream
    CK(cudaStreamSynchronize(C->stream));
  }
  auto it = C->partdata.find(B);
  if (it != C->partdata.end()) C->partdata.erase(it);
  for (OpClass &oc : B->cls) oc.d = nullptr;
  drop_host_copy(B);
  B->state = 2;
  ++C->st_releases;
}

void need(dmrg_ctx *C, BlockPart *B, cudaStream_t s) {
  if (!B) return;
  if (B->state == 2) fail(DMRG_ERR_STATE, "internal: a released block is used");
  reload(C, B, s);
}

// Window steps from sweep position (pass, l) to the next use of L_n (left) or
// R_n; -1 when the sweep rebuilds the block before using it again.  Pass 0
// runs l = 0..N-2 (left to right), pass 1 l = N-2..0; window l uses L_l and
// R_{l+2}.
long long next_use(int N, int pass, int l, bool left, int n) {
  const int w = left ? n : n - 2;
  if (w == l) return 0;
  if (pass == 0) {
    if (left) return w < l ? (long long)(N - 2 - l) + 1 + (N - 2 - w) : -1;
    return w > l ? w - l : -1;
  }
  if (left) return w < l ? l - w : -1;
  return w > l ? (long long)l + 1 + w : -1;
}

void collect_h2d_times(dmrg_ctx *C);

// Before window l of pass `pass`: release stale blocks, bring the window's
// blocks in, offload the blocks used last until the resident ones fit the
// budget, and prefetch the next window's blocks if they fit as well.
void stage_window(dmrg_ctx *C, int pass, int l) {
  const long long budget = (long long)C->cfg.hbm_budget_bytes;
  if (budget <= 0) return;
  const int N = C->N;
  struct Item {
    BlockPart *b;
    long long nu;
  };
  std::vector<Item> items;
  for (size_t n = 0; n < C->L.size(); ++n)
    if (C->L[n] && !C->L[n]->cls.empty()) items.push_back({C->L[n].get(), next_use(N, pass, l, true, (int)n)});
  for (auto &kv : C->R)
    if (kv.second && !kv.second->cls.empty())
      items.push_back({kv.second.get(), next_use(N, pass, l, false, kv.first)});
  for (Item &it : items)
    if (it.nu < 0) release(C, it.b);
  for (Item &it : items)
    if (it.nu == 0) need(C, it.b, C->stream);
  std::sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.nu > b.nu; });
  long long res = resident_bytes(C);
  for (Item &it : items) {
    if (res <= budget) break;
    if (it.nu <= 0 || it.b->state != 0) continue;
    res -= data_bytes(*it.b);
    offload(C, it.b);
  }
  // prefetch: the soonest-used offloaded blocks that fit
  std::sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.nu < b.nu; });
  for (Item &it : items) {
    if (it.nu <= 0 || it.b->state != 1) continue;
    if (res + data_bytes(*it.b) > budget) break;
    res += data_bytes(*it.b);
    reload(C, it.b, C->stream);
  }
  C->st_peak = std::max(C->st_peak, (double)resident_bytes(C));
  if (C->h2d_events.size() > 64) collect_h2d_times(C);
}

void collect_h2d_times(dmrg_ctx *C) {
  for (auto &ev : C->h2d_events) {
    CK(cudaEventSynchronize(ev[1]));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    C->st_h2d_ms += ms;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  C->h2d_events.clear();
}

std::unique_ptr<BlockPart> vacuum(dmrg_ctx *C) {
  std::unique_ptr<BlockPart> v(new BlockPart());
  v->basis.qn.push_back({0, 0});
  v->basis.dim.push_back(1);
  // every operator of the vacuum is zero: no classes, all references empty
  return v;
}

void upload_iso(dmrg_ctx *C, Iso &T) {
  if (T.d) return;
  WinBuf &wb = buf_of(C, nullptr);
  T.d = (double *)wb.alloc(sizeof(double) * std::max<size_t>(T.host.size(), 1));
  CK(cudaMemcpyAsync(T.d, T.host.data(), sizeof(double) * T.host.size(), cudaMemcpyHostToDevice,
                     C->stream));
}

// L_n = T_n^T (L_{n-1} x site_{n-1}) T_n
double part_bytes(const BlockPart &P) {
  double b = 0;
  for (const OpClass &oc : P.cls) b += 8.0 * (double)oc.nnz * oc.nops;
  return b;
}

void note_parts(dmrg_ctx *C, const BlockPart &U, const BlockPart &B) {
  C->mem_max[1] = std::max(C->mem_max[1], part_bytes(U));
  C->mem_max[0] = std::max(C->mem_max[0], part_bytes(B));
}

void grow_left(dmrg_ctx *C, int n, const Iso &T) {
  SitePart st = site_of(C, n - 1);
  BlockPart U;
  WinBuf ub(C->stream);
  need(C, C->L[n - 1].get(), C->stream);
  enlarge(C, *C->L[n - 1], st, false, C->N - n, U, ub);
  std::unique_ptr<BlockPart> B(new BlockPart());
  renormalize(C, U, T, *B, buf_of(C, B.get()));
  note_parts(C, U, *B);
  if ((int)C->L.size() <= n) C->L.resize(n + 1);
  if (C->L[n]) free_part(C, C->L[n].get());
  C->L[n] = std::move(B);
}

// R_n = T_n^T (site_n x R_{n+1}) T_n
void grow_right(dmrg_ctx *C, int n, const Iso &T) {
  SitePart st = site_of(C, n);
  BlockPart U;
  WinBuf ub(C->stream);
  need(C, C->R[n + 1].get(), C->stream);
  enlarge(C, *C->R[n + 1], st, true, n, U, ub);
  std::unique_ptr<BlockPart> B(new BlockPart());
  renormalize(C, U, T, *B, buf_of(C, B.get()));
  note_parts(C, U, *B);
  if (C->R.count(n)) free_part(C, C->R[n].get());
  C->R[n] = std::move(B);
}

// ---------------------------------------------------------------------------
// the window (l, l+1): enlarged blocks, H_eff term stacks, GEMM lists
// ---------------------------------------------------------------------------

void block_src(const BlockPart &P, const Fac &f, int in_sec, int out_sec, SCopy &cp) {
  // operator f restricted to block (out_sec <- in_sec) as a copy source
  cp.src = nullptr;
  cp.ident = 0;
  cp.trans = 0;
  if (f.kind == 2) {
    cp.ident = (in_sec == out_sec);
    return;
  }
  if (f.kind != 1) return;
  const OpClass &oc = P.cls[f.ref.cls];
  const double *base = oc.d + (long long)f.ref.idx * oc.nnz;
  if (!f.trans) {
    int b = oc.in2blk[in_sec];
    if (b < 0 || oc.blk_out[b] != out_sec) return;
    cp.src = base + oc.blk_off[b];
    cp.src_ld = P.basis.dim[in_sec];
  } else {
    int b = oc.in2blk[out_sec];
    if (b < 0 || oc.blk_out[b] != in_sec) return;
    cp.src = base + oc.blk_off[b];
    cp.trans = 1;
    cp.src_ld = P.basis.dim[out_sec];
  }
}

// the window's buffers are freed on the release stream: make it wait for the
// last H_eff*psi that callers enqueued on their own streams
void release_after_use(Window &w) {
  if (w.used) cudaStreamWaitEvent(release_stream(), w.use_ev, 0);
  w.used = false;
}

// after a public H_eff*psi call on stream s (the event exists once a window
// has been built, so recording it allocates nothing)
void note_use(Window &w, cudaStream_t s) {
  CK(cudaEventRecord(w.use_ev, s));
  w.used = true;
}

void build_window(dmrg_ctx *C, int l) {
  Window &w = C->win;
  cudaStream_t s = C->stream;
  w.valid = false;
  // the FP64 stacks are unmapped on the host: the previous window's work ends first
  if (w.used) CK(cudaEventSynchronize(w.use_ev));
  CK(cudaStreamSynchronize(s));
  w.vA.free_all();
  w.vB.free_all();
  w.vT.free_all();
  w.fp64_stacks = false;
  w.stack_copies.clear();
  release_after_use(w);
  if (!w.use_ev) CK(cudaEventCreateWithFlags(&w.use_ev, cudaEventDisableTiming));
  w.buf.clear();
  w.ldbuf.clear();
  w.rdbuf.clear();
  w.tf_ready = false;
  w.tf_copies = false;
  for (auto &g : w.graphs) cudaGraphExecDestroy(g.second);
  w.graphs.clear();
  for (auto &b : w.batch)
    for (auto &g : b.second.graphs) cudaGraphExecDestroy(g.second);
  w.batch.clear();
  for (int i = 0; i < 6; ++i) {
    w.tbl_ptr[i] = nullptr;
    w.tbl_cap[i] = 0;
  }
  static std::atomic<long long> build_counter{0};
  w.gen = ++build_counter;
  w.Ld = BlockPart();
  w.Rd = BlockPart();
  w.hc.clear();
  w.psi.clear();
  w.l = l;
  w.flops1 = w.flops2 = 0;
  double t0 = now();
  {
    SitePart sl = site_of(C, l), sr = site_of(C, l + 1);
    need(C, C->L[l].get(), C->stream);
    need(C, C->R[l + 2].get(), C->stream);
    enlarge(C, *C->L[l], sl, false, C->N - l - 1, w.Ld, w.ldbuf);
    enlarge(C, *C->R[l + 2], sr, true, l + 1, w.Rd, w.rdbuf);
  }
  C->prof[1] += now() - t0;
  t0 = now();
  // psi layout
  w.a2psi.assign(w.Ld.basis.qn.size(), -1);
  long long off = 0;
  for (size_t a = 0; a < w.Ld.basis.qn.size(); ++a) {
    int b = w.Rd.basis.find(partner(C, w.Ld.basis.qn[a]));
    if (b < 0) continue;
    w.a2psi[a] = (int)w.psi.size();
    w.psi.push_back({(int)a, b, off, w.Ld.basis.dim[a], w.Rd.basis.dim[b]});
    off += (long long)w.Ld.basis.dim[a] * w.Rd.basis.dim[b];
  }
  w.psi_len = off;
  // H_eff terms, grouped by the shift of the L. factor
  Side F, G;
  F.b = &w.Ld;
  G.b = &w.Rd;
  std::map<QN, int> cidx;
  AddFn add = [&](const Fac &A, const Fac &B, double coef) {
    if (A.kind == 0 || B.kind == 0) return;
    if (qadd(A.shift, B.shift) != QN{0, 0}) fail(DMRG_ERR_STATE, "internal: H_eff term shift");
    auto it = cidx.find(A.shift);
    int ci;
    if (it == cidx.end()) {
      ci = (int)w.hc.size();
      cidx[A.shift] = ci;
      HClass h;
      h.dA = A.shift;
      h.pB = B.parity;
      w.hc.push_back(h);
    } else {
      ci = it->second;
    }
    w.hc[ci].terms.push_back({A, B, coef});
  };
  if (C->su2) {
    // spin-adapted: H = sum alpha [A^k (x) B^k]^0; component g of A (spin
    // change 2(J_a' - J_a) = g) pairs with component g of B (total S = 0
    // keeps J_a = J_b); adjoint tensors use the transposed component -g
    const SideS sl = side_of_defined(w.Ld), sr = side_of_defined(w.Rd);
    const SU2Terms &al = derive_in(C, derive_table(C, sl, sr), sl, sr, TKey{0, 0, 0, 0});
    auto comp = [](const BlockPart &P, const TKey &k, int adj, int g) {
      Fac f;
      if (k.kind < 0) {
        if (g == 0) f.kind = 2;
        return f;
      }
      const TRef &tr = P.ten.at(k);
      const Ref r = tr.r[((adj ? -g : g) + tr.tk) / 2];
      if (r.cls < 0) return f;
      f.kind = 1;
      f.ref = r;
      f.trans = adj;
      f.shift = adj ? qneg(P.cls[r.cls].shift) : P.cls[r.cls].shift;
      f.parity = P.cls[r.cls].parity;
      return f;
    };
    for (auto &kv : al) {
      const TKey &ka = std::get<0>(kv.first), &kb = std::get<2>(kv.first);
      const int aa = std::get<1>(kv.first), ab = std::get<3>(kv.first);
      const int tka = ka.kind < 0 ? 0 : ka.tk, tkb = kb.kind < 0 ? 0 : kb.tk;
      if (tka != tkb) fail(DMRG_ERR_STATE, "internal: H_eff term of ranks %d, %d", tka, tkb);
      for (int g = -tka; g <= tka; g += 2) {
        const Fac A = comp(w.Ld, ka, aa, g), B = comp(w.Rd, kb, ab, g);
        if (A.kind == 0 || B.kind == 0) continue;
        if (su2::n_of(A.shift) + su2::n_of(B.shift) != 0 || su2::tj_of(A.shift) != su2::tj_of(B.shift))
          fail(DMRG_ERR_STATE, "internal: spin-adapted H_eff term shift");
        auto it = cidx.find(A.shift);
        int ci;
        if (it == cidx.end()) {
          ci = (int)w.hc.size();
          cidx[A.shift] = ci;
          HClass h;
          h.dA = A.shift;
          h.pB = B.parity;
          w.hc.push_back(h);
        } else {
          ci = it->second;
        }
        TermF t{A, B, kv.second};
        t.tk = tka;
        t.adjA = ka.kind < 0 ? 0 : aa;
        t.adjB = kb.kind < 0 ? 0 : ab;
        w.hc[ci].terms.push_back(t);
      }
    }
  } else {
    formula_H(F, G, add, true);
  }
  // stacks and T layout
  long long nA = 0, nB = 0, nT = 0;
  std::vector<SCopy> cps;
  std::vector<S1> s1list;
  for (size_t ci = 0; ci < w.hc.size(); ++ci) {
    HClass &h = w.hc[ci];
    const long long n = (long long)h.terms.size();
    for (size_t pi = 0; pi < w.psi.size(); ++pi) {
      const PsiBlk &p = w.psi[pi];
      int ao = w.Ld.basis.find(qadd(w.Ld.basis.qn[p.a], h.dA));
      if (ao < 0 || w.a2psi[ao] < 0) continue;
      const PsiBlk &q = w.psi[w.a2psi[ao]];
      h.a_off[(int)pi] = nA;
      h.b_off[(int)pi] = nB;
      h.t_off[(int)pi] = nT;
      nA += (long long)q.da * n * p.da;
      nB += (long long)q.db * n * p.db;
      nT += (long long)q.da * n * p.db;
      s1list.push_back({(int)ci, (int)pi, w.a2psi[ao]});
    }
  }
  w.nA = nA;
  w.nB = nB;
  w.nT = nT;
  w.vA.reserve(8 * (size_t)std::max<long long>(nA, 1));
  w.vA.map();
  w.vB.reserve(8 * (size_t)std::max<long long>(nB, 1));
  w.vB.map();
  w.vT.reserve(8 * (size_t)std::max<long long>(nT, 1));   // backed by the first FP64 apply
  w.Astack = w.vA.ptr();
  w.Bstack = w.vB.ptr();
  w.T = w.vT.ptr();
  for (const S1 &e : s1list) {
    HClass &h = w.hc[e.ci];
    const PsiBlk &p = w.psi[e.pi], &q = w.psi[e.po];
    const int n = (int)h.terms.size();
    for (int k = 0; k < n; ++k) {
      const TermF &t = h.terms[k];
      SCopy a;
      memset(&a, 0, sizeof a);
      block_src(w.Ld, t.A, p.a, q.a, a);
      a.coef = t.A.scale;
      a.rows = q.da;
      a.cols = p.da;
      a.dst = w.Astack + h.a_off[e.pi] + (long long)k * p.da;
      a.dst_ld = (long long)n * p.da;
      cps.push_back(a);
      SCopy b;
      memset(&b, 0, sizeof b);
      block_src(w.Rd, t.B, p.b, q.b, b);
      b.coef = t.coef * t.B.scale;
      if (t.tk >= 0) {
        // recoupling of [A^k (x) B^k]^0 between the window's coupled spins
        // (and the adjoint factors of transposed blocks)
        const int ja = su2::tj_of(w.Ld.basis.qn[p.a]), jap = su2::tj_of(w.Ld.basis.qn[q.a]);
        const int jb = su2::tj_of(w.Rd.basis.qn[p.b]), jbp = su2::tj_of(w.Rd.basis.qn[q.b]);
        const int tS = su2::tj_of(C->target);
        double f = su2::coupling(ja, jb, tS, jap, jbp, tS, t.tk, t.tk, 0);
        if (t.adjA) f *= su2::adjoint_factor(ja, jap, t.tk);
        if (t.adjB) f *= su2::adjoint_factor(jb, jbp, t.tk);
        b.coef *= f;
      }
      b.rows = q.db;
      b.cols = p.db;
      b.dst = w.Bstack + h.b_off[e.pi] + (long long)k * p.db;
      b.dst_ld = (long long)n * p.db;
      cps.push_back(b);
    }
  }
  {
    WinBuf tmp(s);
    SCopy *d = upload(tmp, cps, s);
    CK(launch_stack_copy(d, (int)cps.size(), s));
    CK(cudaStreamSynchronize(s));
  }
  w.stack_copies = cps;
  w.fp64_stacks = true;
  C->mem_max[1] = std::max({C->mem_max[1], part_bytes(w.Ld), part_bytes(w.Rd)});
  C->mem_max[3] = (double)(w.vA.size + w.vB.size);
  // stage 1: T[(a',k), b] = A[(a',k), a] psi[a, b] * sign
  // stage 2: sigma[a', b'] = sum_classes T[a', (k,b)] B[b', (k,b)]^T
  std::vector<GemmDesc> d1, d2;
  std::vector<GemmSeg> g1, g2;
  long long t1 = 0, t2 = 0;
  double flops = 0;
  std::vector<std::vector<S1>> into(w.psi.size());
  for (const S1 &e : s1list) {
    HClass &h = w.hc[e.ci];
    const PsiBlk &p = w.psi[e.pi], &q = w.psi[e.po];
    const int n = (int)h.terms.size();
    GemmSeg g;
    memset(&g, 0, sizeof g);
    g.A = w.Astack + h.a_off[e.pi];
    g.a_rs = p.da; g.a_cs = 1;
    g.B = nullptr;            // psi, bound at apply time (offset kept in b_bs)
    g.b_bs = p.off;
    g.b_rs = p.db; g.b_cs = 1;
    g.K = p.da;
    GemmDesc d;
    memset(&d, 0, sizeof d);
    d.C = w.T + h.t_off[e.pi];
    d.c_rs = p.db; d.c_cs = 1;
    d.M = q.da * n; d.N = p.db; d.batch = 1;
    d.seg0 = (int)g1.size(); d.nseg = 1;
    d.tiles_m = (d.M + 63) / 64; d.tiles_n = (d.N + 63) / 64;
    int nl = qnum(w.Ld.basis.qn[p.a]);
    d.alpha = (h.pB && (nl & 1)) ? -1.0 : 1.0;
    d.beta = 0.0;
    d.tile0 = t1;
    t1 += (long long)d.tiles_m * d.tiles_n;
    g1.push_back(g);
    d1.push_back(d);
    into[e.po].push_back(e);
    flops += 2.0 * q.da * (double)n * p.da * p.db + 2.0 * q.da * (double)n * p.db * q.db;
    w.flops1 += 2.0 * q.da * (double)n * p.da * p.db;
    w.flops2 += 2.0 * q.da * (double)n * p.db * q.db;
  }
  // stage 2 in FP64: split-K over ranges of at most KSUB64 of the long K
  // (terms x psi columns); each range writes an FP64 partial block, and the
  // partials are summed in a fixed order (deterministic).
  const int KSUB64 = 2048;
  long long wsn = 0;
  std::vector<PartialSum64> ps64;
  struct Range {
    const S1 *e;
    int k0, K;
  };
  std::vector<std::vector<Range>> ranges(w.psi.size());
  for (size_t po = 0; po < w.psi.size(); ++po) {
    for (const S1 &e : into[po]) {
      const int K = (int)w.hc[e.ci].terms.size() * w.psi[e.pi].db;
      for (int k0 = 0; k0 < K; k0 += KSUB64) ranges[po].push_back({&e, k0, std::min(KSUB64, K - k0)});
    }
    const PsiBlk &q = w.psi[po];
    PartialSum64 p;
    p.ws = nullptr;
    p.stride = (long long)q.da * q.db;
    p.off = q.off;
    p.n = q.da * q.db;
    p.nparts = (int)ranges[po].size();
    ps64.push_back(p);
    wsn += (long long)p.nparts * p.stride;
  }
  w.ws64 = (double *)w.buf.alloc(8 * std::max<long long>(wsn, 1));
  long long wo = 0;
  for (size_t po = 0; po < w.psi.size(); ++po) {
    const PsiBlk &q = w.psi[po];
    ps64[po].ws = w.ws64 + wo;
    for (size_t r = 0; r < ranges[po].size(); ++r) {
      const Range &rg = ranges[po][r];
      const HClass &h = w.hc[rg.e->ci];
      const PsiBlk &p = w.psi[rg.e->pi];
      const int n = (int)h.terms.size();
      GemmSeg g;
      memset(&g, 0, sizeof g);
      g.A = w.T + h.t_off.at(rg.e->pi) + rg.k0;
      g.a_rs = (long long)n * p.db; g.a_cs = 1;
      g.B = w.Bstack + h.b_off.at(rg.e->pi) + rg.k0;
      g.b_rs = 1; g.b_cs = (long long)n * p.db;
      g.K = rg.K;
      GemmDesc d;
      memset(&d, 0, sizeof d);
      d.C = w.ws64 + wo + (long long)r * q.da * q.db;
      d.c_rs = q.db; d.c_cs = 1;
      d.M = q.da; d.N = q.db; d.batch = 1;
      d.seg0 = (int)g2.size(); d.nseg = 1;
      d.tiles_m = (d.M + 63) / 64; d.tiles_n = (d.N + 63) / 64;
      d.alpha = 1.0; d.beta = 0.0;
      d.tile0 = t2;
      t2 += (long long)d.tiles_m * d.tiles_n;
      g2.push_back(g);
      d2.push_back(d);
    }
    wo += (long long)ps64[po].nparts * ps64[po].stride;
  }
  w.ps64 = ps64;
  w.flops = flops;
  w.stage1 = d1;
  w.seg1 = g1;
  w.stage2 = d2;
  w.seg2 = g2;
  w.s1 = upload(w.buf, w.seg1, s);
  w.s2 = upload(w.buf, w.seg2, s);
  // the H_eff stages (one problem per descriptor) run on square tiles; the
  // rectangular ones measured slower there
  w.f64_1 = plan_gemm_f64(w.stage1, w.seg1, w.buf, s, true);
  w.f64_2 = plan_gemm_f64(w.stage2, w.seg2, w.buf, s, true);
  w.d_ps64 = upload(w.buf, w.ps64, s);
  w.s1info = s1list;
  // diagonal of H_eff for the Davidson preconditioner: shift-0 class terms
  w.diag = (double *)w.buf.alloc(8 * std::max<long long>(w.psi_len, 1));
  CK(cudaMemsetAsync(w.diag, 0, 8 * std::max<long long>(w.psi_len, 1), s));
  {
    std::vector<GemmDesc> dd;
    std::vector<GemmSeg> gg;
    long long tt = 0;
    for (size_t ci = 0; ci < w.hc.size(); ++ci) {
      HClass &h = w.hc[ci];
      if (h.dA != QN{0, 0}) continue;
      const int n = (int)h.terms.size();
      for (auto &kv : h.a_off) {
        const PsiBlk &p = w.psi[kv.first];
        GemmSeg g;
        memset(&g, 0, sizeof g);
        g.A = w.Astack + kv.second;            // A[i][k][i]
        g.a_rs = (long long)n * p.da + 1; g.a_cs = p.da;
        g.B = w.Bstack + h.b_off[kv.first];    // B[j][k][j]
        g.b_rs = p.db; g.b_cs = (long long)n * p.db + 1;
        g.K = n;
        GemmDesc d;
        memset(&d, 0, sizeof d);
        d.C = w.diag + p.off;
        d.c_rs = p.db; d.c_cs = 1;
        d.M = p.da; d.N = p.db; d.batch = 1;
        d.seg0 = (int)gg.size(); d.nseg = 1;
        d.tiles_m = (p.da + 63) / 64; d.tiles_n = (p.db + 63) / 64;
        d.alpha = 1.0; d.beta = 0.0;
        d.tile0 = tt;
        tt += (long long)d.tiles_m * d.tiles_n;
        gg.push_back(g);
        dd.push_back(d);
      }
    }
    if (!dd.empty()) {
      WinBuf tmp(s);
      GemmDesc *a = upload(tmp, dd, s);
      GemmSeg *b = upload(tmp, gg, s);
      CK(launch_gemm_f64(a, (int)dd.size(), b, tt, s));
      CK(cudaStreamSynchronize(s));
    }
  }
  C->prof[2] += now() - t0;
  w.valid = true;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
    C->mem_max[5] = std::max(C->mem_max[5], (double)(tot - fr));
}

void collect_timing(dmrg_ctx *C) {
  if (!C->pending) return;
  CK(cudaEventSynchronize(C->ev[4]));
  for (int i = 0; i < 4; ++i) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, C->ev[i], C->ev[i + 1]));
    C->tacc[i] += ms;
  }
  C->tacc[4] += 1;
  C->pending = false;
}

void mark(dmrg_ctx *C, int i, cudaStream_t s) {
  if (!C->timing) return;
  if (i == 0) collect_timing(C);
  CK(cudaEventRecord(C->ev[i], s));
  if (i == 4) C->pending = true;
}

// The FP64 path's memory: T backed on first use; A and B gathered again from
// the window's enlarged blocks if they were given back (stream-ordered on s).
void ensure_fp64(dmrg_ctx *C, cudaStream_t s) {
  Window &w = C->win;
  if (!w.vT.mapped) w.vT.map();
  if (w.fp64_stacks) return;
  w.vA.map();
  w.vB.map();
  WinBuf tmp(s);
  SCopy *d = upload(tmp, w.stack_copies, s);
  CK(launch_stack_copy(d, (int)w.stack_copies.size(), s));
  w.fp64_stacks = true;
}

// Under an HBM budget the split path keeps only its FP16 copies: A, B and T
// of the FP64 path are given back (their addresses stay reserved).
void drop_fp64(dmrg_ctx *C) {
  Window &w = C->win;
  CK(cudaStreamSynchronize(C->stream));
  if (w.used) CK(cudaEventSynchronize(w.use_ev));
  w.vA.unmap();
  w.vB.unmap();
  w.vT.unmap();
  w.fp64_stacks = false;
}

void apply_fp64(dmrg_ctx *C, const double *psi, double *sigma, cudaStream_t s) {
  Window &w = C->win;
  ensure_fp64(C, s);
  mark(C, 0, s);
  mark(C, 1, s);
  run_gemm_f64(w.f64_1, w.s1, s, psi, nullptr);
  mark(C, 2, s);
  run_gemm_f64(w.f64_2, w.s2, s);
  CK(launch_sum_partials64(w.d_ps64, (int)w.ps64.size(), sigma, s));
  mark(C, 3, s);
  mark(C, 4, s);
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// split-precision plan: scaled FP16 (hi, lo) copies of the stacks, tensor maps
// and tile lists of the two tcgen05 stages
// ---------------------------------------------------------------------------
long long r4(long long x) { return (x + 3) & ~3LL; }
long long r8(long long x) { return (x + 7) & ~7LL; }
long long r16(long long x) { return (x + 15) & ~15LL; }
long long a64(long long x) { return (x + 63) & ~63LL; }
int ntile_of(int n) { return n > 128 ? 128 : ((n + 15) / 16) * 16; }

// Sizes of the per-apply scratch of the split path: psi^T split (P, halves,
// hi and lo each), stage-1 intermediate (T, halves, hi and lo each) and
// stage-2 partial tiles (ws, floats).
struct SplitScratch {
  long long nP = 0, nT = 0, nws = 0;
  std::vector<long long> offP, offT, ldP, ldT;
};

const int KSUB_DEFAULT = 1024;   // longest K range of one stage-2 work item
const int KSUB_CANDIDATES[3] = {1024, 2048, 4096};

std::vector<std::vector<int>> entries_into(const Window &w) {
  std::vector<std::vector<int>> into(w.psi.size());
  for (size_t i = 0; i < w.s1info.size(); ++i) into[w.s1info[i].po].push_back((int)i);
  return into;
}

SplitScratch split_scratch_sizes(const Window &w, int KSUB) {
  SplitScratch z;
  const auto &E = w.s1info;
  const size_t ne = E.size(), np = w.psi.size();
  z.offT.assign(ne, 0);
  z.ldT.resize(ne);
  z.offP.resize(np);
  z.ldP.resize(np);
  for (size_t i = 0; i < ne; ++i) {
    const HClass &h = w.hc[E[i].ci];
    const PsiBlk &p = w.psi[E[i].pi], &q = w.psi[E[i].po];
    const long long n = (long long)h.terms.size();
    z.ldT[i] = r8(p.db);   // T rows (a', k), b padded to 8 halves
    z.offT[i] = z.nT;
    z.nT += a64(q.da * n * z.ldT[i]);
  }
  for (size_t i = 0; i < np; ++i) {
    z.ldP[i] = r16(w.psi[i].da);   // K of stage 1, zero-padded to 16 halves
    z.offP[i] = z.nP;
    z.nP += a64(w.psi[i].db * z.ldP[i]);
  }
  const auto into = entries_into(w);
  for (size_t po = 0; po < np; ++po) {
    long long parts = 0;
    for (int i : into[po]) {
      const long long K = (long long)w.hc[E[i].ci].terms.size() * r8(w.psi[E[i].pi].db);
      parts += (K + KSUB - 1) / KSUB;
    }
    z.nws += a64(parts * w.psi[po].da * r4(w.psi[po].db));
  }
  return z;
}

// most 32 x 32 tiles of one F16Split descriptor (CTAs per descriptor worth launching)
int split_tile_count(const std::vector<F16Split> &v) {
  int m = 1;
  for (const F16Split &d : v) m = std::max(m, ((d.rows + 31) / 32) * ((d.cols + 31) / 32));
  return m;
}

// Scaled FP16 (hi, lo) copies of the operator stacks: built once per window
// and owned by the context (inputs of every split-path apply).  Each class
// entry's A and B stacks get one power-of-two scale from their largest
// element; the largest A-row 2-norm bounds the entry's stage-1 output.
void split_operator_copies(dmrg_ctx *C) {
  Window &w = C->win;
  cudaStream_t s = C->stream;
  SplitPlan &P = w.tf;
  const auto &E = w.s1info;
  const size_t ne = E.size();
  w.offA.assign(ne, 0);
  w.ldA.assign(ne, 0);
  w.offBp.assign(ne, 0);
  w.bpad.assign(ne, 0);
  long long nA = 0, nBp = 0;
  std::vector<StatDesc> sd(ne);
  for (size_t i = 0; i < ne; ++i) {
    const HClass &h = w.hc[E[i].ci];
    const PsiBlk &p = w.psi[E[i].pi], &q = w.psi[E[i].po];
    const long long n = (long long)h.terms.size();
    w.ldA[i] = r16(p.da);   // K of stage 1, zero-padded to 16 halves
    w.offA[i] = nA;
    nA += a64(q.da * n * w.ldA[i]);
    w.bpad[i] = r8(p.db);
    w.offBp[i] = nBp;
    nBp += a64(q.db * n * w.bpad[i]);
    memset(&sd[i], 0, sizeof sd[i]);
    sd[i].a = w.Astack + h.a_off.at(E[i].pi);
    sd[i].rowsA = (long long)q.da * n;
    sd[i].colsA = p.da;
    sd[i].b = w.Bstack + h.b_off.at(E[i].pi);
    sd[i].rowsB = (long long)q.db * n;
    sd[i].colsB = p.db;
  }
  WinBuf tmp(s);
  EntryStat *dst = (EntryStat *)tmp.alloc(sizeof(EntryStat) * std::max<size_t>(ne, 1));
  CK(entry_stats(upload(tmp, sd, s), (int)ne, dst, s));
  std::vector<EntryStat> st(ne);
  if (ne) CK(cudaMemcpyAsync(st.data(), dst, sizeof(EntryStat) * ne, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  w.sA.resize(ne);
  w.sB.resize(ne);
  w.rnA.resize(ne);
  for (size_t i = 0; i < ne; ++i) {
    w.sA[i] = pow2_scale_host(st[i].maxA);
    w.sB[i] = pow2_scale_host(st[i].maxB);
    w.rnA[i] = st[i].rnA;
  }
  auto hf = [&](long long n) { return (__half *)w.buf.alloc(2 * std::max<long long>(n, 64)); };
  P.Ah = hf(nA);
  P.Al = hf(nA);
  // B with every term's b segment padded to 8 halves (zeros), so that stage 2
  // runs over K = (k, b) with b padded and each term starts 16-byte aligned
  P.Bh = hf(nBp);
  P.Bl = hf(nBp);
  CK(cudaMemsetAsync(P.Bh, 0, 2 * std::max<long long>(nBp, 64), s));
  CK(cudaMemsetAsync(P.Bl, 0, 2 * std::max<long long>(nBp, 64), s));
  std::vector<F16Split> sp;
  for (size_t i = 0; i < ne; ++i) {
    const PsiBlk &p = w.psi[E[i].pi], &q = w.psi[E[i].po];
    const int n = (int)w.hc[E[i].ci].terms.size();
    F16Split a;
    memset(&a, 0, sizeof a);
    a.src = sd[i].a;
    a.src_ld = p.da;
    a.rows = q.da * n;
    a.cols = p.da;
    a.hi = P.Ah + w.offA[i];
    a.lo = P.Al + w.offA[i];
    a.dst_ld = w.ldA[i];
    a.scale = w.sA[i];
    sp.push_back(a);
    // rows (b', k) of the [b'][k][b] stack, each p.db long, re-strided to bpad
    F16Split b;
    memset(&b, 0, sizeof b);
    b.src = sd[i].b;
    b.src_ld = p.db;
    b.rows = q.db * n;
    b.cols = p.db;
    b.hi = P.Bh + w.offBp[i];
    b.lo = P.Bl + w.offBp[i];
    b.dst_ld = w.bpad[i];
    b.scale = w.sB[i];
    sp.push_back(b);
  }
  CK(f16_split(upload(tmp, sp, s), (int)sp.size(), nullptr, nullptr, s, split_tile_count(sp)));
  CK(cudaStreamSynchronize(s));
  w.tf_copies = true;
  C->mem_max[4] = 4.0 * (double)(nA + nBp);
}

// psi (FP64, [a][b] per sector block) -> scaled FP16 (hi, lo), transposed to
// [b][a]; the scale comes from the block's statistics of this apply
std::vector<F16Split> psi_split_descs(const Window &w, const SplitScratch &z, __half *Ph,
                                      __half *Pl) {
  std::vector<F16Split> out;
  for (size_t i = 0; i < w.psi.size(); ++i) {
    F16Split d;
    memset(&d, 0, sizeof d);
    d.src = nullptr;
    d.src_off = w.psi[i].off;
    d.src_ld = w.psi[i].db;
    d.rows = w.psi[i].da;
    d.cols = w.psi[i].db;
    d.trans = 1;
    d.hi = Ph + z.offP[i];
    d.lo = Pl + z.offP[i];
    d.dst_ld = z.ldP[i];
    d.pblk = (int)i;
    d.scale = 0.f;
    out.push_back(d);
  }
  return out;
}

std::vector<PsiDesc> psi_descs(const Window &w) {
  std::vector<PsiDesc> out(w.psi.size());
  for (size_t i = 0; i < w.psi.size(); ++i) out[i] = {w.psi[i].off, w.psi[i].da, w.psi[i].db};
  return out;
}

// Stage-1 schedule: tiles of psi blocks wider than cap1 (128 or 64) are cap1
// wide; order1 = 0 rounds of one item per SM from the heavy, light and middle
// thirds of the cost-sorted items in turn, 1 cost order alone, 2 heaviest and
// lightest items alternating.
// nv > 1: one plan for nv vectors stored one after the other psi_stride
// apart (psi and sigma); vector v uses the v-th copy of the per-apply scratch
// (z sizes each: P at v * z.nP, T at v * z.nT, partial tiles at v * z.nws)
// and psi statistics v * np + block.  Every work item appears once per
// vector, the copies next to each other in the claim order, so that they run
// at about the same time and the copies after the first take the shared
// operator tile from L2.
void split_tables(const Window &w, const SplitScratch &z, __half *Ph, __half *Pl, __half *Th,
                  __half *Tl, float *ws, SplitTables &out, int KSUB, int cap1 = 128,
                  int order1 = 0, int nv = 1, long long psi_stride = 0) {
  auto ntile1 = [cap1](int n) { return std::min(ntile_of(n), cap1); };
  const SplitPlan &P = w.tf;
  const auto &E = w.s1info;
  const size_t ne = E.size(), np = w.psi.size();
  out = SplitTables();
  for (int v = 0; v < nv; ++v) {
    std::vector<F16Split> d = psi_split_descs(w, z, Ph + (long long)v * z.nP, Pl + (long long)v * z.nP);
    for (F16Split &x : d) {
      x.src_off += v * psi_stride;
      x.pblk += v * (int)np;
    }
    out.psi_split.insert(out.psi_split.end(), d.begin(), d.end());
  }
  auto &maps = out.maps;
  auto mk = [&](const __half *base, long long rows, long long cols, long long ld, int box) {
    CUtensorMap m;
    int rc = encode_map_h(&m, base, rows, cols, ld, box);
    if (rc != 0) fail(DMRG_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) rows %lld cols %lld", rc, rows, cols);
    maps.push_back(m);
    return (int)maps.size() - 1;
  };
  auto mk3h = [&](const __half *base, long long d0, long long d1, long long s1) {
    CUtensorMap m;
    int rc = encode_map3_h(&m, base, d0, d1, 1, s1, d1 * s1, 32, 1);
    if (rc != 0) fail(DMRG_ERR_CUDA, "cuTensorMapEncodeTiled (3-D, store) failed (%d)", rc);
    maps.push_back(m);
    return (int)maps.size() - 1;
  };
  auto mk3 = [&](const float *base, long long d0, long long d1, long long d2, long long s1,
                 long long s2, int b0, int b1, int b2) {
    CUtensorMap m;
    int rc = encode_map3(&m, base, d0, d1, d2, s1, s2, b0, b1, b2);
    if (rc != 0) fail(DMRG_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed (%d)", rc);
    maps.push_back(m);
    return (int)maps.size() - 1;
  };
  std::vector<int> mPh(nv * np), mPl(nv * np);
  for (int v = 0; v < nv; ++v)
    for (size_t i = 0; i < np; ++i) {
      const PsiBlk &p = w.psi[i];
      const long long o = (long long)v * z.nP + z.offP[i];
      mPh[v * np + i] = mk(Ph + o, p.db, z.ldP[i], z.ldP[i], ntile1(p.db));
      mPl[v * np + i] = mk(Pl + o, p.db, z.ldP[i], z.ldP[i], ntile1(p.db));
    }
  auto &segs = out.segs;
  auto &w1 = out.w1;
  auto &w2 = out.w2;
  const auto into = entries_into(w);
  // per entry: stage-1 tiles, and the maps stage 2 reads (T per vector)
  std::vector<int> mThi(nv * ne), mTlo(nv * ne), mBhi(ne), mBlo(ne);
  // stage-2 packing of small sigma blocks: R segments per 128 x 128 tile
  std::vector<int> Rq(np, 1);
  for (size_t po = 0; po < np; ++po) {
    const PsiBlk &q = w.psi[po];
    Rq[po] = (q.da <= 32 && q.db <= 32) ? 4 : ((q.da <= 64 && q.db <= 64) ? 2 : 1);
  }
  std::vector<float> alpha(ne);
  for (size_t i = 0; i < ne; ++i) {
    const HClass &h = w.hc[E[i].ci];
    const PsiBlk &p = w.psi[E[i].pi], &q = w.psi[E[i].po];
    const int n = (int)h.terms.size();
    const int nl = qnum(w.Ld.basis.qn[p.a]);
    alpha[i] = (h.pB && (nl & 1)) ? -1.f : 1.f;
    const long long bp = z.ldT[i];   // = r8(p.db)
    const int ahi = mk(P.Ah + w.offA[i], (long long)q.da * n, w.ldA[i], w.ldA[i], 128);
    const int alo = mk(P.Al + w.offA[i], (long long)q.da * n, w.ldA[i], w.ldA[i], 128);
    // T as stage-1 output: rows (a', k), columns b (padded); as stage-2
    // operand: rows a', K = (k, b)
    const long long rowsT = (long long)q.da * n;
    const int R = Rq[E[i].po];
    std::vector<int> sThi(nv), sTlo(nv), seg(nv);
    for (int v = 0; v < nv; ++v) {
      const long long o = (long long)v * z.nT + z.offT[i];
      sThi[v] = mk3h(Th + o, bp, rowsT, bp);
      sTlo[v] = mk3h(Tl + o, bp, rowsT, bp);
      mThi[v * ne + i] = mk(Th + o, q.da, (long long)n * bp, (long long)n * bp, 128 / R);
      mTlo[v * ne + i] = mk(Tl + o, q.da, (long long)n * bp, (long long)n * bp, 128 / R);
      TSeg sg;
      memset(&sg, 0, sizeof sg);
      sg.mA_hi = ahi; sg.mA_lo = alo;
      sg.mB_hi = mPh[v * np + E[i].pi]; sg.mB_lo = mPl[v * np + E[i].pi];
      sg.K = p.da;
      sg.k0 = 0;
      seg[v] = (int)segs.size();
      segs.push_back(sg);
    }
    int bbox = R > 1 ? 128 / R : ntile_of(q.db);
    mBhi[i] = mk(P.Bh + w.offBp[i], q.db, (long long)n * w.bpad[i], (long long)n * w.bpad[i], bbox);
    mBlo[i] = mk(P.Bl + w.offBp[i], q.db, (long long)n * w.bpad[i], (long long)n * w.bpad[i], bbox);
    const int M = q.da * n, N = p.db, nt = ntile1(N);
    for (int m0 = 0; m0 < M; m0 += 128)
      for (int n0 = 0; n0 < N; n0 += nt)
        for (int v = 0; v < nv; ++v) {
          TWork t;
          memset(&t, 0, sizeof t);
          t.s = segs[seg[v]];
          t.M = M; t.N = N; t.m0 = m0; t.n0 = n0; t.ntile = nt;
          t.mode = TW_SPLIT; t.alpha = alpha[i];
          t.fa = 1.f / w.sA[i];
          t.rn = w.rnA[i];
          t.pblk = v * (int)np + E[i].pi;
          t.mOut_hi = sThi[v]; t.mOut_lo = sTlo[v]; t.zout = 0;
          w1.push_back(t);
        }
  }
  // per sigma block: split-K ranges (one entry each), each one FP32 partial
  // tile per output tile; the partials are summed in a fixed order.
  long long wsn = 0;
  struct PackCand {
    int seg, mOut, z, R, nchunk, entry, vec;
  };
  std::vector<PackCand> pk;
  for (size_t po = 0; po < np; ++po) {
    const PsiBlk &q = w.psi[po];
    const long long ldw = r4(q.db), blk = (long long)q.da * ldw;
    const int M = q.da, N = q.db, nt = ntile_of(N);
    std::vector<int> rent;   // entry of each K range
    std::vector<int> rk0, rK;
    for (int i : into[po]) {
      const HClass &h = w.hc[E[i].ci];
      const int K = (int)(h.terms.size() * w.bpad[i]);
      for (int k0 = 0; k0 < K; k0 += KSUB) {
        rent.push_back(i);
        rk0.push_back(k0);
        rK.push_back(std::min(KSUB, K - k0));
      }
    }
    const int nparts = (int)rent.size();
    std::vector<int> mW(nv, -1);
    for (int v = 0; v < nv; ++v) {
      PartialSum ps;
      memset(&ps, 0, sizeof ps);
      ps.ws = ws + (long long)v * z.nws + wsn;
      ps.stride = blk;
      ps.off = v * psi_stride + q.off;
      ps.ld = ldw;
      ps.n = q.da * q.db;
      ps.cols = q.db;
      ps.nparts = nparts;   // 0: no term reaches this block, sigma = 0
      out.psums.push_back(ps);
      if (nparts) mW[v] = mk3(ws + (long long)v * z.nws + wsn, q.db, q.da, nparts, ldw, blk, 32, 32, 1);
    }
    if (nparts == 0) continue;
    for (int pi = 0; pi < nparts; ++pi) {
      const int i = rent[pi];
      const HClass &h = w.hc[E[i].ci];
      const int K = (int)(h.terms.size() * w.bpad[i]);
      std::vector<int> seg(nv);
      for (int v = 0; v < nv; ++v) {
        TSeg sg;
        memset(&sg, 0, sizeof sg);
        sg.mA_hi = mThi[v * ne + i]; sg.mA_lo = mTlo[v * ne + i];
        sg.mB_hi = mBhi[i]; sg.mB_lo = mBlo[i];
        sg.k0 = rk0[pi];
        sg.K = rK[pi];
        sg.xoob = (K + 63) / 64 * 64;
        seg[v] = (int)segs.size();
        segs.push_back(sg);
      }
      if (Rq[po] > 1) {
        for (int v = 0; v < nv; ++v) pk.push_back({seg[v], mW[v], pi, Rq[po], (rK[pi] + 63) / 64, i, v});
        continue;
      }
      for (int m0 = 0; m0 < M; m0 += 128)
        for (int n0 = 0; n0 < N; n0 += nt)
          for (int v = 0; v < nv; ++v) {
            TWork t;
            memset(&t, 0, sizeof t);
            t.s = segs[seg[v]];
            t.M = M; t.N = N; t.m0 = m0; t.n0 = n0; t.ntile = nt;
            t.mode = TW_PARTIAL; t.alpha = 1.f;
            t.fa = 1.f / w.sB[i];
            t.rn = w.rnA[i];
            t.pblk = v * (int)np + E[i].pi;
            t.mOut_hi = mW[v]; t.mOut_lo = mW[v]; t.zout = pi;
            w2.push_back(t);
          }
    }
    wsn += a64((long long)nparts * blk);
  }
  if (wsn > z.nws) fail(DMRG_ERR_STATE, "internal: partial-tile workspace size");
  // packed stage-2 tiles: segments of equal R, longest first, R per tile
  std::stable_sort(pk.begin(), pk.end(), [](const PackCand &a, const PackCand &b) {
    if (a.R != b.R) return a.R > b.R;
    return a.nchunk > b.nchunk;
  });
  for (size_t i0 = 0; i0 < pk.size();) {
    const int R = pk[i0].R;
    TWork t;
    memset(&t, 0, sizeof t);
    t.M = 128; t.N = 128; t.ntile = 128;
    t.mode = TW_PARTIAL; t.alpha = 1.f;
    t.R = R;
    for (int r = 0; r < 4; ++r) t.pseg[r] = -1;
    size_t i = i0;
    for (int r = 0; r < R && i < pk.size() && pk[i].R == R; ++r, ++i) {
      t.pseg[r] = pk[i].seg;
      t.pout[r] = pk[i].mOut;
      t.pz[r] = pk[i].z;
      t.pfa[r] = 1.f / w.sB[pk[i].entry];
      t.prn[r] = w.rnA[pk[i].entry];
      t.ppb[r] = pk[i].vec * (int)np + E[pk[i].entry].pi;
      t.nchunk = std::max(t.nchunk, pk[i].nchunk);
    }
    t.s = segs[t.pseg[0]];
    w2.push_back(t);
    i0 = i;
  }
  // persistent CTAs claim work items in list order: order them by cost (K chunks
  // x tile width), largest first
  auto cost = [&](const TWork &t) {
    if (t.R > 1) return (long long)t.nchunk * t.ntile;
    return (long long)((t.s.K + 63) / 64) * t.ntile;
  };
  // stage 2 runs as one launch of the 128-wide kernel (it takes any tile
  // width), largest cost first
  std::stable_sort(w2.begin(), w2.end(), [&](const TWork &a, const TWork &b) {
    return cost(a) > cost(b);
  });
  // Stage 1 runs as one launch of the 128-wide kernel (it takes any tile
  // width).  Narrow tiles are bound by per-tile latency and wide ones by HBM
  // bandwidth, so they should run at the same time: the items, sorted by
  // cost, are arranged in rounds of one item per SM, and rounds from the
  // heavy, light and middle thirds follow each other; claimed in that order,
  // they give every CTA a mix of widths and about the same total cost.
  std::stable_sort(w1.begin(), w1.end(), [&](const TWork &a, const TWork &b) {
    return cost(a) > cost(b);
  });
  if (order1 == 2) {
    std::vector<TWork> alt;
    alt.reserve(w1.size());
    for (size_t i = 0, j = w1.size(); i < j;) {
      alt.push_back(w1[i++]);
      if (i < j) alt.push_back(w1[--j]);
    }
    w1.swap(alt);
  } else if (order1 == 0) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 148;
    // full rounds interleaved; the lightest remainder (a partial round) last,
    // so every round stays aligned with the CTAs
    const size_t n = w1.size(), G = (size_t)nsm, rounds = n / G;
    std::vector<TWork> mixed;
    mixed.reserve(n);
    // heavy, light and middle thirds of the rounds taken in turn
    const size_t t1 = rounds / 3, t2 = 2 * rounds / 3;
    auto put_round = [&](size_t r) {
      for (size_t k = r * G; k < (r + 1) * G; ++k) mixed.push_back(w1[k]);
    };
    for (size_t h = 0, m = t1, l = rounds; h < t1 || m < t2 || l > t2;) {
      if (h < t1) put_round(h++);
      if (l > t2) put_round(--l);
      if (m < t2) put_round(m++);
    }
    for (size_t k = rounds * G; k < n; ++k) mixed.push_back(w1[k]);
    w1.swap(mixed);
  }
}

void upload_tables(dmrg_ctx *C, SplitTables &tb, cudaStream_t s);
void launch_split(dmrg_ctx *C, const double *psi, double *sigma, cudaStream_t s);

// Autotuner: the stage-2 split-K range trades FP32 accumulation length against
// partial-tile traffic and tile count.  For windows whose operator stacks are
// large enough for the choice to matter, each candidate is timed on the live
// window (three applies each, CUDA events) and the fastest is kept for the
// rest of the context's life (windows of one run have similar shapes).
void build_split(dmrg_ctx *C) {
  Window &w = C->win;
  cudaStream_t s = C->stream;
  SplitPlan &P = w.tf;
  if (!w.tf_copies) {
    split_operator_copies(C);
    if (C->cfg.hbm_budget_bytes) drop_fp64(C);
  }
  CK(split_prepare());
  const bool tune = C->ksub_choice == 0 && (double)(w.nA + w.nB) * 8.0 > 256e6;
  int best = C->ksub_choice ? C->ksub_choice : KSUB_DEFAULT;
  // scratch sized for the smallest candidate (most partial tiles)
  SplitScratch zmax = split_scratch_sizes(w, tune ? KSUB_CANDIDATES[0] : best);
  auto fl = [&](long long n) { return (float *)w.buf.alloc(4 * std::max<long long>(n, 64)); };
  auto hf = [&](long long n) { return (__half *)w.buf.alloc(2 * std::max<long long>(n, 64)); };
  P.Ph = hf(zmax.nP);
  P.Pl = hf(zmax.nP);
  P.Th = hf(zmax.nT);
  P.Tl = hf(zmax.nT);
  P.ws = fl(zmax.nws);
  P.pstat = (PsiStat *)w.buf.alloc(sizeof(PsiStat) * std::max<size_t>(w.psi.size(), 1));
  P.psi_desc = upload(w.buf, psi_descs(w), s);
  P.err = (int *)w.buf.alloc(sizeof(int));
  P.next = (int *)w.buf.alloc(2 * sizeof(int));
  CK(cudaMemsetAsync(P.err, 0, sizeof(int), s));
  if (tune) {
    WinBuf tb(s);
    double *x = (double *)tb.alloc(8 * std::max<long long>(w.psi_len, 1));
    double *y = (double *)tb.alloc(8 * std::max<long long>(w.psi_len, 1));
    CK(launch_random(x, w.psi_len, 12345, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (int ks : KSUB_CANDIDATES) {
      SplitScratch z = split_scratch_sizes(w, ks);
      split_tables(w, z, P.Ph, P.Pl, P.Th, P.Tl, P.ws, C->tables, ks);
      upload_tables(C, C->tables, s);
      launch_split(C, x, y, s);   // warm
      CK(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) launch_split(C, x, y, s);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      // candidates run smallest range first; a longer range (longer FP32
      // accumulation) must win by more than 1.5% to be taken
      if (ms < best_ms * 0.985f) {
        best_ms = ms;
        best = ks;
      }
      C->tune_log.push_back({(double)ks, ms / 3.0});
    }
    C->ksub_choice = best;
    // stage-1 schedule with that range: tile-width cap x item order, the
    // current default (128, mixed thirds) first; another must win by 1.5 %
    const int cand[6][2] = {{128, 0}, {128, 1}, {128, 2}, {64, 0}, {64, 1}, {64, 2}};
    SplitScratch zb = split_scratch_sizes(w, best);
    float best1 = 1e30f;
    int bc = 128, bo = 0;
    for (auto &c : cand) {
      split_tables(w, zb, P.Ph, P.Pl, P.Th, P.Tl, P.ws, C->tables, best, c[0], c[1]);
      upload_tables(C, C->tables, s);
      launch_split(C, x, y, s);   // warm
      CK(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) launch_split(C, x, y, s);
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best1 * 0.985f) {
        best1 = ms;
        bc = c[0];
        bo = c[1];
      }
      // logged as 100000 + 10 * cap + order, beside the split-K ranges
      C->tune_log.push_back({100000.0 + 10.0 * c[0] + c[1], ms / 3.0});
    }
    C->cap1_choice = bc;
    C->order1_choice = bo;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  w.ksub = best;
  w.cap1 = C->cap1_choice ? C->cap1_choice : 128;
  w.order1 = C->cap1_choice ? C->order1_choice : 0;
  SplitScratch z = split_scratch_sizes(w, best);
  split_tables(w, z, P.Ph, P.Pl, P.Th, P.Tl, P.ws, C->tables, best, w.cap1, w.order1);
  upload_tables(C, C->tables, s);
  CK(cudaStreamSynchronize(s));
  w.tf_ready = true;
}

void upload_tables(dmrg_ctx *C, SplitTables &tb, cudaStream_t s) {
  Window &w = C->win;
  SplitPlan &P = w.tf;
  // table buffers: grow-only, so the tuner's candidates can reuse them
  auto need = [&](void *&ptr, size_t &cap, size_t bytes) {
    if (bytes > cap) {
      ptr = w.buf.alloc(bytes);
      cap = bytes;
    }
  };
  need(w.tbl_ptr[0], w.tbl_cap[0], std::max<size_t>(tb.psi_split.size(), 1) * sizeof(F16Split));
  need(w.tbl_ptr[1], w.tbl_cap[1], std::max<size_t>(tb.maps.size(), 1) * sizeof(CUtensorMap));
  need(w.tbl_ptr[2], w.tbl_cap[2], std::max<size_t>(tb.segs.size(), 1) * sizeof(TSeg));
  need(w.tbl_ptr[3], w.tbl_cap[3], std::max<size_t>(tb.w1.size(), 1) * sizeof(TWork));
  need(w.tbl_ptr[4], w.tbl_cap[4], std::max<size_t>(tb.w2.size(), 1) * sizeof(TWork));
  need(w.tbl_ptr[5], w.tbl_cap[5], std::max<size_t>(tb.psums.size(), 1) * sizeof(PartialSum));

  auto put = [&](void *dst, const void *src, size_t n) {
    if (n) CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s));
  };
  put(w.tbl_ptr[0], tb.psi_split.data(), tb.psi_split.size() * sizeof(F16Split));
  put(w.tbl_ptr[1], tb.maps.data(), tb.maps.size() * sizeof(CUtensorMap));
  put(w.tbl_ptr[2], tb.segs.data(), tb.segs.size() * sizeof(TSeg));
  put(w.tbl_ptr[3], tb.w1.data(), tb.w1.size() * sizeof(TWork));
  put(w.tbl_ptr[4], tb.w2.data(), tb.w2.size() * sizeof(TWork));
  put(w.tbl_ptr[5], tb.psums.data(), tb.psums.size() * sizeof(PartialSum));

  P.psi_split = w.tbl_ptr[0];
  P.npsi = (int)tb.psi_split.size();
  P.psi_tiles = split_tile_count(tb.psi_split);
  P.maps = (CUtensorMap *)w.tbl_ptr[1];
  P.seg = (TSeg *)w.tbl_ptr[2];
  P.work1 = (TWork *)w.tbl_ptr[3];
  P.work2 = (TWork *)w.tbl_ptr[4];
  P.psum = (PartialSum *)w.tbl_ptr[5];
  P.nwork1 = (int)tb.w1.size();
  P.nwork2 = (int)tb.w2.size();
  P.npsum = (int)tb.psums.size();
  CK(cudaStreamSynchronize(s));
  for (auto &g : w.graphs) cudaGraphExecDestroy(g.second);
  w.graphs.clear();
}

void launch_split(dmrg_ctx *C, const double *psi, double *sigma, cudaStream_t s) {
  SplitPlan &P = C->win.tf;
  mark(C, 0, s);
  CK(psi_stats(P.psi_desc, P.npsi, psi, P.pstat, s));
  CK(f16_split((const F16Split *)P.psi_split, P.npsi, P.pstat, psi, s, P.psi_tiles));
  mark(C, 1, s);
  CK(split_gemm(P.work1, P.nwork1, P.next, P.seg, P.maps, P.pstat, P.err, s));
  mark(C, 2, s);
  CK(split_gemm(P.work2, P.nwork2, P.next + 1, P.seg, P.maps, P.pstat, P.err, s));
  mark(C, 3, s);
  CK(sum_partials(P.psum, P.npsum, sigma, s));
  mark(C, 4, s);
}

// The split apply is a handful of launches; it is captured once per (psi, sigma) pair
// into a CUDA graph and replayed (Davidson reuses a fixed set of vector slots).
// With per-stage timing on, the launches go out directly.
void apply_split(dmrg_ctx *C, const double *psi, double *sigma, cudaStream_t s) {
  Window &w = C->win;
  if (!w.tf_ready) {
    cudaStream_t save = C->stream;
    C->stream = s;
    build_split(C);
    C->stream = save;
  }
  if (C->timing || !C->use_graphs) {
    launch_split(C, psi, sigma, s);
    return;
  }
  auto key = std::make_pair((const void *)psi, (const void *)sigma);
  auto it = w.graphs.find(key);
  if (it == w.graphs.end()) {
    // callers that pass ever new buffers would grow the cache without bound:
    // keep at most 64 graphs per window (a destroyed graph still in flight
    // completes first)
    if (w.graphs.size() >= 64) {
      for (auto &g : w.graphs) cudaGraphExecDestroy(g.second);
      w.graphs.clear();
    }
    // record on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on `s`
    if (!C->cap_stream) CK(cudaStreamCreateWithFlags(&C->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = C->cap_stream;
    cudaGraph_t g;
    {
      std::unique_lock<std::shared_mutex> lk(capture_lock());
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      try {
        launch_split(C, psi, sigma, cs);
      } catch (...) {
        cudaStreamEndCapture(cs, &g);
        throw;
      }
      CK(cudaStreamEndCapture(cs, &g));
    }
    cudaGraphExec_t ge;
    CK(cudaGraphInstantiate(&ge, g, 0));
    cudaGraphDestroy(g);
    it = w.graphs.emplace(key, ge).first;
  }
  CK(cudaGraphLaunch(it->second, s));
}

// Synchronous read of the window's bounded-wait error word (split path).  The
// word is cleared once read, so a time-out is reported once.
void apply(dmrg_ctx *C, const double *psi, double *sigma, cudaStream_t s, int precision);

// ---------------------------------------------------------------------------
// multi-vector split apply: nv vectors against one pass over the operators
// ---------------------------------------------------------------------------
BatchPlan &batch_plan(dmrg_ctx *C, int nv, cudaStream_t s) {
  Window &w = C->win;
  auto it = w.batch.find(nv);
  if (it != w.batch.end()) return it->second;
  if (!w.tf_ready) {
    cudaStream_t save = C->stream;
    C->stream = s;
    build_split(C);
    C->stream = save;
  }
  BatchPlan &b = w.batch[nv];
  b.nv = nv;
  const SplitScratch z = split_scratch_sizes(w, w.ksub);
  auto fl = [&](long long n) { return (float *)w.buf.alloc(4 * std::max<long long>(n, 64)); };
  auto hf = [&](long long n) { return (__half *)w.buf.alloc(2 * std::max<long long>(n, 64)); };
  b.Ph = hf(nv * z.nP);
  b.Pl = hf(nv * z.nP);
  b.Th = hf(nv * z.nT);
  b.Tl = hf(nv * z.nT);
  b.ws = fl(nv * z.nws);
  const size_t np = w.psi.size();
  b.pstat = (PsiStat *)w.buf.alloc(sizeof(PsiStat) * std::max<size_t>(nv * np, 1));
  std::vector<PsiDesc> pd;
  for (int v = 0; v < nv; ++v)
    for (const PsiDesc &d : psi_descs(w)) pd.push_back({d.off + v * w.psi_len, d.rows, d.cols});
  b.pdesc = upload(w.buf, pd, s);
  b.next = (int *)w.buf.alloc(2 * sizeof(int));
  split_tables(w, z, b.Ph, b.Pl, b.Th, b.Tl, b.ws, b.tb, w.ksub, w.cap1, w.order1, nv, w.psi_len);
  b.dsplit = upload(w.buf, b.tb.psi_split, s);
  b.dmaps = upload(w.buf, b.tb.maps, s);
  b.dseg = upload(w.buf, b.tb.segs, s);
  b.dw1 = upload(w.buf, b.tb.w1, s);
  b.dw2 = upload(w.buf, b.tb.w2, s);
  b.dps = upload(w.buf, b.tb.psums, s);
  b.psi_tiles = split_tile_count(b.tb.psi_split);
  CK(cudaStreamSynchronize(s));
  return b;
}

void launch_batch(dmrg_ctx *C, BatchPlan &b, const double *psi, double *sigma, cudaStream_t s) {
  Window &w = C->win;
  const int nps = (int)(b.nv * w.psi.size());
  CK(psi_stats(b.pdesc, nps, psi, b.pstat, s));
  CK(f16_split((const F16Split *)b.dsplit, (int)b.tb.psi_split.size(), b.pstat, psi, s, b.psi_tiles));
  CK(split_gemm((const TWork *)b.dw1, (int)b.tb.w1.size(), b.next, (const TSeg *)b.dseg,
                (const CUtensorMap *)b.dmaps, b.pstat, w.tf.err, s));
  CK(split_gemm((const TWork *)b.dw2, (int)b.tb.w2.size(), b.next + 1, (const TSeg *)b.dseg,
                (const CUtensorMap *)b.dmaps, b.pstat, w.tf.err, s));
  CK(sum_partials((const PartialSum *)b.dps, (int)b.tb.psums.size(), sigma, s));
}

// nv vectors psi[v * psi_len ...] -> sigma[v * psi_len ...]; FP64 precision
// applies them one by one, the split precision in one batched pass (graph
// replay per (psi, sigma) pair as for single vectors)
void apply_batch(dmrg_ctx *C, int nv, const double *psi, double *sigma, cudaStream_t s) {
  Window &w = C->win;
  if (C->precision == DMRG_FP64 || nv == 1) {
    for (int v = 0; v < nv; ++v)
      apply(C, psi + (long long)v * w.psi_len, sigma + (long long)v * w.psi_len, s, C->precision);
    return;
  }
  BatchPlan &b = batch_plan(C, nv, s);
  if (!C->use_graphs) {
    launch_batch(C, b, psi, sigma, s);
    return;
  }
  auto key = std::make_pair((const void *)psi, (const void *)sigma);
  auto it = b.graphs.find(key);
  if (it == b.graphs.end()) {
    if (b.graphs.size() >= 16) {
      for (auto &g : b.graphs) cudaGraphExecDestroy(g.second);
      b.graphs.clear();
    }
    if (!C->cap_stream) CK(cudaStreamCreateWithFlags(&C->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = C->cap_stream;
    cudaGraph_t g;
    {
      std::unique_lock<std::shared_mutex> lk(capture_lock());
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      try {
        launch_batch(C, b, psi, sigma, cs);
      } catch (...) {
        cudaStreamEndCapture(cs, &g);
        throw;
      }
      CK(cudaStreamEndCapture(cs, &g));
    }
    cudaGraphExec_t ge;
    CK(cudaGraphInstantiate(&ge, g, 0));
    cudaGraphDestroy(g);
    it = b.graphs.emplace(key, ge).first;
  }
  CK(cudaGraphLaunch(it->second, s));
}

void check_err_flag(dmrg_ctx *C, cudaStream_t s) {
  Window &w = C->win;
  if (!w.tf_ready) return;
  int e = 0;
  CK(cudaMemcpyAsync(&e, w.tf.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e) {
    CK(cudaMemsetAsync(w.tf.err, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    fail(DMRG_ERR_TIMEOUT, "tcgen05 kernel: bounded wait %d gave up", e);
  }
}

// After a public split apply on stream s: queue a copy of the device error
// word (which = 0: the window's, 1: the static scratch's) into the context's
// pinned host word.  poll_flags reads it once the copy has landed.
void post_flag(dmrg_ctx *C, int which, const int *dflag, cudaStream_t s) {
  if (!C->hflag) return;
  CK(cudaMemcpyAsync(C->hflag + which, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(C->flag_ev[which], s));
  C->flag_pending[which] = true;
}

// Reads the posted error words whose copies have landed (wait: all of them).
// A set word becomes the context's sticky error (owed to the caller) and is
// cleared on the device on stream s.
void poll_flags(dmrg_ctx *C, bool wait, cudaStream_t s) {
  for (int i = 0; i < 2; ++i) {
    if (!C->flag_pending[i]) continue;
    if (wait) {
      CK(cudaEventSynchronize(C->flag_ev[i]));
    } else {
      cudaError_t q = cudaEventQuery(C->flag_ev[i]);
      if (q == cudaErrorNotReady) continue;
      CK(q);
    }
    C->flag_pending[i] = false;
    const int e = C->hflag[i];
    if (!e) continue;
    C->hflag[i] = 0;
    if (i == 0 && C->win.tf_ready) CK(cudaMemsetAsync(C->win.tf.err, 0, sizeof(int), s));
    if (i == 1) {
      void *b = nullptr;
      size_t cap = 0;
      CK(static_scratch(&b, &cap));
      CK(cudaMemsetAsync(b, 0, sizeof(int), s));
    }
    if (C->sticky == DMRG_OK) {
      C->sticky = DMRG_ERR_TIMEOUT;
      char buf[160];
      snprintf(buf, sizeof buf, "tcgen05 kernel (%s path): bounded wait %d gave up in an earlier "
               "H_eff*psi; its sigma is incomplete", i == 0 ? "window" : "static", e);
      C->sticky_msg = buf;
    }
  }
}

// Raise the error owed to the caller, once.
void take_sticky(dmrg_ctx *C) {
  if (C->sticky == DMRG_OK) return;
  Err e{C->sticky, C->sticky_msg};
  C->sticky = DMRG_OK;
  C->sticky_msg.clear();
  throw e;
}

void apply(dmrg_ctx *C, const double *psi, double *sigma, cudaStream_t s, int precision) {
  if (precision == DMRG_SPLIT) apply_split(C, psi, sigma, s);
  else apply_fp64(C, psi, sigma, s);
}

// ---------------------------------------------------------------------------
// Davidson (FP64 orthogonalisation, subspace, residual)
// ---------------------------------------------------------------------------
void jacobi_eig(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
        double c = 1 / std::sqrt(t * t + 1), sn = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - sn * akq;
          A[k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - sn * aqk;
          A[q * n + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - sn * vkq;
          V[k * n + q] = sn * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

struct DavBuf {
  double *V, *AV, *t, *u, *work, *coef, *dots;
};

DavBuf dav_buffers(dmrg_ctx *C, long long n, int m) {
  if (C->dav_n != n || !C->V) {
    C->dav.clear();
    C->dav = WinBuf::lasting_buf();
    C->V = (double *)C->dav.alloc(8 * (size_t)n * m);
    C->AV = (double *)C->dav.alloc(8 * (size_t)n * m);
    C->r = (double *)C->dav.alloc(8 * (size_t)n * 2);
    C->rs = (double *)C->dav.alloc(8 * (size_t)n * 3);
    C->jd = (double *)C->dav.alloc(8 * (size_t)n * 4);
    C->work = (double *)C->dav.alloc(8 * 296 * (size_t)(m + 2));
    C->small = (double *)C->dav.alloc(8 * 4 * (size_t)(m + 2));
    C->dav_n = n;
  }
  return {C->V, C->AV, C->r, C->r + n, C->work, C->small, C->small + 2 * (m + 2)};
}

double dot1(dmrg_ctx *C, const double *a, const double *b, long long n, DavBuf &B, cudaStream_t s) {
  CK(launch_dots(a, 1, n, b, n, B.work, B.dots, s));
  double v;
  CK(cudaMemcpyAsync(&v, B.dots, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return v;
}

void dots(dmrg_ctx *C, const double *V, int k, long long n, const double *x, DavBuf &B,
          std::vector<double> &out, cudaStream_t s) {
  out.resize(k);
  CK(launch_dots(V, k, n, x, n, B.work, B.dots, s));
  CK(cudaMemcpyAsync(out.data(), B.dots, 8 * k, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
}

// out = a*out + sum c_i V_i (coefficients by value: no copy, no host wait)
void lincomb(double *out, const double *V, const std::vector<double> &c, double a, long long n,
             DavBuf &B, cudaStream_t s) {
  if (c.size() <= (size_t)kLincombMax) {
    LincombCoef h;
    for (size_t i = 0; i < c.size(); ++i) h.c[i] = c[i];
    CK(launch_lincomb_v(out, V, (int)c.size(), n, h, a, n, s));
    return;
  }
  std::vector<double> h(c);
  h.push_back(a);
  CK(cudaMemcpyAsync(B.coef, h.data(), 8 * h.size(), cudaMemcpyHostToDevice, s));
  CK(launch_lincomb(out, V, (int)c.size(), n, B.coef, a != 0.0 ? B.coef + c.size() : nullptr, n, s));
  CK(cudaStreamSynchronize(s));
}

// Correction of the mixed-precision refinement (Jacobi-Davidson form):
// approximately solve  (I - u u^T)(H - theta)(I - u u^T) t = -r,  t orthogonal
// to the Ritz vector u (B.u), with `steps` preconditioned conjugate-gradient
// steps whose products use the split-precision path.  theta is the lowest
// Ritz value, so the projected operator is positive definite on u's
// complement; the diagonal preconditioner is (diag - theta)^-1, projected.
// On entry B.t holds the residual r = (H - theta) u (orthogonal to u); on
// exit the correction.  The FP64 Rayleigh-Ritz step that uses it keeps the
// result exact to FP64: the split product only shapes the search direction.
void jd_correction(dmrg_ctx *C, DavBuf &B, long long n, double theta, const double *th_dev,
                   int steps, cudaStream_t s) {
  Window &w = C->win;
  double *res = C->jd, *z = C->jd + n, *p = C->jd + 2 * n, *q = C->jd + 3 * n;
  auto project = [&](double *v) {
    const double a = dot1(C, B.u, v, n, B, s);
    lincomb(v, B.u, {-a}, 1.0, n, B, s);
  };
  auto precond = [&]() {
    CK(cudaMemcpyAsync(z, res, 8 * n, cudaMemcpyDeviceToDevice, s));
    CK(launch_precond(z, w.diag, th_dev, n, s));
    project(z);
  };
  CK(cudaMemcpyAsync(res, B.t, 8 * n, cudaMemcpyDeviceToDevice, s));
  lincomb(res, res, {}, -1.0, n, B, s);
  CK(cudaMemsetAsync(B.t, 0, 8 * n, s));
  const double r0 = std::sqrt(std::max(0.0, dot1(C, res, res, n, B, s)));
  precond();
  CK(cudaMemcpyAsync(p, z, 8 * n, cudaMemcpyDeviceToDevice, s));
  double rz = dot1(C, res, z, n, B, s);
  for (int it = 0; it < steps && rz > 0.0; ++it) {
    apply(C, p, q, s, DMRG_SPLIT);
    lincomb(q, p, {-theta}, 1.0, n, B, s);
    project(q);
    const double pq = dot1(C, p, q, n, B, s);
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    lincomb(B.t, p, {alpha}, 1.0, n, B, s);
    lincomb(res, q, {-alpha}, 1.0, n, B, s);
    const double rr = std::sqrt(std::max(0.0, dot1(C, res, res, n, B, s)));
    if (rr < 1e-3 * r0) break;
    precond();
    const double rz2 = dot1(C, res, z, n, B, s);
    const double beta = rz2 / rz;
    rz = rz2;
    lincomb(p, z, {1.0}, beta, n, B, s);
  }
}

constexpr double kSplitResidualFloor = 4e-6;
constexpr int kKrylovWarmup = 12;

// patience: split path only, iterations without halving the best residual
// before a residual near the noise floor is accepted.  probe: before
// accepting, add one random direction to the search space and go on for
// another `patience` iterations; accept only once such a probe has not
// lowered the Ritz value (a start vector with almost no weight on the ground
// state lets an excited state reach the floor first).
int davidson_run(dmrg_ctx *C, double *x, double *energy, int *iters, cudaStream_t s, int prec,
                 int patience, bool probe, double *rnorm_out, int jd_steps = 0) {
  Window &w = C->win;
  const long long n = w.psi_len;
  const int m = std::max(4, std::min(C->cfg.davidson_max_sub, 64));
  const int maxit = std::max(1, C->cfg.davidson_max_iter);
  const double tol = C->cfg.davidson_tol > 0 ? C->cfg.davidson_tol : 1e-8;
  DavBuf B = dav_buffers(C, n, m);
  double t0 = now();
  int nmv = 0;
  // start vector
  double nx = dot1(C, x, x, n, B, s);
  const bool random_start = !(nx > 0);
  if (random_start) {
    // seeded random start, weighted towards configurations with a low
    // diagonal energy: x_i = u_i / (diag_i - min(diag) + 1)
    // seeded per context: the same solve starts from the same vector whatever
    // other contexts do (results are the same alone and in a mix)
    CK(launch_random(x, n, C->cfg.seed + 7919 * (++C->start_count), s));
    std::vector<double> dh(n);
    CK(cudaMemcpyAsync(dh.data(), w.diag, 8 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double dmin = n ? *std::min_element(dh.begin(), dh.end()) : 0.0;
    double shift = dmin - 1.0;
    double *th = B.coef;
    CK(cudaMemcpyAsync(th, &shift, 8, cudaMemcpyHostToDevice, s));
    CK(launch_precond(x, w.diag, th, n, s));
    nx = dot1(C, x, x, n, B, s);
  }
  CK(cudaMemcpyAsync(B.V, x, 8 * n, cudaMemcpyDeviceToDevice, s));
  lincomb(B.V, B.V, {}, 1.0 / std::sqrt(nx), n, B, s);
  apply(C, B.V, B.AV, s, prec);
  ++nmv;
  std::vector<double> S(m * m, 0.0), col;
  dots(C, B.V, 1, n, B.AV, B, col, s);
  S[0] = col[0];
  int k = 1, it = 0;
  double theta = S[0], rnorm = 1e300, best_r = 1e300;
  int best_it = 0;
  bool probed = false, inject = false;
  double theta_probe = 0.0;
  std::vector<double> y(1, 1.0);
  bool conv = false;
  for (it = 0; it < maxit; ++it) {
    std::vector<double> Sk(k * k), ev, evec;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Sk[i * k + j] = 0.5 * (S[i * m + j] + S[j * m + i]);
    jacobi_eig(k, Sk, ev, evec);
    int imin = (int)(std::min_element(ev.begin(), ev.end()) - ev.begin());
    theta = ev[imin];
    y.assign(k, 0.0);
    for (int i = 0; i < k; ++i) y[i] = evec[i * k + imin];
    // residual r = AV y - theta V y
    std::vector<double> ny(k);
    for (int i = 0; i < k; ++i) ny[i] = -theta * y[i];
    lincomb(B.t, B.AV, y, 0.0, n, B, s);
    lincomb(B.t, B.V, ny, 1.0, n, B, s);
    rnorm = std::sqrt(std::max(0.0, dot1(C, B.t, B.t, n, B, s)));
    // The split product is accurate to ~1e-6 relative, so its residual cannot
    // fall much below that times |theta|; the reported energy is the FP64
    // Rayleigh quotient, whose error is second order in the residual.
    const double floor = prec == DMRG_SPLIT ? kSplitResidualFloor * std::max(1.0, std::fabs(theta)) : 0.0;
    // A start vector already at the floor is accepted as is.  Otherwise the
    // split path does not stop on reaching the floor: an excited state can
    // converge first from a start with little ground-state weight (early
    // windows of a sweep from a random MPS), and the ground state appears
    // only after further iterations, as it does in the FP64 path whose
    // tolerance is tighter.  It stops once the residual has stagnated.
    if (rnorm < tol || (it == 0 && rnorm < floor)) {
      conv = true;
      break;
    }
    // stagnation near the split product's noise floor: stop if the best
    // residual has not halved over the last `patience` iterations
    if (rnorm < 0.5 * best_r) {
      best_r = rnorm;
      best_it = it;
    } else if (prec == DMRG_SPLIT && it - best_it >= patience &&
               rnorm < 10.0 * std::max(tol, floor)) {
      const bool lowered = theta < theta_probe - 1e-5 * std::max(1.0, std::fabs(theta));
      if (probe && (!probed || lowered)) {
        probed = true;
        theta_probe = theta;
        inject = true;
        best_it = it;
      } else {
        conv = true;
        break;
      }
    }
    if (k == m) {
      // thick restart: keep the Ritz vectors of the lowest nk Ritz values
      const int nk = std::min(3, k);
      std::vector<int> order(k);
      std::iota(order.begin(), order.end(), 0);
      std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] < ev[b]; });
      std::vector<std::vector<double>> Y(nk, std::vector<double>(k));
      for (int r = 0; r < nk; ++r)
        for (int i = 0; i < k; ++i) Y[r][i] = evec[i * k + order[r]];
      // new V_r = V Y_r and AV_r = AV Y_r, staged through the restart scratch
      std::vector<double *> tmpv;
      for (int r = 0; r < nk; ++r) {
        double *dst = C->rs + (long long)r * n;
        lincomb(dst, B.V, Y[r], 0.0, n, B, s);
        tmpv.push_back(dst);
      }
      for (int r = 0; r < nk; ++r)
        CK(cudaMemcpyAsync(B.V + (long long)r * n, tmpv[r], 8 * n, cudaMemcpyDeviceToDevice, s));
      for (int r = 0; r < nk; ++r)
        lincomb(tmpv[r], B.AV, Y[r], 0.0, n, B, s);
      for (int r = 0; r < nk; ++r)
        CK(cudaMemcpyAsync(B.AV + (long long)r * n, tmpv[r], 8 * n, cudaMemcpyDeviceToDevice, s));
      std::fill(S.begin(), S.end(), 0.0);
      for (int r = 0; r < nk; ++r) S[r * m + r] = ev[order[r]];
      k = nk;
      y.assign(k, 0.0);
      y[0] = 1.0;
    }
    // correction vector: preconditioned residual
    double *th = B.coef + m + 1;
    CK(cudaMemcpyAsync(th, &theta, 8, cudaMemcpyHostToDevice, s));
    // The first iterations expand a plain Krylov space (t = r): it converges to
    // the extremal eigenvalue first, so the diagonal preconditioner, which
    // amplifies whatever eigenvalue theta is close to, cannot lock onto an
    // interior state from an unlucky start.
    // (a caller's start vector, e.g. the StVec guess of a sweep, is already
    // close to the ground state and is preconditioned from the first step)
    if (inject) {
      // the probe direction replaces this iteration's correction
      CK(launch_random(B.t, n, C->cfg.seed + 104729 * (++C->start_count), s));
      inject = false;
    } else if (jd_steps > 0) {
      // mixed-precision refinement: split-precision correction equation
      lincomb(B.u, B.V, y, 0.0, n, B, s);
      jd_correction(C, B, n, theta, th, jd_steps, s);
    } else if (!random_start || it >= kKrylovWarmup) {
      CK(launch_precond(B.t, w.diag, th, n, s));
    }
    // classical Gram-Schmidt, twice: t -= V (V^T t), coefficients kept on the device
    for (int pass = 0; pass < 2; ++pass) {
      CK(launch_dots(B.V, k, n, B.t, n, B.work, B.dots, s));
      CK(launch_lincomb_d(B.t, B.V, k, n, B.dots, -1.0, 1.0, n, s));
    }
    // the product is taken of the unnormalised t: its norm and the new column
    // of V^T A V come back in one transfer, and both are scaled afterwards
    double *vk = B.V + (long long)k * n;
    double *avk = B.AV + (long long)k * n;
    CK(cudaMemcpyAsync(vk, B.t, 8 * n, cudaMemcpyDeviceToDevice, s));
    apply(C, vk, avk, s, prec);
    ++nmv;
    CK(launch_dots(B.V, k + 1, n, avk, n, B.work, B.dots, s));
    CK(launch_dots(vk, 1, n, vk, n, B.work, B.dots + k + 1, s));
    col.resize(k + 2);
    CK(cudaMemcpyAsync(col.data(), B.dots, 8 * (k + 2), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double nt = std::sqrt(std::max(0.0, col[k + 1]));
    if (!(nt > 1e-14)) {
      conv = rnorm < 10 * tol;
      break;
    }
    lincomb(vk, vk, {}, 1.0 / nt, n, B, s);
    lincomb(avk, avk, {}, 1.0 / nt, n, B, s);
    for (int i = 0; i < k; ++i) col[i] /= nt;
    col[k] /= nt * nt;
    for (int i = 0; i <= k; ++i) {
      S[i * m + k] = col[i];
      S[k * m + i] = col[i];
    }
    ++k;
  }
  // Ritz vector
  lincomb(x, B.V, y, 0.0, n, B, s);
  double nn = dot1(C, x, x, n, B, s);
  lincomb(x, x, {}, 1.0 / std::sqrt(nn), n, B, s);
  *energy = theta;
  if (iters) *iters = it;
  if (rnorm_out) *rnorm_out = rnorm;
  C->prof[0] += now() - t0;
  C->prof[6] += nmv;
  return conv ? DMRG_OK : DMRG_ERR_NOT_CONVERGED;
}

// Lowest eigenpair of the window's H_eff.  The split path's residual stops
// near the split product's noise floor (about 4e-6 |theta|), above
// davidson_tol, so its result is refined by Davidson iterations with the FP64
// product started from it (mixed-precision refinement: the bulk of the
// matvecs stays split, a few FP64 ones take the residual to davidson_tol).
// The reported energy is then the Rayleigh quotient of the FP64 product, and
// the result has the FP64 path's accuracy.
int davidson(dmrg_ctx *C, double *x, double *energy, int *iters, cudaStream_t s,
             int patience = 6, bool probe = true) {
  const int prec = (C->precision == DMRG_SPLIT && C->win.flops < C->split_min_flops)
                       ? DMRG_FP64 : C->precision;
  double rn = 0;
  int it = 0;
  int rc = davidson_run(C, x, energy, &it, s, prec, patience, probe, &rn);
  if (prec == DMRG_SPLIT) {
    check_err_flag(C, s);
    int it2 = 0;
    const int jd = C->win.flops >= C->refine_min_flops ? C->refine_steps : 0;
    rc = davidson_run(C, x, energy, &it2, s, DMRG_FP64, patience, false, &rn, jd);
    it += it2;
  }
  if (iters) *iters = it;
  return rc;
}

// ---------------------------------------------------------------------------
// truncation: reduced density matrix per sector, cuSOLVER eigensolver
// ---------------------------------------------------------------------------
void truncate(dmrg_ctx *C, const double *psi, int side, int D, double *disc, double *ent,
              cudaStream_t s) {
  Window &w = C->win;
  double t0 = now();
  if (!C->solver) {
    if (cusolverDnCreate(&C->solver) != CUSOLVER_STATUS_SUCCESS) fail(DMRG_ERR_CUDA, "cusolverDnCreate failed");
  }
  cusolverDnSetStream(C->solver, s);
  const size_t np = w.psi.size();
  // Blocks up to 256 are padded to a power of two and solved in batches
  // (cusolverDnXsyevBatched) with -1 on the padded diagonal: rho is positive
  // semi-definite, so the padding eigenpairs separate exactly and come first
  // in ascending order.  Larger blocks use syevd one by one.
  std::vector<int> dim(np), npad(np);
  std::vector<long long> roff(np), eoff(np);
  std::map<int, std::vector<int>> bucket;
  for (size_t i = 0; i < np; ++i) {
    dim[i] = side == 0 ? w.psi[i].da : w.psi[i].db;
    int q = 8;
    while (q < dim[i]) q <<= 1;
    npad[i] = dim[i] <= 256 ? q : dim[i];
    bucket[npad[i] <= 256 ? npad[i] : -(int)i - 1].push_back((int)i);
  }
  long long tot = 0, eo = 0;
  for (auto &kv : bucket)
    for (int i : kv.second) {
      roff[i] = tot;
      tot += (long long)npad[i] * npad[i];
      eoff[i] = eo;
      eo += npad[i];
    }
  WinBuf tmp(s);
  double *rho = (double *)tmp.alloc(8 * std::max<long long>(tot, 1));
  double *eval = (double *)tmp.alloc(8 * std::max<long long>(eo, 1));
  CK(cudaMemsetAsync(rho, 0, 8 * std::max<long long>(tot, 1), s));
  std::vector<GemmDesc> dd;
  std::vector<GemmSeg> gg;
  std::vector<SCopy> pads;
  long long tt = 0;
  for (size_t i = 0; i < np; ++i) {
    const PsiBlk &p = w.psi[i];
    GemmSeg g;
    memset(&g, 0, sizeof g);
    g.A = psi + p.off;
    g.B = psi + p.off;
    if (side == 0) {
      g.a_rs = p.db; g.a_cs = 1; g.b_rs = 1; g.b_cs = p.db; g.K = p.db;
    } else {
      g.a_rs = 1; g.a_cs = p.db; g.b_rs = p.db; g.b_cs = 1; g.K = p.da;
    }
    GemmDesc d;
    memset(&d, 0, sizeof d);
    d.C = rho + roff[i];
    d.c_rs = npad[i]; d.c_cs = 1;
    d.M = dim[i]; d.N = dim[i]; d.batch = 1;
    d.seg0 = (int)gg.size(); d.nseg = 1;
    d.tiles_m = (dim[i] + 63) / 64; d.tiles_n = d.tiles_m;
    d.alpha = 1.0; d.beta = 0.0;
    d.tile0 = tt;
    tt += (long long)d.tiles_m * d.tiles_n;
    gg.push_back(g);
    dd.push_back(d);
    if (npad[i] > dim[i]) {
      SCopy c;
      memset(&c, 0, sizeof c);
      c.src = nullptr;
      c.ident = 1;
      c.coef = -1.0;
      c.rows = c.cols = npad[i] - dim[i];
      c.dst = rho + roff[i] + (long long)dim[i] * npad[i] + dim[i];
      c.dst_ld = npad[i];
      pads.push_back(c);
    }
  }
  {
    GemmDesc *a = upload(tmp, dd, s);
    GemmSeg *b = upload(tmp, gg, s);
    CK(launch_gemm_f64(a, (int)dd.size(), b, tt, s));
    if (!pads.empty()) {
      SCopy *c = upload(tmp, pads, s);
      CK(launch_stack_copy(c, (int)pads.size(), s));
    }
  }
  if (!C->solver_params) {
    if (cusolverDnCreateParams(&C->solver_params) != CUSOLVER_STATUS_SUCCESS)
      fail(DMRG_ERR_CUDA, "cusolverDnCreateParams failed");
  }
  int *info = (int *)tmp.alloc(sizeof(int) * np);
  int info_off = 0;
  std::vector<int> info_of(np);
  std::list<std::vector<char>> hwork;   // cuSOLVER host workspaces (stable addresses)
  for (auto &kv : bucket) {
    const std::vector<int> &ids = kv.second;
    const int first = ids[0];
    const int64_t n = npad[first];
    if (kv.first > 0) {
      size_t dws = 0, hws = 0;
      if (cusolverDnXsyevBatched_bufferSize(C->solver, C->solver_params, CUSOLVER_EIG_MODE_VECTOR,
                                            CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, rho + roff[first],
                                            n, CUDA_R_64F, eval + eoff[first], CUDA_R_64F, &dws,
                                            &hws, (int64_t)ids.size()) != CUSOLVER_STATUS_SUCCESS)
        fail(DMRG_ERR_CUDA, "syevBatched bufferSize failed");
      void *dw = tmp.alloc(std::max<size_t>(dws, 8));
      // host workspaces stay alive until the stream synchronisation below,
      // so the buckets' solves are queued back to back
      hwork.emplace_back(std::max<size_t>(hws, 8));
      std::vector<char> &hw = hwork.back();
      if (cusolverDnXsyevBatched(C->solver, C->solver_params, CUSOLVER_EIG_MODE_VECTOR,
                                 CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, rho + roff[first], n,
                                 CUDA_R_64F, eval + eoff[first], CUDA_R_64F, dw, dws, hw.data(), hws,
                                 info + info_off, (int64_t)ids.size()) != CUSOLVER_STATUS_SUCCESS)
        fail(DMRG_ERR_CUDA, "syevBatched failed");
      for (size_t j = 0; j < ids.size(); ++j) info_of[ids[j]] = info_off + (int)j;
      info_off += (int)ids.size();
    } else {
      int lw = 0;
      if (cusolverDnDsyevd_bufferSize(C->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                      (int)n, rho + roff[first], (int)n, eval + eoff[first], &lw) !=
          CUSOLVER_STATUS_SUCCESS)
        fail(DMRG_ERR_CUDA, "syevd bufferSize failed");
      double *wk = (double *)tmp.alloc(8 * (size_t)std::max(lw, 1));
      if (cusolverDnDsyevd(C->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)n,
                           rho + roff[first], (int)n, eval + eoff[first], wk, lw, info + info_off) !=
          CUSOLVER_STATUS_SUCCESS)
        fail(DMRG_ERR_CUDA, "syevd failed");
      info_of[first] = info_off++;
    }
  }
  std::vector<double> evp(eo);
  std::vector<int> hinfo(std::max(info_off, 1));
  CK(cudaMemcpyAsync(evp.data(), eval, 8 * eo, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * info_off, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < info_off; ++i)
    if (hinfo[i] != 0) fail(DMRG_ERR_CUDA, "eigensolver info %d", hinfo[i]);
  // genuine eigenvalues of block i: the last dim[i] of its npad[i] (ascending)
  std::vector<double> ev(eo, 0.0);
  for (size_t i = 0; i < np; ++i)
    for (int k = 0; k < dim[i]; ++k) ev[eoff[i] + k] = evp[eoff[i] + npad[i] - dim[i] + k];
  // candidates: (-weight, sector, position in descending order)
  struct Cand {
    double v;
    int sec, k;
  };
  std::vector<Cand> cand;
  for (size_t i = 0; i < np; ++i)
    for (int k = 0; k < dim[i]; ++k) cand.push_back({std::max(0.0, ev[eoff[i] + dim[i] - 1 - k]), (int)i, k});
  std::sort(cand.begin(), cand.end(), [](const Cand &a, const Cand &b) {
    if (a.v != b.v) return a.v > b.v;
    if (a.sec != b.sec) return a.sec < b.sec;
    return a.k < b.k;
  });
  const size_t keep = std::min<size_t>(D, cand.size());
  double wk_tot = 0, wk_keep = 0;
  for (auto &c : cand) wk_tot += c.v;
  std::vector<std::vector<int>> kept(np);
  for (size_t j = 0; j < keep; ++j) {
    kept[cand[j].sec].push_back(cand[j].k);
    wk_keep += cand[j].v;
  }
  double e = 0;
  for (size_t j = 0; j < keep; ++j) {
    double pj = cand[j].v / std::max(wk_keep, 1e-300);
    if (pj > 0) e -= pj * std::log(pj);
    // a kept multiplet of spin j carries its weight in 2j+1 equal Schmidt values
    if (C->su2 && pj > 0) {
      const QN q = side == 0 ? w.Ld.basis.qn[w.psi[cand[j].sec].a] : w.Rd.basis.qn[w.psi[cand[j].sec].b];
      e += pj * std::log(su2::tj_of(q) + 1.0);
    }
  }
  if (disc) *disc = wk_tot - wk_keep;
  if (ent) *ent = e;
  // isometry, sectors in ascending QN order of the new block
  std::vector<std::pair<QN, int>> order;
  for (size_t i = 0; i < np; ++i)
    if (!kept[i].empty()) {
      QN q = side == 0 ? w.Ld.basis.qn[w.psi[i].a] : w.Rd.basis.qn[w.psi[i].b];
      order.push_back({q, (int)i});
    }
  std::sort(order.begin(), order.end());
  Iso T;
  long long off = 0;
  for (auto &o : order) {
    std::sort(kept[o.second].begin(), kept[o.second].end());
    T.qn.push_back(o.first);
    T.rows.push_back(dim[o.second]);
    T.cols.push_back((int)kept[o.second].size());
    T.off.push_back(off);
    off += (long long)dim[o.second] * kept[o.second].size();
  }
  std::unique_ptr<BlockPart> Bn(new BlockPart());
  WinBuf &bb = buf_of(C, Bn.get());
  T.d = (double *)bb.alloc(8 * std::max<long long>(off, 1));
  // the kept columns of all sectors in one upload
  std::vector<int> colsel, coff;
  for (size_t j = 0; j < order.size(); ++j) {
    coff.push_back((int)colsel.size());
    for (int k : kept[order[j].second]) colsel.push_back(npad[order[j].second] - 1 - k);
  }
  int *dcs = upload(tmp, colsel, s);
  for (size_t j = 0; j < order.size(); ++j) {
    int i = order[j].second;
    CK(launch_select_cols(rho + roff[i], npad[i], dim[i], dcs + coff[j], (int)kept[i].size(),
                          T.d + T.off[j], s));
  }
  CK(cudaStreamSynchronize(s));
  C->prof[3] += now() - t0;
  t0 = now();
  cudaStream_t save = C->stream;
  C->stream = s;
  if (side == 0) {
    renormalize(C, w.Ld, T, *Bn, bb);
    int n = w.l + 1;
    if ((int)C->L.size() <= n) C->L.resize(n + 1);
    if (C->L[n]) free_part(C, C->L[n].get());
    C->L[n] = std::move(Bn);
    C->Lmap[n] = T;
  } else {
    renormalize(C, w.Rd, T, *Bn, bb);
    int n = w.l + 1;
    if (C->R.count(n)) free_part(C, C->R[n].get());
    C->R[n] = std::move(Bn);
    C->Rmap[n] = T;
  }
  C->stream = save;
  C->prof[1] += now() - t0;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// StVec: carry the converged psi of one window over to the next (a8)
// ---------------------------------------------------------------------------
struct WinMeta {
  int l = -1;
  std::vector<PsiBlk> psi;
  Basis Lb, Rb;
  std::vector<std::vector<Piece>> Lp, Rp;
};

WinMeta meta_of(const Window &w) {
  WinMeta m;
  m.l = w.l;
  m.psi = w.psi;
  m.Lb = w.Ld.basis;
  m.Rb = w.Rd.basis;
  m.Lp = w.Ld.pieces;
  m.Rp = w.Rd.pieces;
  return m;
}

int iso_find(const Iso &T, const QN &q) {
  for (size_t i = 0; i < T.qn.size(); ++i)
    if (T.qn[i] == q) return (int)i;
  return -1;
}

void push_gemm(std::vector<GemmDesc> &dd, std::vector<GemmSeg> &gg, long long &tt, double *Cp,
               long long c_rs, int M, int N, int K, const double *A, long long a_rs,
               long long a_cs, const double *Bp, long long b_rs, long long b_cs,
               double alpha = 1.0) {
  if (M <= 0 || N <= 0) return;
  GemmSeg g;
  memset(&g, 0, sizeof g);
  g.A = A; g.a_rs = a_rs; g.a_cs = a_cs;
  g.B = Bp; g.b_rs = b_rs; g.b_cs = b_cs;
  g.K = K;
  GemmDesc d;
  memset(&d, 0, sizeof d);
  d.C = Cp; d.c_rs = c_rs; d.c_cs = 1;
  d.M = M; d.N = N; d.batch = 1;
  d.seg0 = (int)gg.size(); d.nseg = 1;
  d.tiles_m = (M + 63) / 64; d.tiles_n = (N + 63) / 64;
  d.alpha = alpha; d.beta = 0.0;
  d.tile0 = tt;
  tt += (long long)d.tiles_m * d.tiles_n;
  gg.push_back(g);
  dd.push_back(d);
}

void run_gemms(std::vector<GemmDesc> &dd, std::vector<GemmSeg> &gg, long long tt, cudaStream_t s) {
  if (dd.empty()) return;
  WinBuf tmp(s);
  GemmDesc *a = upload(tmp, dd, s);
  GemmSeg *b = upload(tmp, gg, s);
  CK(launch_gemm_f64(a, (int)dd.size(), b, tt, s));
  CK(cudaStreamSynchronize(s));
}

// side 0: old window l was truncated to the left (L_{l+1} = U^T L.); the guess
// for window l+1 is psi'[(l', s1), (s2, r')] = sum_r (U^T psi)[l', (s1, r)] TR[(s2, r'), r]
// with TR the isometry of R_{l+2}.  side 1 mirrors it with V (R_{l+1}) and TL
// (the isometry of L_l).  Spin-adapted windows also recouple the three spins
// of L, the moved site and R: |(L (s R) b) S> -> |((L s) a R) S> with the
// coefficient <((L s) a R) S | (L (s R) b) S> (and its transpose for side 1).
inline int site_tj(int k) { return k == 1 ? 1 : 0; }   // spin-adapted site multiplets
void stvec(dmrg_ctx *C, const WinMeta &old, const double *psi_old, int side, double *psi_new,
           cudaStream_t s) {
  Window &w = C->win;
  double t0 = now();
  CK(cudaMemsetAsync(psi_new, 0, 8 * std::max<long long>(w.psi_len, 1), s));
  WinBuf tmp(s);
  std::vector<GemmDesc> dd;
  std::vector<GemmSeg> gg;
  long long tt = 0;
  std::map<int, int> a2p, b2p;
  for (size_t i = 0; i < old.psi.size(); ++i) {
    a2p[old.psi[i].a] = (int)i;
    b2p[old.psi[i].b] = (int)i;
  }
  if (side == 0) {
    const Iso &U = C->Lmap.at(old.l + 1);
    const Iso &TR = C->Rmap.at(old.l + 2);
    std::vector<long long> xo(old.psi.size(), -1);
    std::vector<int> kx(old.psi.size(), 0);
    long long nx = 0;
    for (size_t i = 0; i < old.psi.size(); ++i) {
      int ui = iso_find(U, old.Lb.qn[old.psi[i].a]);
      if (ui < 0) continue;
      xo[i] = nx;
      kx[i] = U.cols[ui];
      nx += (long long)kx[i] * old.psi[i].db;
    }
    double *X = (double *)tmp.alloc(8 * std::max<long long>(nx, 1));
    for (size_t i = 0; i < old.psi.size(); ++i) {
      if (xo[i] < 0) continue;
      const PsiBlk &p = old.psi[i];
      int ui = iso_find(U, old.Lb.qn[p.a]);
      push_gemm(dd, gg, tt, X + xo[i], p.db, kx[i], p.db, p.da, U.d + U.off[ui], 1, kx[i],
                psi_old + p.off, p.db, 1);
    }
    run_gemms(dd, gg, tt, s);
    dd.clear();
    gg.clear();
    tt = 0;
    const BlockPart &Lnew = *C->L[old.l + 1];
    const BlockPart &R2 = *C->R[old.l + 2];
    for (const PsiBlk &P : w.psi) {
      const int dB = w.Rd.basis.dim[P.b];
      for (const Piece &pc : w.Ld.pieces[P.a]) {
        int ia = old.Lb.find(Lnew.basis.qn[pc.blk_sector]);
        if (ia < 0 || !a2p.count(ia)) continue;
        int pi = a2p[ia];
        if (xo[pi] < 0) continue;
        const PsiBlk &p = old.psi[pi];
        const Piece *rp = nullptr;
        for (const Piece &q : old.Rp[p.b])
          if (q.site_state == pc.site_state &&
              (!C->su2 || R2.basis.qn[q.blk_sector] == w.Rd.basis.qn[P.b]))
            rp = &q;
        if (!rp) continue;
        const QN qr = R2.basis.qn[rp->blk_sector];
        if (qr != w.Rd.basis.qn[P.b]) continue;
        int ti = iso_find(TR, qr);
        if (ti < 0 || TR.rows[ti] != dB) continue;
        double f = 1.0;
        if (C->su2)
          f = su2::recouple(su2::tj_of(Lnew.basis.qn[pc.blk_sector]), site_tj(pc.site_state),
                            su2::tj_of(qr), su2::tj_of(w.Ld.basis.qn[P.a]), su2::tj_of(old.Rb.qn[p.b]),
                            su2::tj_of(C->target));
        push_gemm(dd, gg, tt, psi_new + P.off + (long long)pc.off * dB, dB, pc.dim, dB, rp->dim,
                  X + xo[pi] + rp->off, p.db, 1, TR.d + TR.off[ti], 1, TR.cols[ti], f);
      }
    }
    run_gemms(dd, gg, tt, s);
  } else {
    const Iso &V = C->Rmap.at(old.l + 1);
    const Iso &TL = C->Lmap.at(old.l);
    std::vector<long long> yo(old.psi.size(), -1);
    std::vector<int> ky(old.psi.size(), 0);
    long long ny = 0;
    for (size_t i = 0; i < old.psi.size(); ++i) {
      int vi = iso_find(V, old.Rb.qn[old.psi[i].b]);
      if (vi < 0) continue;
      yo[i] = ny;
      ky[i] = V.cols[vi];
      ny += (long long)old.psi[i].da * ky[i];
    }
    double *Y = (double *)tmp.alloc(8 * std::max<long long>(ny, 1));
    for (size_t i = 0; i < old.psi.size(); ++i) {
      if (yo[i] < 0) continue;
      const PsiBlk &p = old.psi[i];
      int vi = iso_find(V, old.Rb.qn[p.b]);
      push_gemm(dd, gg, tt, Y + yo[i], ky[i], p.da, ky[i], p.db, psi_old + p.off, p.db, 1,
                V.d + V.off[vi], ky[i], 1);
    }
    run_gemms(dd, gg, tt, s);
    dd.clear();
    gg.clear();
    tt = 0;
    const BlockPart &Rnew = *C->R[old.l + 1];
    for (const PsiBlk &P : w.psi) {
      const int dA = w.Ld.basis.dim[P.a];
      const int dB = w.Rd.basis.dim[P.b];
      const QN qA = w.Ld.basis.qn[P.a];
      int ti = iso_find(TL, qA);
      if (ti < 0 || TL.rows[ti] != dA) continue;
      for (const Piece &pc : w.Rd.pieces[P.b]) {
        // old L. sector holding (site state, L_l sector with QN qA): spin-
        // adapted, the one whose spin pairs with the R_{l+1} sector's
        const QN qR = Rnew.basis.qn[pc.blk_sector];
        const QN qa_old = C->su2 ? su2::label(su2::n_of(qA) + (pc.site_state == 0 ? 0 : pc.site_state == 1 ? 1 : 2),
                                              su2::tj_of(qR))
                                 : qadd(qA, qsub(w.Rd.basis.qn[P.b], qR));
        int ia = old.Lb.find(qa_old);
        if (ia < 0 || !a2p.count(ia)) continue;
        int pi = a2p[ia];
        if (yo[pi] < 0) continue;
        const PsiBlk &p = old.psi[pi];
        const Piece *lp = nullptr;
        for (const Piece &q : old.Lp[p.a])
          if (q.site_state == pc.site_state && C->L[old.l]->basis.qn[q.blk_sector] == qA) lp = &q;
        if (!lp) continue;
        if (ky[pi] != pc.dim) continue;
        double f = 1.0;
        if (C->su2)
          f = su2::recouple(su2::tj_of(qA), site_tj(pc.site_state), su2::tj_of(qR), su2::tj_of(qa_old),
                            su2::tj_of(w.Rd.basis.qn[P.b]), su2::tj_of(C->target));
        push_gemm(dd, gg, tt, psi_new + P.off + pc.off, dB, dA, pc.dim, lp->dim,
                  TL.d + TL.off[ti], TL.cols[ti], 1, Y + yo[pi] + (long long)lp->off * ky[pi],
                  ky[pi], 1, f);
      }
    }
    run_gemms(dd, gg, tt, s);
  }
  C->prof[4] += now() - t0;
}

// ---------------------------------------------------------------------------
// one-particle reduced density matrix at the window (Sec. II.B, III.C)
// ---------------------------------------------------------------------------
// gamma_ij = <c+_j c_i> = <c_j psi | c_i psi>: with w_k = c_k psi for every
// mode k of the window (block products with the window's operators, in the
// layout of the state space with one particle fewer), gamma = W W^T.
// Spin-adapted: w_k = c~_k psi is a spin-1/2 state; its reduced coefficients
// on the coupled pairs (a', b') carry the recoupling of [c~ (x) 1]^(1/2) (or
// [1 (x) c~]^(1/2)) from the S = 0 window, and the spin-summed
// gamma_ij = sum_sigma <c+_{j sigma} c_{i sigma}> = 2 w_j . w_i.
// Output: spatial, spin-summed, in the rotated mode basis, gamma[i*N + j].
void rdm1(dmrg_ctx *C, const double *psi, double *gamma, cudaStream_t s) {
  Window &w = C->win;
  const int N = C->N;
  std::fill(gamma, gamma + (size_t)N * N, 0.0);
  struct ModeOp {
    int row;       // row of W
    int spatial;   // output index
    bool left;     // mode of L. (else .R)
    const BlockPart *P;
    std::vector<Ref> comps;
  };
  // classes of modes whose annihilators share one target layout
  std::vector<std::vector<ModeOp>> classes;
  if (C->su2) {
    std::vector<ModeOp> v;
    for (int side = 0; side < 2; ++side) {
      const BlockPart &P = side == 0 ? w.Ld : w.Rd;
      std::vector<int> sp;
      for (int p : P.modes)
        if (!has(sp, p >> 1)) sp.push_back(p >> 1);
      for (int x : sp) {
        auto it = P.ten.find(TKey{1, x, 0, 1});
        if (it == P.ten.end()) continue;
        ModeOp m{(int)v.size(), x, side == 0, &P, {}};
        for (const Ref &r : it->second.r)
          if (r.cls >= 0) m.comps.push_back(r);
        v.push_back(m);
      }
    }
    classes.push_back(v);
  } else {
    const int ncls = C->spinful ? 2 : 1;
    classes.resize(ncls);
    for (int side = 0; side < 2; ++side) {
      const BlockPart &P = side == 0 ? w.Ld : w.Rd;
      for (int p : P.modes) {
        auto it = P.c.find(p);
        if (it == P.c.end() || it->second.cls < 0) continue;
        auto &v = classes[C->spinful ? (p & 1) : 0];
        v.push_back(ModeOp{(int)v.size(), C->spinful ? p >> 1 : p, side == 0, &P, {it->second}});
      }
    }
  }
  const int tS = su2::tj_of(C->target);
  WinBuf tmp(s);
  for (auto &modes : classes) {
    if (modes.empty()) continue;
    // target layout: every (a', b') some w_k reaches
    std::map<std::pair<int, int>, long long> off;
    struct Job {
      const ModeOp *m;
      const PsiBlk *p;
      int ao, bo;
      const double *blk;
      int ld;
      double coef;
    };
    std::vector<Job> jobs;
    for (const ModeOp &m : modes)
      for (const Ref &r : m.comps) {
        const OpClass &oc = m.P->cls[r.cls];
        for (const PsiBlk &p : w.psi) {
          const int in = m.left ? p.a : p.b;
          const int b = oc.in2blk[in];
          if (b < 0) continue;
          const int out = oc.blk_out[b];
          const int ao = m.left ? out : p.a, bo = m.left ? p.b : out;
          double coef = 1.0;
          if (!m.left && (qnum(w.Ld.basis.qn[p.a]) & 1)) coef = -1.0;   // c on .R passes L.'s particles
          if (C->su2) {
            const int ja = su2::tj_of(w.Ld.basis.qn[p.a]), jb = su2::tj_of(w.Rd.basis.qn[p.b]);
            const int jao = su2::tj_of(w.Ld.basis.qn[ao]), jbo = su2::tj_of(w.Rd.basis.qn[bo]);
            coef *= m.left ? su2::coupling(ja, jb, tS, jao, jbo, 1, 1, 0, 1)
                           : su2::coupling(ja, jb, tS, jao, jbo, 1, 0, 1, 1);
            if (coef == 0.0) continue;
          }
          const std::pair<int, int> key{ao, bo};
          if (!off.count(key)) {
            off[key] = 0;
          }
          jobs.push_back({&m, &p, ao, bo, oc.d + (long long)r.idx * oc.nnz + oc.blk_off[b],
                          m.left ? p.da : p.db, coef});
        }
      }
    long long len = 0;
    for (auto &kv : off) {
      kv.second = len;
      len += (long long)w.Ld.basis.dim[kv.first.first] * w.Rd.basis.dim[kv.first.second];
    }
    const int nm = (int)modes.size();
    double *W = (double *)tmp.alloc(8 * std::max<long long>(1, (long long)nm * len));
    CK(cudaMemsetAsync(W, 0, 8 * std::max<long long>(1, (long long)nm * len), s));
    std::vector<GemmDesc> dd;
    std::vector<GemmSeg> gg;
    long long tt = 0;
    // blocks reached by several components of one mode accumulate (beta = 1)
    for (const Job &j : jobs) {
      const int dao = w.Ld.basis.dim[j.ao], dbo = w.Rd.basis.dim[j.bo];
      double *dst = W + (long long)j.m->row * len + off[{j.ao, j.bo}];
      const double *ps = psi + j.p->off;
      if (j.m->left)   // (dao x da) . (da x db)
        push_gemm(dd, gg, tt, dst, dbo, dao, dbo, j.p->da, j.blk, j.ld, 1, ps, j.p->db, 1, j.coef);
      else             // (da x db) . (dbo x db)^T
        push_gemm(dd, gg, tt, dst, dbo, dao, dbo, j.p->db, ps, j.p->db, 1, j.blk, 1, j.ld, j.coef);
      dd.back().beta = 1.0;
    }
    // the beta = 1 accumulation needs the descriptors of one output block in
    // order: run them in separate launches per component index
    {
      std::vector<GemmDesc> d1;
      std::vector<GemmSeg> g1;
      long long t1 = 0;
      std::map<double *, int> seen;
      std::vector<std::pair<GemmDesc, GemmSeg>> later;
      for (size_t i = 0; i < dd.size(); ++i) {
        if (seen[dd[i].C]++) {
          later.push_back({dd[i], gg[dd[i].seg0]});
          continue;
        }
        GemmDesc d = dd[i];
        d.seg0 = (int)g1.size();
        d.tile0 = t1;
        t1 += (long long)d.tiles_m * d.tiles_n;
        g1.push_back(gg[dd[i].seg0]);
        d1.push_back(d);
      }
      run_gemms(d1, g1, t1, s);
      for (auto &pr : later) {
        std::vector<GemmDesc> d2{pr.first};
        std::vector<GemmSeg> g2{pr.second};
        d2[0].seg0 = 0;
        d2[0].tile0 = 0;
        run_gemms(d2, g2, (long long)d2[0].tiles_m * d2[0].tiles_n, s);
      }
    }
    // G = W W^T, split over K ranges, partials summed in a fixed order
    const long long KS = 16384;
    const int nparts = (int)std::max<long long>(1, (len + KS - 1) / KS);
    double *ws = (double *)tmp.alloc(8 * (size_t)nparts * nm * nm);
    double *G = (double *)tmp.alloc(8 * (size_t)nm * nm);
    dd.clear();
    gg.clear();
    tt = 0;
    for (int pch = 0; pch < nparts; ++pch) {
      const long long k0 = (long long)pch * KS, kl = std::min(KS, len - k0);
      push_gemm(dd, gg, tt, ws + (size_t)pch * nm * nm, nm, nm, nm, (int)std::max<long long>(kl, 0),
                W + k0, len, 1, W + k0, 1, len);
    }
    run_gemms(dd, gg, tt, s);
    PartialSum64 ps;
    ps.ws = ws;
    ps.stride = (long long)nm * nm;
    ps.off = 0;
    ps.n = nm * nm;
    ps.nparts = nparts;
    std::vector<PartialSum64> psv{ps};
    PartialSum64 *dps = upload(tmp, psv, s);
    CK(launch_sum_partials64(dps, 1, G, s));
    std::vector<double> Gh((size_t)nm * nm);
    CK(cudaMemcpyAsync(Gh.data(), G, 8 * Gh.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double f = C->su2 ? 2.0 : 1.0;
    for (const ModeOp &a : modes)
      for (const ModeOp &b : modes)   // gamma_ij = w_j . w_i, modes on opposite sides
        if (a.left != b.left) gamma[(size_t)a.spatial * N + b.spatial] += f * Gh[(size_t)b.row * nm + a.row];
  }
  // Two modes of one side: the renormalized single operators of a block are
  // projections, so <c_j psi | c_i psi> would miss the part of c_i psi outside
  // the kept basis; the pair operator c+_j c_i renormalized as a whole gives
  // the exact value, <psi| O (x) 1 |psi> = <O, rho_L.> with rho_L. = psi psi^T
  // per sector (.R: psi^T psi).  Spin-adapted: E_ji = -sqrt(2) B^0_ji.
  for (int side = 0; side < 2; ++side) {
    const BlockPart &P = side == 0 ? w.Ld : w.Rd;
    int c0 = -1;
    for (size_t c = 0; c < P.cls.size(); ++c)
      if (P.cls[c].shift == QN{0, 0} && P.cls[c].nnz > 0) c0 = (int)c;
    if (c0 < 0) continue;
    const OpClass &oc = P.cls[c0];
    double *rho = (double *)tmp.alloc(8 * std::max<long long>(1, oc.nnz));
    CK(cudaMemsetAsync(rho, 0, 8 * std::max<long long>(1, oc.nnz), s));
    std::vector<GemmDesc> dd;
    std::vector<GemmSeg> gg;
    long long tt = 0;
    for (size_t b = 0; b < oc.blk_in.size(); ++b) {
      const int sec = oc.blk_in[b];
      for (const PsiBlk &p : w.psi) {
        if ((side == 0 ? p.a : p.b) != sec) continue;
        double *dst = rho + oc.blk_off[b];
        const double *ps = psi + p.off;
        if (side == 0)   // psi psi^T (da x da)
          push_gemm(dd, gg, tt, dst, p.da, p.da, p.da, p.db, ps, p.db, 1, ps, 1, p.db);
        else             // psi^T psi (db x db)
          push_gemm(dd, gg, tt, dst, p.db, p.db, p.db, p.da, ps, 1, p.db, ps, p.db, 1);
      }
    }
    run_gemms(dd, gg, tt, s);
    // <O_k, rho> for every operator k of the class: (nops x nnz) . (nnz)
    double *vals = (double *)tmp.alloc(8 * std::max(1, oc.nops));
    dd.clear();
    gg.clear();
    tt = 0;
    push_gemm(dd, gg, tt, vals, 1, oc.nops, 1, (int)oc.nnz, oc.d, oc.nnz, 1, rho, 1, 0);
    run_gemms(dd, gg, tt, s);
    std::vector<double> vh(oc.nops);
    CK(cudaMemcpyAsync(vh.data(), vals, 8 * vh.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int> sp;
    for (int p : P.modes)
      if (!has(sp, C->spinful ? p >> 1 : p)) sp.push_back(C->spinful ? p >> 1 : p);
    auto val = [&](const Ref &r) { return (r.cls == c0) ? vh[r.idx] : 0.0; };
    for (int j : sp)
      for (int i : sp) {
        double g = 0.0;
        if (C->su2) {
          auto it = P.ten.find(TKey{4, j, i, 0});
          if (it != P.ten.end()) g = -std::sqrt(2.0) * val(it->second.r[0]);
        } else {
          for (int sgm = 0; sgm < (C->spinful ? 2 : 1); ++sgm) {
            const int pj = C->spinful ? 2 * j + sgm : j, pi = C->spinful ? 2 * i + sgm : i;
            auto it = P.cdc.find({pj, pi});
            if (it != P.cdc.end()) g += val(it->second);
          }
        }
        gamma[(size_t)i * N + j] = g;   // gamma_ij = <c+_j c_i>
      }
  }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {

int guard(dmrg_ctx *C, const std::function<void()> &f) {
  try {
    f();
    if (C) C->err.clear();
    return DMRG_OK;
  } catch (const Err &e) {
    if (C) C->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    if (C) C->err = "host allocation failed";
    return DMRG_ERR_OOM;
  }
}

void sweep_impl(dmrg_ctx *C, int nsw, const int *dsched, double *E, cudaStream_t s) {
  const int N = C->N;
  if (!C->ham) fail(DMRG_ERR_STATE, "dmrg_set_hamiltonian first");
  for (int n = 1; n <= N - 1; ++n)
    if (!C->riso.count(n)) fail(DMRG_ERR_STATE, "right isometry %d missing", n);
  C->stream = s;
  for (double &p : C->prof) p = 0;
  C->unconverged = 0;
  C->swept = false;
  C->center_l = -1;
  C->center_psi.clear();
  double t0 = now();
  clear_blocks(C);
  C->R[N] = vacuum(C);
  for (int n = N - 1; n >= 2; --n) {
    upload_iso(C, C->riso[n]);
    grow_right(C, n, C->riso[n]);
    // under a budget, the blocks used last in the first pass go to host memory
    if (C->cfg.hbm_budget_bytes) stage_window(C, 0, 0);
  }
  C->L.push_back(vacuum(C));
  C->prof[1] += now() - t0;
  C->Lmap.clear();
  C->Rmap.clear();
  for (int n = 2; n <= N - 1; ++n) C->Rmap[n] = C->riso[n];
  WinBuf xb[2] = {WinBuf(s), WinBuf(s)};
  int cur = 0;
  double *prev = nullptr;
  WinMeta pm;
  int prev_trunc = -1;   // -1 none, 0 left, 1 right, 2 same window follows
  double e = 0;
  int it;
  int patience = 6;
  bool probe = true;
  auto step = [&](int pass, int l, int trunc_side, int D) {
    stage_window(C, pass, l);
    build_window(C, l);
    const long long n = C->win.psi_len;
    xb[cur].clear();
    double *x = (double *)xb[cur].alloc(8 * std::max<long long>(n, 1));
    if (prev && prev_trunc == 2 && pm.l == l) {
      CK(cudaMemcpyAsync(x, prev, 8 * n, cudaMemcpyDeviceToDevice, s));
    } else if (prev && (prev_trunc == 0 || prev_trunc == 1)) {
      stvec(C, pm, prev, prev_trunc, x, s);
    } else {
      CK(cudaMemsetAsync(x, 0, 8 * std::max<long long>(n, 1), s));
    }
    if (davidson(C, x, &e, &it, s, patience, probe) == DMRG_ERR_NOT_CONVERGED) ++C->unconverged;
    pm = meta_of(C->win);
    if (trunc_side >= 0) truncate(C, x, trunc_side, D, nullptr, nullptr, s);
    prev = x;
    prev_trunc = trunc_side >= 0 ? trunc_side : 2;
    cur ^= 1;
  };
  for (int sw = 0; sw < nsw; ++sw) {
    const int D = dsched ? dsched[sw] : C->cfg.d_max;
    // the first sweep starts from a random MPS: an excited state of an early
    // window can reach the noise floor before the ground state shows up, so
    // the split Davidson probes with a random direction before it accepts
    // stagnation there; later sweeps start from the transformed previous state
    probe = sw == 0;
    patience = sw == 0 ? 6 : 4;
    for (int l = 0; l <= N - 2; ++l) step(0, l, l < N - 2 ? 0 : -1, D);
    for (int l = N - 2; l >= 0; --l) step(1, l, l > 0 ? 1 : -1, D);
    if (E) E[sw] = e;
  }
  // the MPS the sweeps ended with: right isometries R_2..R_{N-1} (Rmap) and
  // the normalized two-site center tensor of window 0
  C->swept = true;
  C->center_l = C->win.l;
  C->center_psi.resize(C->win.psi_len);
  if (prev && C->win.psi_len)
    CK(cudaMemcpyAsync(C->center_psi.data(), prev, 8 * C->win.psi_len, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  C->prof[5] = std::max(0.0, now() - t0 - C->prof[0] - C->prof[1] - C->prof[2] - C->prof[3] - C->prof[4]);
  if (C->unconverged)
    fail(DMRG_ERR_NOT_CONVERGED, "%d window solve(s) of the sweeps hit the Davidson iteration limit "
         "(energies are still written)", C->unconverged);
}

}  // namespace

extern "C" {

const char *dmrg_error_string(int code) {
  switch (code) {
    case DMRG_OK: return "ok";
    case DMRG_ERR_ARG: return "invalid argument";
    case DMRG_ERR_OOM: return "out of memory";
    case DMRG_ERR_CUDA: return "CUDA error";
    case DMRG_ERR_STATE: return "call out of order";
    case DMRG_ERR_TIMEOUT: return "bounded device wait gave up";
    case DMRG_ERR_NOT_CONVERGED: return "Davidson not converged";
    default: return "unknown error";
  }
}

const char *dmrg_last_error(const dmrg_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int dmrg_create(dmrg_ctx **out, const dmrg_config *cfg) {
  if (!out || !cfg) return DMRG_ERR_ARG;
  *out = nullptr;
  if ((cfg->sym != DMRG_U1 && cfg->sym != DMRG_U1U1 && cfg->sym != DMRG_U1SU2) ||
      cfg->n_sites < 2 || cfg->n_up < 0 || cfg->d_max < 1)
    return DMRG_ERR_ARG;
  // spin-adapted windows are built for total spin S = 0 (N even)
  if (cfg->sym == DMRG_U1SU2 && (cfg->twice_s != 0 || (cfg->n_up & 1) || cfg->n_up > 2 * cfg->n_sites))
    return DMRG_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return DMRG_ERR_CUDA;
  }
  dmrg_ctx *C = new (std::nothrow) dmrg_ctx();
  if (!C) return DMRG_ERR_OOM;
  C->cfg = *cfg;
  if (C->cfg.davidson_max_sub < 4) C->cfg.davidson_max_sub = 20;
  if (C->cfg.davidson_max_iter < 1) C->cfg.davidson_max_iter = 200;
  C->spinful = cfg->sym == DMRG_U1U1 || cfg->sym == DMRG_U1SU2;
  C->su2 = cfg->sym == DMRG_U1SU2;
  C->N = cfg->n_sites;
  C->M = C->spinful ? 2 * C->N : C->N;
  C->target = C->su2 ? su2::label(cfg->n_up, cfg->twice_s)
                     : (C->spinful ? QN{cfg->n_up, cfg->n_dn} : QN{cfg->n_up, 0});
  C->precision = cfg->precision;
  // pinned host status words for the stream-ordered time-out report
  if (cudaHostAlloc((void **)&C->hflag, 2 * sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
      cudaEventCreateWithFlags(&C->flag_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&C->flag_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (C->hflag) cudaFreeHost(C->hflag);
    for (auto &e : C->flag_ev)
      if (e) cudaEventDestroy(e);
    delete C;
    return DMRG_ERR_OOM;
  }
  C->hflag[0] = C->hflag[1] = 0;
  *out = C;
  return DMRG_OK;
}

int dmrg_destroy(dmrg_ctx *ctx) {
  if (!ctx) return DMRG_OK;
  // wait for this context's own work only (other contexts may be running)
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->cap_stream) cudaStreamSynchronize(ctx->cap_stream);
  for (auto &g : ctx->win.graphs) cudaGraphExecDestroy(g.second);
  ctx->win.graphs.clear();
  // the FP64 stacks are unmapped at once: wait for the last apply callers enqueued
  if (ctx->win.used) cudaEventSynchronize(ctx->win.use_ev);
  ctx->win.vA.free_all();
  ctx->win.vB.free_all();
  ctx->win.vT.free_all();
  release_after_use(ctx->win);
  ctx->win.buf.clear();
  ctx->win.ldbuf.clear();
  ctx->win.rdbuf.clear();
  clear_blocks(ctx);
  ctx->partbuf.clear();
  ctx->partdata.clear();
  for (auto &ev : ctx->h2d_events) {
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
  }
  if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
  if (ctx->stage_stream) {
    cudaStreamSynchronize(ctx->stage_stream);
    cudaStreamDestroy(ctx->stage_stream);
  }
  ctx->dav.clear();
  if (ctx->solver_params) cusolverDnDestroyParams(ctx->solver_params);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->win.use_ev) cudaEventDestroy(ctx->win.use_ev);
  for (auto &e : ctx->flag_ev)
    if (e) {
      cudaEventSynchronize(e);
      cudaEventDestroy(e);
    }
  if (ctx->hflag) cudaFreeHost(ctx->hflag);
  delete ctx;
  return DMRG_OK;
}

int dmrg_lattice_hamiltonian(int model, int Lx, int Ly, double t, double tp, double v,
                             double *t_out, double *V_out) {
  if (Lx < 3 || Ly < 3 || !t_out || !V_out) return DMRG_ERR_ARG;
  if (model != DMRG_MODEL_SPINLESS_TV && model != DMRG_MODEL_HUBBARD) return DMRG_ERR_ARG;
  const int N = Lx * Ly;
  std::fill(t_out, t_out + (size_t)N * N, 0.0);
  std::fill(V_out, V_out + (size_t)N * N * N * N, 0.0);
  std::vector<std::pair<int, int>> nn, nnn;
  torus_bonds(Lx, Ly, false, nn);
  for (auto &b : nn) {
    t_out[(size_t)b.first * N + b.second] += -t;
    t_out[(size_t)b.second * N + b.first] += -t;
    if (model == DMRG_MODEL_SPINLESS_TV)
      V_out[(((size_t)b.first * N + b.second) * N + b.second) * N + b.first] += v;
  }
  if (model == DMRG_MODEL_SPINLESS_TV && tp != 0.0) {
    torus_bonds(Lx, Ly, true, nnn);
    for (auto &b : nnn) {
      t_out[(size_t)b.first * N + b.second] += -tp;
      t_out[(size_t)b.second * N + b.first] += -tp;
    }
  }
  if (model == DMRG_MODEL_HUBBARD)
    for (int i = 0; i < N; ++i) V_out[(((size_t)i * N + i) * N + i) * N + i] = v / 2.0;
  return DMRG_OK;
}

int dmrg_momentum_basis(int Lx, int Ly, double *U) {
  if (Lx < 1 || Ly < 1 || !U) return DMRG_ERR_ARG;
  const int N = Lx * Ly;
  const double PI = 3.14159265358979323846;
  struct Mode {
    double eps;
    int nx, ny, sn;
    bool self;
  };
  std::vector<Mode> modes;
  std::vector<char> seen(N, 0);
  for (int ny = 0; ny < Ly; ++ny)
    for (int nx = 0; nx < Lx; ++nx) {
      if (seen[ny * Lx + nx]) continue;
      int mx = (Lx - nx) % Lx, my = (Ly - ny) % Ly;
      seen[ny * Lx + nx] = seen[my * Lx + mx] = 1;
      int rx = nx, ry = ny;
      if (std::make_pair(mx, my) < std::make_pair(nx, ny)) rx = mx, ry = my;
      double eps = -2.0 * (std::cos(2 * PI * rx / Lx) + std::cos(2 * PI * ry / Ly));
      eps = std::round(eps * 1e12) / 1e12;
      bool self = (mx == nx && my == ny);
      modes.push_back({eps, rx, ry, 0, self});
      if (!self) modes.push_back({eps, rx, ry, 1, false});
    }
  std::sort(modes.begin(), modes.end(), [](const Mode &a, const Mode &b) {
    if (a.eps != b.eps) return a.eps < b.eps;
    if (a.nx != b.nx) return a.nx < b.nx;
    if (a.ny != b.ny) return a.ny < b.ny;
    return a.sn < b.sn;
  });
  for (int m = 0; m < N; ++m) {
    const Mode &md = modes[m];
    double kx = 2 * PI * md.nx / Lx, ky = 2 * PI * md.ny / Ly;
    for (int i = 0; i < N; ++i) {
      double ph = kx * (i % Lx) + ky * (i / Lx);
      double amp = md.self ? std::sqrt(1.0 / N) : std::sqrt(2.0 / N);
      U[(size_t)i * N + m] = amp * (md.sn ? std::sin(ph) : std::cos(ph));
    }
  }
  return DMRG_OK;
}

int dmrg_set_hamiltonian(dmrg_ctx *C, const double *t, const double *V, const double *U) {
  if (!C || !t || !V) return DMRG_ERR_ARG;
  return guard(C, [&] {
    C->derive_cache.clear();
    C->derive_cache_terms = 0;
    const int N = C->N;
    const size_t N2 = (size_t)N * N, N4 = N2 * N2;
    double vmax = 0;
    for (size_t e = 0; e < N4; ++e) vmax = std::max(vmax, std::fabs(V[e]));
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        if (std::fabs(t[(size_t)i * N + j] - t[(size_t)j * N + i]) > 1e-12 * (1 + std::fabs(t[(size_t)i * N + j])))
          fail(DMRG_ERR_ARG, "t is not symmetric at (%d,%d)", i, j);
        for (int k = 0; k < N; ++k)
          for (int l = 0; l < N; ++l) {
            double a = V[((i * (size_t)N + j) * N + k) * N + l];
            double b = V[((l * (size_t)N + k) * N + j) * N + i];
            if (std::fabs(a - b) > 1e-12 * (1 + vmax))
              fail(DMRG_ERR_ARG, "V is not Hermitian: V[%d,%d,%d,%d] != V[%d,%d,%d,%d]", i, j, k, l, l, k, j, i);
          }
      }
    std::vector<double> tt(t, t + N2), VV(V, V + N4);
    if (U) {
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
          double s = 0;
          for (int i = 0; i < N; ++i) s += U[(size_t)i * N + a] * U[(size_t)i * N + b];
          if (std::fabs(s - (a == b)) > 1e-10) fail(DMRG_ERR_ARG, "mode rotation is not orthogonal");
        }
      std::vector<double> tmp(N2, 0.0);
      for (int i = 0; i < N; ++i)
        for (int b = 0; b < N; ++b) {
          double s = 0;
          for (int j = 0; j < N; ++j) s += t[(size_t)i * N + j] * U[(size_t)j * N + b];
          tmp[(size_t)i * N + b] = s;
        }
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
          double s = 0;
          for (int i = 0; i < N; ++i) s += U[(size_t)i * N + a] * tmp[(size_t)i * N + b];
          tt[(size_t)a * N + b] = s;
        }
      std::vector<double> w2;
      for (int ax = 0; ax < 4; ++ax) {
        quarter(VV, w2, U, N, ax);
        VV.swap(w2);
      }
    }
    const int M = C->M;
    C->h.assign((size_t)M * M, 0.0);
    C->W.assign((size_t)M * M * M * M, 0.0);
    auto sp = [&](int p) { return C->spinful ? p / 2 : p; };
    auto sg = [&](int p) { return C->spinful ? p % 2 : 0; };
    for (int p = 0; p < M; ++p)
      for (int q = 0; q < M; ++q)
        if (sg(p) == sg(q)) C->h[(size_t)p * M + q] = tt[(size_t)sp(p) * N + sp(q)];
    auto X = [&](int p, int q, int r, int s) -> double {
      if (sg(p) != sg(s) || sg(q) != sg(r)) return 0.0;
      return VV[(((size_t)sp(p) * N + sp(q)) * N + sp(r)) * N + sp(s)];
    };
    for (int p = 0; p < M; ++p)
      for (int q = 0; q < M; ++q)
        for (int r = 0; r < M; ++r)
          for (int s = 0; s < M; ++s)
            C->W[(((size_t)p * M + q) * M + r) * M + s] =
                0.25 * (X(p, q, r, s) - X(q, p, r, s) - X(p, q, s, r) + X(q, p, s, r));
    C->ham = true;
    clear_blocks(C);
    C->win.valid = false;
  });
}

int dmrg_random_start(dmrg_ctx *C, uint64_t seed) {
  if (!C) return DMRG_ERR_ARG;
  return guard(C, [&] {
    // site states (the enlargement's order)
    std::vector<QN> sq;
    std::vector<int> stj;
    if (C->su2) {
      sq = {su2::label(0, 0), su2::label(1, 1), su2::label(2, 0)};
      stj = {0, 1, 0};
    } else if (C->spinful) {
      sq = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};
    } else {
      sq = {{0, 0}, {1, 0}};
    }
    // counter-based normal deviates (splitmix64 + Box-Muller)
    uint64_t ctr = seed * 0x9E3779B97F4A7C15ull + 1;
    auto u01 = [&]() {
      uint64_t z = (ctr += 0x9E3779B97F4A7C15ull);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    auto normal = [&]() { return std::sqrt(-2.0 * std::log(u01())) * std::cos(6.283185307179586 * u01()); };
    const int D = std::max(1, C->cfg.d_max);
    std::map<QN, int> dims{{QN{0, 0}, 1}};
    for (int n = C->N - 1; n >= 1; --n) {
      // sectors of site_n x R_{n+1} that can still reach the target
      std::map<QN, int> e;
      for (size_t k = 0; k < sq.size(); ++k)
        for (auto &kv : dims) {
          if (C->su2) {
            const int t1 = su2::tj_of(kv.first), t2 = stj[k];
            for (int tj = std::abs(t1 - t2); tj <= t1 + t2; tj += 2) {
              const QN Q = su2::label(su2::n_of(kv.first) + su2::n_of(sq[k]), tj);
              if (allowed_q(C, Q, n)) e[Q] += kv.second;
            }
          } else {
            const QN Q = qadd(kv.first, sq[k]);
            if (allowed_q(C, Q, n)) e[Q] += kv.second;
          }
        }
      long long tot = 0;
      for (auto &kv : e) tot += kv.second;
      std::map<QN, int> keep;
      for (auto &kv : e) {
        int d = tot <= D ? kv.second : (int)((long long)D * kv.second / tot);
        d = std::min(kv.second, std::max(d, 1));
        keep[kv.first] = d;
      }
      Iso T;
      long long off = 0;
      for (auto &kv : keep) {
        const int rows = e[kv.first], cols = kv.second;
        std::vector<double> m((size_t)rows * cols);
        for (double &x : m) x = normal();
        // orthonormal columns: modified Gram-Schmidt, twice
        for (int c = 0; c < cols; ++c)
          for (int pass = 0; pass < 2; ++pass) {
            for (int c2 = 0; c2 < c; ++c2) {
              double d = 0;
              for (int r = 0; r < rows; ++r) d += m[(size_t)r * cols + c] * m[(size_t)r * cols + c2];
              for (int r = 0; r < rows; ++r) m[(size_t)r * cols + c] -= d * m[(size_t)r * cols + c2];
            }
            double nn = 0;
            for (int r = 0; r < rows; ++r) nn += m[(size_t)r * cols + c] * m[(size_t)r * cols + c];
            nn = std::sqrt(nn);
            if (!(nn > 1e-12)) fail(DMRG_ERR_STATE, "internal: degenerate random isometry");
            for (int r = 0; r < rows; ++r) m[(size_t)r * cols + c] /= nn;
          }
        T.qn.push_back(kv.first);
        T.rows.push_back(rows);
        T.cols.push_back(cols);
        T.off.push_back(off);
        off += (long long)rows * cols;
        T.host.insert(T.host.end(), m.begin(), m.end());
      }
      C->riso[n] = std::move(T);
      dims = keep;
    }
  });
}

int dmrg_set_isometry(dmrg_ctx *C, int side, int site, int ns, const int *qn, const int *rows,
                      const int *cols, const double *data) {
  if (!C || (side != 0 && side != 1) || site < 1 || site > C->N - 1 || ns < 1 || !qn || !rows ||
      !cols || !data)
    return DMRG_ERR_ARG;
  return guard(C, [&] {
    Iso T;
    const int nq = C->spinful ? 2 : 1;
    long long off = 0;
    for (int k = 0; k < ns; ++k) {
      QN q{qn[k * nq], nq == 2 ? qn[k * nq + 1] : 0};
      if (C->su2) {   // (N, 2J) -> highest-weight label
        if (q[0] < 0 || q[1] < 0 || ((q[0] + q[1]) & 1) || q[1] > q[0])
          fail(DMRG_ERR_ARG, "bad spin-adapted sector (%d, %d)", q[0], q[1]);
        q = su2::label(q[0], q[1]);
      }
      if (rows[k] < 1 || cols[k] < 1 || cols[k] > rows[k]) fail(DMRG_ERR_ARG, "bad isometry shape in sector %d", k);
      T.qn.push_back(q);
      T.rows.push_back(rows[k]);
      T.cols.push_back(cols[k]);
      T.off.push_back(off);
      off += (long long)rows[k] * cols[k];
    }
    T.host.assign(data, data + off);
    auto &m = side == 0 ? C->liso : C->riso;
    m[site] = std::move(T);
  });
}

int dmrg_build_block_ops(dmrg_ctx *C, int l, void *stream) {
  if (!C) return DMRG_ERR_ARG;
  return guard(C, [&] {
    const int N = C->N;
    if (!C->ham) fail(DMRG_ERR_STATE, "dmrg_set_hamiltonian first");
    if (l < 0 || l > N - 2) fail(DMRG_ERR_ARG, "window %d out of range", l);
    for (int n = 1; n <= l; ++n)
      if (!C->liso.count(n)) fail(DMRG_ERR_STATE, "left isometry %d missing", n);
    for (int n = l + 2; n <= N - 1; ++n)
      if (!C->riso.count(n)) fail(DMRG_ERR_STATE, "right isometry %d missing", n);
    cudaStream_t s = (cudaStream_t)stream;
    C->stream = s;
    double t0 = now();
    clear_blocks(C);
    C->L.push_back(vacuum(C));
    // under a budget, a block is released once the next one is built from it
    const bool lean = C->cfg.hbm_budget_bytes > 0;
    for (int n = 1; n <= l; ++n) {
      upload_iso(C, C->liso[n]);
      grow_left(C, n, C->liso[n]);
      if (lean) release(C, C->L[n - 1].get());
    }
    C->R[N] = vacuum(C);
    for (int n = N - 1; n >= l + 2; --n) {
      upload_iso(C, C->riso[n]);
      grow_right(C, n, C->riso[n]);
      if (lean) release(C, C->R[n + 1].get());
    }
    C->prof[1] += now() - t0;
    build_window(C, l);
  });
}

int dmrg_heff_layout(dmrg_ctx *C, long long *psi_len, int *n_blocks, int *blocks) {
  if (!C) return DMRG_ERR_ARG;
  if (!C->win.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  const Window &w = C->win;
  if (psi_len) *psi_len = w.psi_len;
  if (n_blocks) *n_blocks = (int)w.psi.size();
  if (blocks) {
    const int nq = C->spinful ? 2 : 1;
    int k = 0;
    auto ext = [&](const QN &q) { return C->su2 ? QN{su2::n_of(q), su2::tj_of(q)} : q; };
    for (const PsiBlk &p : w.psi) {
      for (int i = 0; i < nq; ++i) blocks[k++] = ext(w.Ld.basis.qn[p.a])[i];
      for (int i = 0; i < nq; ++i) blocks[k++] = ext(w.Rd.basis.qn[p.b])[i];
      blocks[k++] = p.da;
      blocks[k++] = p.db;
    }
  }
  return DMRG_OK;
}

int dmrg_gemm_tile_choice(int M, int N, int batch, int fold_rows_ok, int fold_cols_ok,
                          int square_only, int *out3) {
  if (M < 1 || N < 1 || batch < 1 || !out3) return DMRG_ERR_ARG;
  int q = 0, f = 0;
  gemm_tile_choice(M, N, batch, fold_rows_ok != 0, fold_cols_ok != 0, square_only != 0, &q, &f);
  out3[0] = kGemmShapes[q][0];
  out3[1] = kGemmShapes[q][1];
  out3[2] = f;
  return DMRG_OK;
}

int dmrg_set_split_min_flops(dmrg_ctx *C, double min_window_flops) {
  if (!C || !(min_window_flops >= 0.0)) return DMRG_ERR_ARG;
  C->split_min_flops = min_window_flops;
  return DMRG_OK;
}

int dmrg_set_refinement(dmrg_ctx *C, int inner_steps, double min_window_flops) {
  if (!C || inner_steps < 0 || inner_steps > 1000 || !(min_window_flops >= 0.0)) return DMRG_ERR_ARG;
  C->refine_steps = inner_steps;
  C->refine_min_flops = min_window_flops;
  return DMRG_OK;
}

int dmrg_set_precision(dmrg_ctx *C, int precision) {
  if (!C || (precision != DMRG_FP64 && precision != DMRG_SPLIT)) return DMRG_ERR_ARG;
  C->precision = precision;
  return DMRG_OK;
}

int dmrg_heff_apply(dmrg_ctx *C, const double *psi, double *sigma, void *stream) {
  if (!C || !psi || !sigma) return DMRG_ERR_ARG;
  if (!C->win.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  return guard(C, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    poll_flags(C, false, s);
    take_sticky(C);
    apply(C, psi, sigma, s, C->precision);
    if (C->precision == DMRG_SPLIT) post_flag(C, 0, C->win.tf.err, s);
    note_use(C->win, s);
  });
}

int dmrg_heff_apply_batch(dmrg_ctx *C, int nv, const double *psi, double *sigma, void *stream) {
  if (!C || !psi || !sigma || nv < 1 || nv > 64) return DMRG_ERR_ARG;
  if (!C->win.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  return guard(C, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    poll_flags(C, false, s);
    take_sticky(C);
    apply_batch(C, nv, psi, sigma, s);
    if (C->precision == DMRG_SPLIT) post_flag(C, 0, C->win.tf.err, s);
    note_use(C->win, s);
  });
}

int dmrg_sync(dmrg_ctx *C, void *stream) {
  if (!C) return DMRG_ERR_ARG;
  return guard(C, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(s));
    poll_flags(C, true, s);
    take_sticky(C);
    check_err_flag(C, s);
  });
}

int dmrg_heff_apply_host(dmrg_ctx *C, const double *psi_h, double *sigma_h, void *stream) {
  if (!C || !psi_h || !sigma_h) return DMRG_ERR_ARG;
  if (!C->win.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  return guard(C, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    poll_flags(C, false, s);
    take_sticky(C);
    const long long n = C->win.psi_len;
    WinBuf b(s);   // stream-ordered from the pool: no device synchronisation
    double *dp = (double *)b.alloc(8 * std::max<long long>(n, 1));
    double *ds = (double *)b.alloc(8 * std::max<long long>(n, 1));
    CK(cudaMemcpyAsync(dp, psi_h, 8 * n, cudaMemcpyHostToDevice, s));
    apply(C, dp, ds, s, C->precision);
    CK(cudaMemcpyAsync(sigma_h, ds, 8 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    check_err_flag(C, s);
  });
}

int dmrg_heff_apply_split_static(dmrg_ctx *C, const double *psi, double *sigma, void *stream) {
  if (!C || !psi || !sigma) return DMRG_ERR_ARG;
  if (!C->win.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  return guard(C, [&] {
    Window &w = C->win;
    cudaStream_t s = (cudaStream_t)stream;
    if (!w.tf_copies)
      fail(DMRG_ERR_STATE, "split operator copies not built: call dmrg_heff_apply once with "
                           "DMRG_SPLIT after dmrg_build_block_ops");
    void *base = nullptr;
    size_t cap = 0;
    CK(static_scratch(&base, &cap));
    CK(split_prepare());
    int dev = 0;
    CK(cudaGetDevice(&dev));
    // layout: [error flag, item counters (bytes 16..23) | tables | psi statistics |
    //          psi^T hi, lo | T hi, lo | partial tiles]
    struct Owner {
      long long gen = -1;
      bool word_cleared = false;
      SplitTables tb;
      size_t o_maps, o_seg, o_w1, o_w2, o_ps, o_split, o_pdesc, o_pstat;
    };
    static std::mutex mu;
    static std::map<int, Owner> owners;
    std::lock_guard<std::mutex> lk(mu);
    Owner &ow = owners[dev];
    // a time-out recorded by an earlier call is reported here once its status
    // copy has landed (dmrg_sync waits for it)
    poll_flags(C, false, s);
    take_sticky(C);
    if (!ow.word_cleared) {   // the error word starts at zero; later only a read clears it
      CK(cudaMemsetAsync(base, 0, sizeof(int), s));
      ow.word_cleared = true;
    }
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    unsigned char *b = (unsigned char *)base;
    const int ks = w.ksub ? w.ksub : KSUB_DEFAULT;
    const size_t np = w.psi.size();
    if (ow.gen != w.gen) {
      SplitScratch z = split_scratch_sizes(w, ks);
      // table sizes do not depend on the pointers: size them with a dry run
      SplitTables probe;
      __half *hb = (__half *)b;
      split_tables(w, z, hb, hb, hb, hb, (float *)b, probe, ks, w.cap1, w.order1);
      size_t off = 256;
      ow.o_maps = off; off = al(off + probe.maps.size() * sizeof(CUtensorMap));
      ow.o_seg = off; off = al(off + probe.segs.size() * sizeof(TSeg));
      ow.o_w1 = off; off = al(off + probe.w1.size() * sizeof(TWork));
      ow.o_w2 = off; off = al(off + probe.w2.size() * sizeof(TWork));
      ow.o_ps = off; off = al(off + probe.psums.size() * sizeof(PartialSum));
      ow.o_split = off; off = al(off + probe.psi_split.size() * sizeof(F16Split));
      ow.o_pdesc = off; off = al(off + np * sizeof(PsiDesc));
      ow.o_pstat = off; off = al(off + np * sizeof(PsiStat));
      const size_t oPh = off;
      off = al(off + 2 * (size_t)z.nP);
      const size_t oPl = off;
      off = al(off + 2 * (size_t)z.nP);
      const size_t oTh = off;
      off = al(off + 2 * (size_t)z.nT);
      const size_t oTl = off;
      off = al(off + 2 * (size_t)z.nT);
      const size_t oW = off;
      off = al(off + 4 * (size_t)z.nws);
      if (off > cap)
        fail(DMRG_ERR_ARG, "window needs %zu bytes of scratch; the static scratch holds %zu bytes "
                           "(use dmrg_heff_apply for larger windows)", off, cap);
      ow.gen = -1;
      split_tables(w, z, (__half *)(b + oPh), (__half *)(b + oPl), (__half *)(b + oTh),
                   (__half *)(b + oTl), (float *)(b + oW), ow.tb, ks, w.cap1, w.order1);
      const SplitTables &t = ow.tb;
      const std::vector<PsiDesc> pd = psi_descs(w);
      auto put = [&](size_t o, const void *src, size_t n) {
        if (n) CK(cudaMemcpyAsync(b + o, src, n, cudaMemcpyHostToDevice, s));
      };
      put(ow.o_maps, t.maps.data(), t.maps.size() * sizeof(CUtensorMap));
      put(ow.o_seg, t.segs.data(), t.segs.size() * sizeof(TSeg));
      put(ow.o_w1, t.w1.data(), t.w1.size() * sizeof(TWork));
      put(ow.o_w2, t.w2.data(), t.w2.size() * sizeof(TWork));
      put(ow.o_ps, t.psums.data(), t.psums.size() * sizeof(PartialSum));
      put(ow.o_split, t.psi_split.data(), t.psi_split.size() * sizeof(F16Split));
      put(ow.o_pdesc, pd.data(), pd.size() * sizeof(PsiDesc));
      ow.gen = w.gen;
    }
    const SplitTables &t = ow.tb;
    int *err = (int *)b;
    PsiStat *pst = (PsiStat *)(b + ow.o_pstat);
    CK(psi_stats((const PsiDesc *)(b + ow.o_pdesc), (int)np, psi, pst, s));
    CK(f16_split((const F16Split *)(b + ow.o_split), (int)t.psi_split.size(), pst, psi, s,
                 split_tile_count(t.psi_split)));
    CK(split_gemm((const TWork *)(b + ow.o_w1), (int)t.w1.size(), (int *)(b + 16),
                  (const TSeg *)(b + ow.o_seg),
                  (const CUtensorMap *)(b + ow.o_maps), pst, err, s));
    CK(split_gemm((const TWork *)(b + ow.o_w2), (int)t.w2.size(), (int *)(b + 20),
                  (const TSeg *)(b + ow.o_seg),
                  (const CUtensorMap *)(b + ow.o_maps), pst, err, s));
    CK(sum_partials((const PartialSum *)(b + ow.o_ps), (int)t.psums.size(), sigma, s));
    post_flag(C, 1, err, s);
    note_use(w, s);
  });
}

int dmrg_selftest_bounded_wait(void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int *d = nullptr, h = 0;
  if (cudaMallocAsync(&d, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return DMRG_ERR_OOM;
  }
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) e = wait_selftest(d, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DMRG_ERR_CUDA;
  }
  return h == 7 ? DMRG_ERR_TIMEOUT : DMRG_ERR_CUDA;
}

int dmrg_selftest_timeout_report(dmrg_ctx *C, int which, void *stream) {
  if (!C || (which != 0 && which != 1)) return DMRG_ERR_ARG;
  return guard(C, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    int *word = nullptr;
    if (which == 0) {
      if (!C->win.valid || !C->win.tf_ready) fail(DMRG_ERR_STATE, "no split plan: apply once with DMRG_SPLIT");
      word = C->win.tf.err;
    } else {
      void *b = nullptr;
      size_t cap = 0;
      CK(static_scratch(&b, &cap));
      word = (int *)b;
    }
    CK(cudaMemsetAsync(word, 0, sizeof(int), s));
    CK(wait_selftest(word, s));
    post_flag(C, which, word, s);
  });
}

int dmrg_heff_flops(dmrg_ctx *C, double *flops) {
  if (!C || !flops) return DMRG_ERR_ARG;
  if (!C->win.valid) return DMRG_ERR_STATE;
  *flops = C->win.flops;
  return DMRG_OK;
}

int dmrg_davidson(dmrg_ctx *C, double *psi, double *energy, int *iters, void *stream) {
  if (!C || !psi || !energy) return DMRG_ERR_ARG;
  if (!C->win.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  int rc = DMRG_OK;
  int g = guard(C, [&] { rc = davidson(C, psi, energy, iters, (cudaStream_t)stream); });
  return g != DMRG_OK ? g : rc;
}

int dmrg_truncate(dmrg_ctx *C, const double *psi, int side, int d_max, double *disc, double *ent,
                  void *stream) {
  if (!C || !psi || (side != 0 && side != 1) || d_max < 1) return DMRG_ERR_ARG;
  if (!C->win.valid) return DMRG_ERR_STATE;
  return guard(C, [&] { truncate(C, psi, side, d_max, disc, ent, (cudaStream_t)stream); });
}

int dmrg_sweep(dmrg_ctx *C, int n_sweeps, const int *d_schedule, double *E, void *stream) {
  if (!C || n_sweeps < 1) return DMRG_ERR_ARG;
  return guard(C, [&] { sweep_impl(C, n_sweeps, d_schedule, E, (cudaStream_t)stream); });
}

int dmrg_heff_stage_info(dmrg_ctx *C, double *out6) {
  if (!C || !out6) return DMRG_ERR_ARG;
  if (!C->win.valid) return DMRG_ERR_STATE;
  const Window &w = C->win;
  out6[0] = w.flops1;
  out6[1] = w.flops2;
  out6[2] = (double)w.nA;
  out6[3] = (double)w.nB;
  out6[4] = (double)w.nT;
  out6[5] = (double)w.psi_len;
  return DMRG_OK;
}

int dmrg_heff_split_plan(dmrg_ctx *C, double *out4) {
  if (!C || !out4) return DMRG_ERR_ARG;
  const Window &w = C->win;
  if (!w.valid || !w.tf_ready) {
    C->err = "split plan not built: apply once with DMRG_SPLIT first";
    return DMRG_ERR_STATE;
  }
  const SplitPlan &P = w.tf;
  const int launches = 2 + (P.npsum > 0 ? 1 : 0) + (P.nwork1 > 0) + (P.nwork2 > 0);
  out4[0] = launches;
  out4[1] = P.nwork1;
  out4[2] = P.nwork2;
  out4[3] = (double)w.ksub;
  return DMRG_OK;
}

long long dmrg_sweep_next_use(int n_sites, int pass, int l, int left, int n) {
  if (n_sites < 2 || (pass != 0 && pass != 1) || l < 0 || l > n_sites - 2) return -2;
  return next_use(n_sites, pass, l, left != 0, n);
}

int dmrg_rdm1(dmrg_ctx *C, const double *psi, double *gamma, void *stream) {
  if (!C || !psi || !gamma) return DMRG_ERR_ARG;
  if (!C->win.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  return guard(C, [&] { rdm1(C, psi, gamma, (cudaStream_t)stream); });
}

int dmrg_staging_stats(dmrg_ctx *C, double *out8) {
  if (!C || !out8) return DMRG_ERR_ARG;
  return guard(C, [&] {
    collect_h2d_times(C);
    out8[0] = C->st_h2d_bytes;
    out8[1] = C->st_h2d_ms * 1e-3;
    out8[2] = C->st_d2h_bytes;
    out8[3] = C->st_peak;
    out8[4] = (double)C->st_offloads;
    out8[5] = (double)C->st_reloads;
    out8[6] = (double)C->st_releases;
    out8[7] = (double)C->cfg.hbm_budget_bytes;
  });
}

int dmrg_heff_fp64_state(dmrg_ctx *C, long long *out4) {
  if (!C || !out4) return DMRG_ERR_ARG;
  const Window &w = C->win;
  if (!w.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  out4[0] = (w.fp64_stacks && w.vA.mapped && w.vB.mapped) ? 1 : 0;
  out4[1] = w.vT.mapped ? 1 : 0;
  out4[2] = (long long)(w.vA.size + w.vB.size);
  out4[3] = (long long)w.vT.size;
  return DMRG_OK;
}

int dmrg_heff_split_paths(dmrg_ctx *C, long long *out8) {
  if (!C || !out8) return DMRG_ERR_ARG;
  const Window &w = C->win;
  if (!w.valid || !w.tf_ready) {
    C->err = "split plan not built: apply once with DMRG_SPLIT first";
    return DMRG_ERR_STATE;
  }
  const SplitTables &t = C->tables;
  for (int i = 0; i < 8; ++i) out8[i] = 0;
  out8[0] = (long long)t.w1.size();
  out8[1] = (long long)t.w2.size();
  for (const PsiBlk &p : w.psi)
    if (p.da > 128 || p.db > 128) ++out8[2];
  for (const TWork &x : t.w2) {
    if (x.R == 2) ++out8[3];
    if (x.R == 4) ++out8[4];
    if (x.R <= 1 && (x.m0 > 0 || x.n0 > 0)) ++out8[7];
  }
  for (const PartialSum &p : t.psums) {
    out8[5] = std::max<long long>(out8[5], p.nparts);
    if (p.nparts > 1) ++out8[6];
  }
  return DMRG_OK;
}

int dmrg_get_mps(dmrg_ctx *C, int side, int site, int *n_sectors, long long *n_elems, int *qn,
                 int *rows, int *cols, double *data) {
  if (!C || (side != 0 && side != 1) || !n_sectors || !n_elems) return DMRG_ERR_ARG;
  return guard(C, [&] {
    const std::map<int, Iso> &m = C->swept ? (side == 0 ? C->Lmap : C->Rmap)
                                           : (side == 0 ? C->liso : C->riso);
    auto it = m.find(site);
    if (it == m.end())
      fail(DMRG_ERR_ARG, "no %s isometry %d in the current MPS", side == 0 ? "left" : "right", site);
    const Iso &T = it->second;
    const int nq = C->spinful ? 2 : 1;
    long long tot = 0;
    for (size_t k = 0; k < T.qn.size(); ++k) tot += (long long)T.rows[k] * T.cols[k];
    *n_sectors = (int)T.qn.size();
    *n_elems = tot;
    for (size_t k = 0; k < T.qn.size(); ++k) {
      const QN q = C->su2 ? QN{su2::n_of(T.qn[k]), su2::tj_of(T.qn[k])} : T.qn[k];
      if (qn)
        for (int i = 0; i < nq; ++i) qn[k * nq + i] = q[i];
      if (rows) rows[k] = T.rows[k];
      if (cols) cols[k] = T.cols[k];
    }
    if (data && tot) {
      if ((long long)T.host.size() == tot) {
        memcpy(data, T.host.data(), 8 * tot);
      } else if (T.d) {
        CK(cudaMemcpy(data, T.d, 8 * tot, cudaMemcpyDeviceToHost));
      } else {
        fail(DMRG_ERR_STATE, "isometry %d has no data", site);
      }
    }
  });
}

int dmrg_get_center(dmrg_ctx *C, int *l, long long *psi_len, double *psi) {
  if (!C || !l || !psi_len) return DMRG_ERR_ARG;
  if (!C->swept || C->center_l < 0) {
    C->err = "no sweep has run";
    return DMRG_ERR_STATE;
  }
  *l = C->center_l;
  *psi_len = (long long)C->center_psi.size();
  if (psi && !C->center_psi.empty()) memcpy(psi, C->center_psi.data(), 8 * C->center_psi.size());
  return DMRG_OK;
}

int dmrg_heff_entries(dmrg_ctx *C, int *out, int max_entries, int *n_entries) {
  if (!C || !n_entries) return DMRG_ERR_ARG;
  const Window &w = C->win;
  if (!w.valid) {
    C->err = "no window built";
    return DMRG_ERR_STATE;
  }
  *n_entries = (int)w.s1info.size();
  if (out)
    for (int i = 0; i < std::min(max_entries, *n_entries); ++i) {
      const S1 &e = w.s1info[i];
      out[3 * i] = e.pi;
      out[3 * i + 1] = e.po;
      out[3 * i + 2] = (int)w.hc[e.ci].terms.size();
    }
  return DMRG_OK;
}

int dmrg_heff_timing(dmrg_ctx *C, int enable, double *out5) {
  if (!C) return DMRG_ERR_ARG;
  return guard(C, [&] {
    if (!C->ev[0])
      for (auto &e : C->ev) CK(cudaEventCreate(&e));
    collect_timing(C);
    if (out5)
      for (int i = 0; i < 5; ++i) out5[i] = C->tacc[i];
    if (enable && !C->timing)
      for (double &t : C->tacc) t = 0;
    C->timing = enable != 0;
  });
}

int dmrg_heff_tuning(dmrg_ctx *C, double *out, int max_entries, int *n_entries) {
  if (!C || !n_entries) return DMRG_ERR_ARG;
  *n_entries = (int)C->tune_log.size();
  if (out)
    for (int i = 0; i < std::min(max_entries, *n_entries); ++i) {
      out[2 * i] = C->tune_log[i][0];
      out[2 * i + 1] = C->tune_log[i][1];
    }
  return DMRG_OK;
}

int dmrg_set_graphs(dmrg_ctx *C, int enable) {
  if (!C) return DMRG_ERR_ARG;
  C->use_graphs = enable != 0;
  return DMRG_OK;
}

int dmrg_memory_stats(dmrg_ctx *C, double *out6) {
  if (!C || !out6) return DMRG_ERR_ARG;
  for (int i = 0; i < 6; ++i) out6[i] = C->mem_max[i];
  return DMRG_OK;
}

int dmrg_profile(dmrg_ctx *C, double *out7) {
  if (!C || !out7) return DMRG_ERR_ARG;
  for (int i = 0; i < 7; ++i) out7[i] = C->prof[i];
  return DMRG_OK;
}

}  // extern "C"
