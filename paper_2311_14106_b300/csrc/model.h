// Host-side data model of libdmrgb300: quantum numbers, bases, operator
// classes, block parts and the window of two-site DMRG.
#pragma once
#include <array>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "kernels.h"

namespace dmrg {

using QN = std::array<int, 2>;   // (N) or (N_up, N_dn); unused entries are 0

inline QN qadd(const QN &a, const QN &b) { return {a[0] + b[0], a[1] + b[1]}; }
inline QN qsub(const QN &a, const QN &b) { return {a[0] - b[0], a[1] - b[1]}; }
inline QN qneg(const QN &a) { return {-a[0], -a[1]}; }
inline int qparity(const QN &a) { return (a[0] + a[1]) & 1; }
inline int qnum(const QN &a) { return a[0] + a[1]; }

struct Basis {
  std::vector<QN> qn;
  std::vector<int> dim;
  int find(const QN &q) const {
    for (size_t i = 0; i < qn.size(); ++i)
      if (qn[i] == q) return (int)i;
    return -1;
  }
  long long total() const {
    long long t = 0;
    for (int d : dim) t += d;
    return t;
  }
};

// Piece of an enlarged sector: one site state times one block sector.
struct Piece {
  int site_state;
  int blk_sector;
  int off;
  int dim;
};

// Operators with the same QN shift on the same basis share one block
// structure and are stored op-major in one device array.
struct OpClass {
  QN shift{0, 0};
  int parity = 0;
  int nops = 0;
  std::vector<int> blk_in, blk_out;
  std::vector<long long> blk_off;
  std::vector<int> in2blk;
  long long nnz = 0;
  double *d = nullptr;
  int *d_in2blk = nullptr, *d_blk_out = nullptr;
  long long *d_blk_off = nullptr;
};

struct Ref {
  int cls = -1;   // -1 = zero operator
  int idx = 0;
};

using PairKey = std::pair<int, int>;

// Spin-adapted (U(1)xSU(2)) operators are SU(2) tensors; a tensor is named
// by its kind (0 H, 1 c~, 2 S~, 3 A~, 4 B, 5 P, 6 Q, as the spin-orbital
// OpSpec kinds), spatial indices and twice its rank.
struct TKey {
  int kind = 0, i = 0, j = 0, tk = 0;
  bool operator<(const TKey &o) const {
    if (kind != o.kind) return kind < o.kind;
    if (i != o.i) return i < o.i;
    if (j != o.j) return j < o.j;
    return tk < o.tk;
  }
  bool operator==(const TKey &o) const {
    return kind == o.kind && i == o.i && j == o.j && tk == o.tk;
  }
  int parity() const { return (kind == 1 || kind == 2) ? 1 : 0; }
};

// A tensor of rank k stored as its spin-change components J' - J = -k..k:
// r[(2(J'-J) + 2k) / 2], each a block-sparse operator of one class.
struct TRef {
  int tk = 0;
  Ref r[3];
};

// A renormalized block, an enlarged block (block x site) or the vacuum.
struct BlockPart {
  Basis basis;
  std::vector<int> modes;
  std::vector<OpClass> cls;
  Ref H;
  std::map<int, Ref> c, S;
  std::map<PairKey, Ref> cc, cdc, P, Q;
  std::map<TKey, TRef> ten;   // spin-adapted parts: all operators as tensors
  // HBM staging of renormalized blocks: 0 resident, 1 offloaded (class data
  // only in pinned host memory, host[c] per class), 2 released (stale: rebuilt
  // before any further use; host metadata kept)
  int state = 0;
  std::vector<double *> host;
  // enlarged blocks only
  bool enlarged = false;
  int site_first = 0;
  std::vector<std::vector<Piece>> pieces;
  long long bytes() const {
    long long b = 0;
    for (auto &c : cls) b += c.nnz * c.nops * 8;
    return b;
  }
};

// Exact operators of one site (1 or 2 modes): d x d matrix stored in a
// 4 x 4 row-major frame, m[i*4 + j] (unused rows/columns are zero).
struct SiteOp {
  QN shift{0, 0};
  int parity = 0;
  double m[16] = {0};
};

// Reduced matrix of a site tensor between the site multiplets (3 x 3 used in
// the 4 x 4 frame, m[so*4 + si]).
struct SiteTen {
  int tk = 0;
  int parity = 0;
  double m[16] = {0};
};

struct SitePart {
  int site = 0;
  int d = 2;
  std::vector<int> modes;
  std::vector<QN> sq;   // QN of each site state (ordered by QN)
  SiteOp H, I;
  std::map<int, SiteOp> c, S;
  std::map<PairKey, SiteOp> cc, cdc, P, Q;
  std::map<TKey, SiteTen> ten;   // spin-adapted site: multiplets {0}, {up,dn}, {updn}
  std::vector<int> tj;           // spin-adapted site: twice the spin of each multiplet
};

// Factor of an operator product: block op / block identity / site matrix.
struct Fac {
  int kind = 0;        // 0 zero, 1 block ref, 2 block identity, 3 site op
  Ref ref;
  int trans = 0;
  double scale = 1.0;
  SiteOp so;           // kind 3 (already transposed if trans)
  QN shift{0, 0};
  int parity = 0;
};

}  // namespace dmrg
