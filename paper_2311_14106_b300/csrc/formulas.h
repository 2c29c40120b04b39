// Normal / complementary operator formulas of two-site ab initio DMRG.
//
// The paper (Sec. II.A) states that H_eff is assembled from renormalized
// block operators and that a sweep costs D^3 N^3 (Sec. III.A); the
// operator algebra below is the textbook form with that cost.  Spin-orbital
// modes, h and the antisymmetrised W of Eq. 1.  For a part Z and modes
// x, z outside Z:
//   S^Z_y  = 1/2 sum_{q in Z} h_yq c_q + 2 sum_{q,r,t in Z} W_yqrt c+_q c_r c_t
//   P^Z_xz = sum_{a,b in Z} W_xzab c_a c_b
//   Q^Z_xz = sum_{a,b in Z} W_xazb c+_a c_b
// and normal operators c_x, cc_pq = c_p c_q (p < q), cdc_pr = c+_p c_r on Z.
// For two parts F (first in the Jordan-Wigner order) and G (second), each
// product is written with the F factor on the left; the adjoint of a product
// A_F B_G is (-1)^(p(A) p(B)) A^T_F B^T_G.  The pair terms use the part with
// fewer modes as the "normal" side (ties: F).
#pragma once
#include <functional>

#include "model.h"

namespace dmrg {

struct Side {
  const BlockPart *b = nullptr;
  const SitePart *s = nullptr;
  QN shift_c(int p, bool spinful) const {
    if (!spinful) return {-1, 0};
    return (p % 2 == 0) ? QN{-1, 0} : QN{0, -1};
  }
  const std::vector<int> &modes() const { return b ? b->modes : s->modes; }
  int nmodes() const { return (int)modes().size(); }

  Fac from_ref(const Ref &r, double scale = 1.0) const {
    Fac f;
    if (r.cls < 0) return f;
    f.kind = 1;
    f.ref = r;
    f.scale = scale;
    f.shift = b->cls[r.cls].shift;
    f.parity = b->cls[r.cls].parity;
    return f;
  }
  static Fac from_site(const SiteOp &o, double scale = 1.0) {
    Fac f;
    f.kind = 3;
    f.so = o;
    f.scale = scale;
    f.shift = o.shift;
    f.parity = o.parity;
    return f;
  }
  template <class K>
  Fac bget(const std::map<K, Ref> &m, const K &k, double scale = 1.0) const {
    auto it = m.find(k);
    return it == m.end() ? Fac() : from_ref(it->second, scale);
  }
  template <class K>
  Fac sget(const std::map<K, SiteOp> &m, const K &k, double scale = 1.0) const {
    auto it = m.find(k);
    return it == m.end() ? Fac() : from_site(it->second, scale);
  }
  Fac c(int x) const { return b ? bget(b->c, x) : sget(s->c, x); }
  Fac S(int y) const { return b ? bget(b->S, y) : sget(s->S, y); }
  Fac cc(int p, int q) const {
    PairKey k{p, q};
    return b ? bget(b->cc, k) : sget(s->cc, k);
  }
  Fac cdc(int p, int r) const {
    PairKey k{p, r};
    return b ? bget(b->cdc, k) : sget(s->cdc, k);
  }
  Fac P(int x, int z) const {
    if (x == z) return Fac();
    double sc = x < z ? 1.0 : -1.0;
    PairKey k{x < z ? x : z, x < z ? z : x};
    return b ? bget(b->P, k, sc) : sget(s->P, k, sc);
  }
  Fac Q(int x, int z) const {
    PairKey k{x, z};
    return b ? bget(b->Q, k) : sget(s->Q, k);
  }
  Fac H() const { return b ? from_ref(b->H) : from_site(s->H); }
  Fac I() const {
    if (s) return from_site(s->I);
    Fac f;
    f.kind = 2;
    return f;
  }
};

inline Fac transpose(const Fac &f) {
  Fac t = f;
  t.trans ^= 1;
  t.shift = qneg(f.shift);
  if (f.kind == 3) {
    t.so.shift = qneg(f.so.shift);
    // site matrices live in a 4 x 4 frame whatever the site dimension
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) t.so.m[i * 4 + j] = f.so.m[j * 4 + i];
  }
  return t;
}

using AddFn = std::function<void(const Fac &, const Fac &, double)>;

// The formulas below are templates over the part type (Side: spin-orbital
// operators of the U(1) and U(1)xU(1) code; SideS in su2.h: spin-adapted
// tensors) and the callback add(A, B, coef) that receives every product.
template <class AddF, class FacT>
void add_hc(const AddF &add, const FacT &A, const FacT &B, double c) {
  add(A, B, c);
  add(transpose(A), transpose(B), (A.parity & B.parity) ? -c : c);
}

// Cross terms of H^{F u G} - H^F - H^G (plus H^F x 1 and 1 x H^G if whole).
template <class SideT, class AddF>
void formula_H(const SideT &F, const SideT &G, const AddF &add, bool whole) {
  if (whole) {
    add(F.H(), G.I(), 1.0);
    add(F.I(), G.H(), 1.0);
  }
  for (int x : F.modes()) add_hc(add, transpose(F.c(x)), G.S(x), 1.0);
  for (int y : G.modes()) add_hc(add, transpose(F.S(y)), G.c(y), 1.0);
  const bool f_normal = F.nmodes() <= G.nmodes();
  if (f_normal) {
    const auto &fm = F.modes();
    for (size_t i = 0; i < fm.size(); ++i)
      for (size_t j = i + 1; j < fm.size(); ++j)
        add_hc(add, transpose(F.cc(fm[i], fm[j])), G.P(fm[i], fm[j]), -2.0);
    for (int x : fm)
      for (int z : fm) add(F.cdc(x, z), G.Q(x, z), -4.0);
  } else {
    const auto &gm = G.modes();
    for (size_t i = 0; i < gm.size(); ++i)
      for (size_t j = i + 1; j < gm.size(); ++j)
        add_hc(add, transpose(F.P(gm[i], gm[j])), G.cc(gm[i], gm[j]), -2.0);
    for (int x : gm)
      for (int z : gm) add(F.Q(x, z), G.cdc(x, z), -4.0);
  }
}

inline bool has(const std::vector<int> &v, int x) {
  for (int y : v)
    if (y == x) return true;
  return false;
}

template <class SideT, class AddF>
void formula_c(const SideT &F, const SideT &G, int x, const AddF &add) {
  if (has(F.modes(), x)) add(F.c(x), G.I(), 1.0);
  else add(F.I(), G.c(x), 1.0);
}

template <class SideT, class AddF>
void formula_S(const SideT &F, const SideT &G, int y, const AddF &add) {
  add(F.S(y), G.I(), 1.0);
  add(F.I(), G.S(y), 1.0);
  for (int t : G.modes()) add(F.Q(y, t), G.c(t), -4.0);
  for (int t : F.modes()) add(F.c(t), G.Q(y, t), -4.0);
  for (int q : F.modes()) add(transpose(F.c(q)), G.P(y, q), 2.0);
  for (int q : G.modes()) add(F.P(y, q), transpose(G.c(q)), 2.0);
}

template <class SideT, class AddF>
void formula_cc(const SideT &F, const SideT &G, int p, int q, const AddF &add) {
  bool pf = has(F.modes(), p), qf = has(F.modes(), q);
  if (pf && qf) add(F.cc(p, q), G.I(), 1.0);
  else if (!pf && !qf) add(F.I(), G.cc(p, q), 1.0);
  else add(F.c(p), G.c(q), 1.0);   // p < q, so p in F and q in G
}

template <class SideT, class AddF>
void formula_cdc(const SideT &F, const SideT &G, int p, int r, const AddF &add) {
  bool pf = has(F.modes(), p), rf = has(F.modes(), r);
  if (pf && rf) add(F.cdc(p, r), G.I(), 1.0);
  else if (!pf && !rf) add(F.I(), G.cdc(p, r), 1.0);
  else if (pf) add(transpose(F.c(p)), G.c(r), 1.0);
  else add(F.c(r), transpose(G.c(p)), -1.0);
}

template <class SideT, class AddF>
void formula_P(const SideT &F, const SideT &G, int x, int z, const double *W, int M,
               const AddF &add) {
  add(F.P(x, z), G.I(), 1.0);
  add(F.I(), G.P(x, z), 1.0);
  for (int a : F.modes())
    for (int b : G.modes()) {
      double w = W[(((long long)x * M + z) * M + a) * M + b];
      if (w != 0.0) add(F.c(a), G.c(b), 2.0 * w);
    }
}

template <class SideT, class AddF>
void formula_Q(const SideT &F, const SideT &G, int x, int z, const double *W, int M,
               const AddF &add) {
  add(F.Q(x, z), G.I(), 1.0);
  add(F.I(), G.Q(x, z), 1.0);
  for (int a : F.modes())
    for (int b : G.modes()) {
      double w = W[(((long long)x * M + a) * M + z) * M + b];
      if (w != 0.0) add(transpose(F.c(a)), G.c(b), w);
    }
  for (int a : G.modes())
    for (int b : F.modes()) {
      double w = W[(((long long)x * M + a) * M + z) * M + b];
      if (w != 0.0) add(F.c(b), transpose(G.c(a)), -w);
    }
}

}  // namespace dmrg
