// U(1)xSU(2) spin adaptation of the block operators (Sec. IV: the Hubbard
// runs keep D SU(2) multiplets).
//
// Sectors are spin multiplets (N, 2J), labelled internally by the (N_up,
// N_dn) of their highest-weight member, ((N + 2J)/2, (N - 2J)/2): particle
// number, parity and QN shifts then work as in the U(1)xU(1) code.  Every
// stored operator is an SU(2) tensor of rank k with reduced matrix elements
// R(j' <- j), defined by <j' m'| T_q |j m> = <j m k q | j' m'> R(j' <- j).
// A tensor of rank k is kept as up to 2k+1 "components", one per spin change
// J' - J (each a block-sparse operator with a definite QN shift), so that the
// sector tables, renormalisation and H_eff stacks of the U(1) code apply
// unchanged; the recoupling scalars enter as per-block coefficients.
//
// Tensors of a part Z (modes x, z outside Z; p, q, r in Z; m = +-1/2):
//   c~_p   [c~]_{+1/2} = c_{p dn}, [c~]_{-1/2} = -c_{p up}          rank 1/2
//   S~_y   the same combination of the complementary S_{y sigma}     rank 1/2
//   A~^k_pq = [c~_p x c~_q]^k  (p <= q; k = 0 only for p = q)          k = 0, 1
//   B^k_pr  = [c+_p x c~_r]^k                                           k = 0, 1
//   P^k_xz, Q^k_xz   the complementary pair operators coupled alike     k = 0, 1
//   H (scalar)
// where [X x Y]^k_M = sum <1/2 m1 1/2 m2 | k M> X_m1 Y_m2 and every
// spin-orbital operator is a fixed combination of tensor components (see
// the decomposition in SideS).  The formulas of the enlarged blocks and of
// H_eff are the spin-orbital ones of formulas.h: evaluating one component of
// a target tensor through them and projecting every product of components
// onto the coupled form [X^kx (x) Y^ky]^k gives the spin-adapted formula.
#pragma once
#include <array>
#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "model.h"

namespace dmrg {
namespace su2 {

// ---------------------------------------------------------------------------
// Clebsch-Gordan coefficients, Racah's closed form (doubled arguments)
// ---------------------------------------------------------------------------
inline long double lfact(int n) {
  static std::vector<long double> f = [] {
    std::vector<long double> v(200, 1.0L);
    for (int i = 1; i < 200; ++i) v[i] = v[i - 1] * i;
    return v;
  }();
  return f[n];
}

inline double cg_raw(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
  if (tm1 + tm2 != tM) return 0.0;
  if (tJ < std::abs(tj1 - tj2) || tJ > tj1 + tj2 || ((tj1 + tj2 + tJ) & 1)) return 0.0;
  if (std::abs(tm1) > tj1 || std::abs(tm2) > tj2 || std::abs(tM) > tJ) return 0.0;
  if (((tj1 + tm1) & 1) || ((tj2 + tm2) & 1) || ((tJ + tM) & 1)) return 0.0;
  const int a = (tj1 + tj2 - tJ) / 2, b = (tj1 - tj2 + tJ) / 2, c = (-tj1 + tj2 + tJ) / 2;
  const int d = (tj1 + tj2 + tJ) / 2 + 1;
  long double pref = (tJ + 1) * lfact(a) * lfact(b) * lfact(c) / lfact(d);
  pref *= lfact((tJ + tM) / 2) * lfact((tJ - tM) / 2) * lfact((tj1 - tm1) / 2) *
          lfact((tj1 + tm1) / 2) * lfact((tj2 - tm2) / 2) * lfact((tj2 + tm2) / 2);
  long double s = 0.0L;
  for (int k = 0; k <= a; ++k) {
    const int e[6] = {k, a - k, (tj1 - tm1) / 2 - k, (tj2 + tm2) / 2 - k,
                      (tJ - tj2 + tm1) / 2 + k, (tJ - tj1 - tm2) / 2 + k};
    bool ok = true;
    long double den = 1.0L;
    for (int x : e) {
      if (x < 0) {
        ok = false;
        break;
      }
      den *= lfact(x);
    }
    if (ok) s += ((k & 1) ? -1.0L : 1.0L) / den;
  }
  return (double)(s * std::sqrt(pref));
}

// Cached per host thread (no lock: concurrent solves run on their own
// threads and each fills its own small table).
inline double cg(int tj1, int tm1, int tj2, int tm2, int tJ, int tM) {
  thread_local std::unordered_map<unsigned long long, double> cache;
  auto enc = [](int x) { return (unsigned long long)(x + 128) & 0xff; };
  const unsigned long long key = enc(tj1) | enc(tm1) << 8 | enc(tj2) << 16 | enc(tm2) << 24 |
                                 enc(tJ) << 32 | enc(tM) << 40;
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const double v = cg_raw(tj1, tm1, tj2, tm2, tJ, tM);
  cache.emplace(key, v);
  return v;
}

// K of a coupled product of tensors on two parts F (first) and G:
//   <(jF' jG') J' M'| [X^kF (x) Y^kG]^k_q |(jF jG) J M>
//     = <J M k q | J' M'> K R_X(jF' <- jF) R_Y(jG' <- jG)
// (fermion sign aside), evaluated by summing the Clebsch-Gordan products at
// M' = J' and projecting with sum_{M,q} <J M k q | J' J'>^2 = 1.
inline double coupling_raw(int tjF, int tjG, int tJ, int tjFp, int tjGp, int tJp, int tkF,
                           int tkG, int tk) {
  double K = 0.0;
  for (int tM = -tJ; tM <= tJ; tM += 2) {
    const int tq = tJp - tM;
    if (std::abs(tq) > tk) continue;
    const double outer = cg(tJ, tM, tk, tq, tJp, tJp);
    if (outer == 0.0) continue;
    double inner = 0.0;
    for (int mF = -tjF; mF <= tjF; mF += 2) {
      const int mG = tM - mF;
      if (std::abs(mG) > tjG) continue;
      const double cin = cg(tjF, mF, tjG, mG, tJ, tM);
      if (cin == 0.0) continue;
      for (int qF = -tkF; qF <= tkF; qF += 2) {
        const int qG = tq - qF;
        if (std::abs(qG) > tkG) continue;
        const double cop = cg(tkF, qF, tkG, qG, tk, tq);
        if (cop == 0.0) continue;
        const int mFp = mF + qF, mGp = mG + qG;
        const double cout = cg(tjFp, mFp, tjGp, mGp, tJp, tJp);
        if (cout == 0.0) continue;
        inner += cout * cin * cop * cg(tjF, mF, tkF, qF, tjFp, mFp) * cg(tjG, mG, tkG, qG, tjGp, mGp);
      }
    }
    K += outer * inner;
  }
  return K;
}

inline double coupling(int tjF, int tjG, int tJ, int tjFp, int tjGp, int tJp, int tkF, int tkG,
                       int tk) {
  // cached per host thread; the doubled spins of a key fit in 7 bits each
  thread_local std::unordered_map<unsigned long long, double> cache;
  const int v9[9] = {tjF, tjG, tJ, tjFp, tjGp, tJp, tkF, tkG, tk};
  unsigned long long key = 0;
  bool fits = true;
  for (int i = 0; i < 9; ++i) {
    fits = fits && v9[i] >= 0 && v9[i] < 128;
    key = (key << 7) | (unsigned long long)(v9[i] & 127);
  }
  if (!fits) return coupling_raw(tjF, tjG, tJ, tjFp, tjGp, tJp, tkF, tkG, tk);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const double v = coupling_raw(tjF, tjG, tJ, tjFp, tjGp, tJp, tkF, tkG, tk);
  cache.emplace(key, v);
  return v;
}

// The adjoint tensor T^+ (components (T^+)_q = (-1)^(k-q) (T_{-q})^dagger, a
// proper rank-k tensor) has the reduced block (out <- in) =
// gamma(in, out, k) * [R_T block (in <- out)]^T with
//   gamma = (-1)^(j_in - j_out + k) sqrt((2 j_in + 1) / (2 j_out + 1)).
inline double adjoint_factor(int tj_in, int tj_out, int tk) {
  const int e = (tj_in - tj_out + tk) / 2;
  const double s = (e & 1) ? -1.0 : 1.0;
  return s * std::sqrt((tj_in + 1.0) / (tj_out + 1.0));
}

// <((L s) a' R) S M | (L (s R) b) S M>: recoupling of three spins from
// L x (s x R) to (L x s) x R, by Clebsch-Gordan sums at M = S.
inline double recouple(int tjL, int tjs, int tjR, int tja, int tjb, int tS) {
  double v = 0.0;
  for (int mL = -tjL; mL <= tjL; mL += 2)
    for (int ms = -tjs; ms <= tjs; ms += 2) {
      const int mR = tS - mL - ms;
      if (std::abs(mR) > tjR) continue;
      const int ma = mL + ms, mb = ms + mR;
      if (std::abs(ma) > tja || std::abs(mb) > tjb) continue;
      v += cg(tjL, mL, tjs, ms, tja, ma) * cg(tja, ma, tjR, mR, tS, tS) *
           cg(tjs, ms, tjR, mR, tjb, mb) * cg(tjL, mL, tjb, mb, tS, tS);
    }
  return v;
}

// (N, 2J) of an internal label
inline int tj_of(const QN &q) { return q[0] - q[1]; }
inline int n_of(const QN &q) { return q[0] + q[1]; }
inline QN label(int n, int tj) { return {(n + tj) / 2, (n - tj) / 2}; }

}  // namespace su2

// ---------------------------------------------------------------------------
// Spin-adapted operator references (TKey: model.h)
// ---------------------------------------------------------------------------

// One component of a linear combination of tensor components:
// a * (T or T^+)_q.
struct TComp {
  TKey key;
  int adj = 0;
  int tq = 0;
  double a = 0.0;
};

// A spin-orbital operator as such a combination (empty: zero).
struct SFac {
  std::vector<TComp> c;
  int parity = 0;
  int side = -1;   // identity marker kept for the block identity: kind 0, tk 0
};

inline double sgn_m(int tm) { return tm > 0 ? 1.0 : -1.0; }   // s_{+1/2} = 1, s_{-1/2} = -1

// Hermitian conjugate of every component: (T_q)^dagger = (-1)^(k+q) (T^+)_{-q},
// ((T^+)_q)^dagger = (-1)^(k+q) (-1)^(2k) T_{-q}.
inline SFac transpose(const SFac &f) {
  SFac t = f;
  for (TComp &x : t.c) {
    const int e = (x.key.tk + x.tq) / 2;
    double s = (e & 1) ? -1.0 : 1.0;
    if (x.adj && (x.key.tk & 1)) s = -s;
    x.a *= s;
    x.adj ^= 1;
    x.tq = -x.tq;
  }
  return t;
}

// Side of a spin-adapted product for the formulas of formulas.h: the same
// accessors as the spin-orbital Side (spin-orbital mode arguments p = 2i +
// (0 up, 1 down)), returning combinations of tensor components.  `has`
// tells whether a tensor is stored (non-zero) on this part.
struct SideS {
  std::vector<int> so_modes;                       // spin-orbital modes of the part
  std::function<bool(const TKey &)> has;
  const std::vector<int> &modes() const { return so_modes; }
  int nmodes() const { return (int)so_modes.size(); }
  static int sp(int p) { return p >> 1; }
  static int tm(int p) { return (p & 1) ? -1 : 1; }

  SFac one(const TKey &k, int tq, double a) const {
    SFac f;
    f.parity = k.parity();
    if (has(k)) f.c.push_back({k, 0, tq, a});
    return f;
  }
  // c_{i m} = s_{-m} [c~_i]_{-m}
  SFac c(int p) const { return one({1, sp(p), 0, 1}, -tm(p), sgn_m(-tm(p))); }
  SFac S(int p) const { return one({2, sp(p), 0, 1}, -tm(p), sgn_m(-tm(p))); }
  // products of two annihilation-like indices (cc, P): X_{(i,m1),(j,m2)} =
  // s_{-m1} s_{-m2} sum_k <1/2 -m1 1/2 -m2 | k -m1-m2> [X^k_ij]_{-m1-m2}
  SFac pair_aa(int kind, int p, int q) const {
    SFac f;
    f.parity = 0;
    const int i = sp(p), j = sp(q), m1 = tm(p), m2 = tm(q);
    if (i > j) return f;
    for (int tk = 0; tk <= 2; tk += 2) {
      if (i == j && tk == 2) continue;
      const double w = su2::cg(1, -m1, 1, -m2, tk, -m1 - m2) * sgn_m(-m1) * sgn_m(-m2);
      const TKey k{kind, i, j, tk};
      if (w != 0.0 && has(k)) f.c.push_back({k, 0, -m1 - m2, w});
    }
    return f;
  }
  SFac cc(int p, int q) const { return pair_aa(3, p, q); }
  SFac P(int x, int z) const {
    if (x == z) return SFac();
    if (sp(x) > sp(z) || (sp(x) == sp(z) && x > z)) {   // P_xz = -P_zx
      SFac f = pair_aa(5, z, x);
      for (auto &t : f.c) t.a = -t.a;
      return f;
    }
    return pair_aa(5, x, z);
  }
  // c+_{(i,m1)} c_{(j,m2)} = s_{-m2} sum_k <1/2 m1 1/2 -m2 | k m1-m2> [B^k_ij]_{m1-m2}
  SFac cdc(int p, int r) const {
    SFac f;
    const int i = sp(p), j = sp(r), m1 = tm(p), m2 = tm(r);
    for (int tk = 0; tk <= 2; tk += 2) {
      const double w = su2::cg(1, m1, 1, -m2, tk, m1 - m2) * sgn_m(-m2);
      const TKey k{4, i, j, tk};
      if (w != 0.0 && has(k)) f.c.push_back({k, 0, m1 - m2, w});
    }
    return f;
  }
  // Q_{(x,s),(z,t)} transforms like c+_{(z,t)} c_{(x,s)}:
  // = s_{-s} sum_k <1/2 t 1/2 -s | k t-s> [Q^k_xz]_{t-s}
  SFac Q(int x, int z) const {
    SFac f;
    const int i = sp(x), j = sp(z), ms = tm(x), mt = tm(z);
    for (int tk = 0; tk <= 2; tk += 2) {
      const double w = su2::cg(1, mt, 1, -ms, tk, mt - ms) * sgn_m(-ms);
      const TKey k{6, i, j, tk};
      if (w != 0.0 && has(k)) f.c.push_back({k, 0, mt - ms, w});
    }
    return f;
  }
  SFac H() const { return one({0, 0, 0, 0}, 0, 1.0); }
  SFac I() const {
    SFac f;
    f.c.push_back({TKey{-1, 0, 0, 0}, 0, 0, 1.0});   // kind -1: identity
    return f;
  }
};

}  // namespace dmrg
