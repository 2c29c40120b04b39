"""Two-site DMRG with normal and complementary block operators (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper runs DMRG on the generic Hamiltonian of Eq. 1 with an MPS (Eq. 4)
and states that the effective-Hamiltonian diagonalisation dominates the cost
(Sec. II.A) and that a sweep costs D^3 N^3 (Sec. III.A, citing White-1999).
It does not spell out the block-operator algebra; this module writes out the
textbook normal / complementary operator form that has that cost.

Spin-orbital modes (see hamiltonian.py), h and antisymmetric W.  For a part Z
of the chain and modes x, z outside Z:
  c_x            annihilator, x in Z                              (normal)
  S^Z_y          1/2 sum_{q in Z} h_yq c_q
                 + 2 sum_{q,r,t in Z} W_yqrt c^+_q c_r c_t         (complementary)
  cc_pq = c_p c_q (p<q in Z),  cdc_pr = c^+_p c_r (p,r in Z)      (normal pairs)
  P^Z_xz = sum_{a,b in Z} W_xzab c_a c_b      (x<z not in Z)    (complementary)
  Q^Z_xz = sum_{a,b in Z} W_xazb c^+_a c_b    (x,z not in Z)    (complementary)
For two parts F (first) and G (second) the Hamiltonian restricted to F u G is
  H = H^F + H^G + sum_{x in F} (c^+_x S^G_x + h.c.)
      + sum_{y in G} ((S^F_y)^+ c_y + h.c.)
      + sum_{x<z in F} (2 (c^+_x c^+_z) P^G_xz + h.c.)
      - 4 sum_{x,z in F} (c^+_x c_z) Q^G_xz,
where every product is written with the F factor on the left.  This is used
both to build enlarged blocks (block + site) and as H_eff at a cut.  This
oracle keeps the normal AND the complementary pairs on every block (the
simplest policy; it is slower than necessary but needs no switching).
"""
import numpy as np
import scipy.sparse.linalg as spla

from .blocks import (Basis, Op, identity, kron, n_of, qadd, qsub,
                     renormalize, union_basis, zero_op)


class Model:
    """Chain of sites with their spin-orbital modes and the target sector."""

    def __init__(self, h, W, spinful, target):
        self.h = h
        self.W = W
        self.spinful = spinful
        self.M = h.shape[0]
        self.n_sites = self.M // 2 if spinful else self.M
        self.target = tuple(target)
        self.nq = 2 if spinful else 1

    def site_modes(self, i):
        return [2 * i, 2 * i + 1] if self.spinful else [i]

    def shift_c(self, p):
        """QN shift of c_p."""
        if not self.spinful:
            return (-1,)
        return (-1, 0) if p % 2 == 0 else (0, -1)

    def zero(self):
        return tuple(0 for _ in range(self.nq))

    def allowed_left(self, n_left_sites):
        cap = self.n_sites - n_left_sites
        return lambda q: all(0 <= t - x <= cap for t, x in zip(self.target, q))

    def allowed_right(self, first_site):
        cap = first_site
        return lambda q: all(0 <= t - x <= cap for t, x in zip(self.target, q))


class Part:
    """A block or a site together with all its operator families."""

    def __init__(self, basis, modes):
        self.basis = basis
        self.modes = list(modes)
        self.H = None
        self.c = {}
        self.S = {}
        self.cc = {}
        self.cdc = {}
        self.P = {}
        self.Q = {}

    def Pget(self, x, z, model):
        if x == z:
            return zero_op(qadd(model.shift_c(x), model.shift_c(z)), 0)
        if x < z:
            return self.P[(x, z)]
        return self.P[(z, x)].scaled(-1.0)

    def ident(self):
        return identity(self.basis)


def vacuum_part(model):
    z = model.zero()
    part = Part(Basis([(z, 1)]), [])
    part.H = Op(z, 0, {z: np.zeros((1, 1))})
    others = list(range(model.M))
    for y in others:
        part.S[y] = zero_op(model.shift_c(y), 1)
    for i, x in enumerate(others):
        for z2 in others[i + 1:]:
            part.P[(x, z2)] = zero_op(qadd(model.shift_c(x), model.shift_c(z2)), 0)
    for x in others:
        for z2 in others:
            part.Q[(x, z2)] = zero_op(qsub(model.shift_c(x), model.shift_c(z2)), 0)
    return part


def site_part(model, i):
    """Exact operator families of one site (its 1 or 2 modes)."""
    m = model.site_modes(i)
    k = len(m)
    d = 2 ** k

    def qn(b):
        if not model.spinful:
            return (bin(b).count("1"),)
        return (b & 1, (b >> 1) & 1)
    order = sorted(range(d), key=qn)          # site basis = states sorted by QN
    pos = {b: n for n, b in enumerate(order)}
    cl = {}
    for j, p in enumerate(m):
        C = np.zeros((d, d))
        for b in range(d):
            if (b >> j) & 1:
                sgn = (-1) ** bin(b & ((1 << j) - 1)).count("1")
                C[pos[b & ~(1 << j)], pos[b]] = sgn
        cl[p] = C
    qns = [qn(b) for b in order]
    B = Basis([(q, 1) for q in qns])

    def to_op(Mat, shift, parity):
        blocks = {}
        for jj, qj in enumerate(qns):
            qo = qadd(qj, shift)
            if qo in B.index:
                ii = qns.index(qo)
                blocks[qj] = np.array([[Mat[ii, jj]]])
        chk = Op(shift, parity, blocks).dense(B)
        assert np.allclose(chk, Mat, atol=1e-13), "site operator shift mismatch"
        return Op(shift, parity, blocks)

    h, W = model.h, model.W
    part = Part(B, m)
    Hs = np.zeros((d, d))
    for p in m:
        for q in m:
            Hs += h[p, q] * cl[p].T @ cl[q]
    for p in m:
        for q in m:
            for r in m:
                for s in m:
                    if W[p, q, r, s] != 0.0:
                        Hs += W[p, q, r, s] * cl[p].T @ cl[q].T @ cl[r] @ cl[s]
    part.H = to_op(Hs, model.zero(), 0)
    for p in m:
        part.c[p] = to_op(cl[p], model.shift_c(p), 1)
    for a in range(k):
        for b in range(a + 1, k):
            p, q = m[a], m[b]
            part.cc[(p, q)] = to_op(cl[p] @ cl[q], qadd(model.shift_c(p), model.shift_c(q)), 0)
    for p in m:
        for r in m:
            part.cdc[(p, r)] = to_op(cl[p].T @ cl[r], qsub(model.shift_c(r), model.shift_c(p)), 0)
    others = [y for y in range(model.M) if y not in m]
    for y in others:
        Sm = np.zeros((d, d))
        for q in m:
            Sm += 0.5 * h[y, q] * cl[q]
        for q in m:
            for r in m:
                for t in m:
                    if W[y, q, r, t] != 0.0:
                        Sm += 2.0 * W[y, q, r, t] * cl[q].T @ cl[r] @ cl[t]
        part.S[y] = to_op(Sm, model.shift_c(y), 1)
    for ii, x in enumerate(others):
        for z in others[ii + 1:]:
            Pm = np.zeros((d, d))
            for a in m:
                for b in m:
                    Pm += W[x, z, a, b] * cl[a] @ cl[b]
            part.P[(x, z)] = to_op(Pm, qadd(model.shift_c(x), model.shift_c(z)), 0)
    for x in others:
        for z in others:
            Qm = np.zeros((d, d))
            for a in m:
                for b in m:
                    Qm += W[x, a, z, b] * cl[a].T @ cl[b]
            part.Q[(x, z)] = to_op(Qm, qsub(model.shift_c(x), model.shift_c(z)), 0)
    return part


def cross_terms(F, G, model):
    """Terms (A on F, B on G, coef) of H^{FuG} - H^F - H^G (F normal side).

    Hermitian conjugates are listed explicitly: the adjoint of the product
    A_F B_G is (-1)^(p(A) p(B)) A^+_F B^+_G.
    """
    terms = []

    def with_hc(A, B, c):
        terms.append((A, B, c))
        sgn = -1.0 if (A.parity and B.parity) else 1.0
        terms.append((A.dagger(), B.dagger(), c * sgn))

    for x in F.modes:
        with_hc(F.c[x].dagger(), G.S[x], 1.0)
    for y in G.modes:
        with_hc(F.S[y].dagger(), G.c[y], 1.0)
    Fm = F.modes
    for i, x in enumerate(Fm):
        for z in Fm[i + 1:]:
            # c^+_x c^+_z = -(c_x c_z)^+
            with_hc(F.cc[(x, z)].dagger().scaled(-1.0), G.Pget(x, z, model), 2.0)
    for x in Fm:
        for z in Fm:
            terms.append((F.cdc[(x, z)], G.Q[(x, z)], -4.0))
    return terms


def combine(terms, U, shift, parity):
    out = zero_op(shift, parity)
    for A, B, c in terms:
        out.add(kron(A, B, U), c)
    return out


def union(F, G, model, site_is_first, allowed):
    """Operator families of the two-part block F u G (F first)."""
    U = union_basis(F.basis, G.basis, site_is_first, allowed)
    part = Part(U, F.modes + G.modes)
    IF, IG = F.ident(), G.ident()
    in_u = set(part.modes)
    out_modes = [y for y in range(model.M) if y not in in_u]

    part.H = combine([(F.H, IG, 1.0), (IF, G.H, 1.0)] + cross_terms(F, G, model),
                     U, model.zero(), 0)
    for x in F.modes:
        part.c[x] = kron(F.c[x], IG, U)
    for x in G.modes:
        part.c[x] = kron(IF, G.c[x], U)
    for (p, q), op in F.cc.items():
        part.cc[(p, q)] = kron(op, IG, U)
    for (p, q), op in G.cc.items():
        part.cc[(p, q)] = kron(IF, op, U)
    for p in F.modes:
        for q in G.modes:
            part.cc[(p, q)] = kron(F.c[p], G.c[q], U)
    for (p, r), op in F.cdc.items():
        part.cdc[(p, r)] = kron(op, IG, U)
    for (p, r), op in G.cdc.items():
        part.cdc[(p, r)] = kron(IF, op, U)
    for p in F.modes:
        for r in G.modes:
            part.cdc[(p, r)] = kron(F.c[p].dagger(), G.c[r], U)
            part.cdc[(r, p)] = kron(F.c[p], G.c[r].dagger(), U).scaled(-1.0)
    cc_FG = {(a, b): kron(F.c[a], G.c[b], U) for a in F.modes for b in G.modes}
    cdc_FG = {(a, b): kron(F.c[a].dagger(), G.c[b], U) for a in F.modes for b in G.modes}
    ccd_FG = {(b, a): kron(F.c[b], G.c[a].dagger(), U) for b in F.modes for a in G.modes}
    W = model.W
    for y in out_modes:
        S = kron(F.S[y], IG, U).add(kron(IF, G.S[y], U))
        for t in G.modes:
            S.add(kron(F.Q[(y, t)], G.c[t], U), -4.0)
        for t in F.modes:
            S.add(kron(F.c[t], G.Q[(y, t)], U), -4.0)
        for q in F.modes:
            S.add(kron(F.c[q].dagger(), G.Pget(y, q, model), U), 2.0)
        for q in G.modes:
            S.add(kron(F.Pget(y, q, model), G.c[q].dagger(), U), 2.0)
        part.S[y] = S
    for i, x in enumerate(out_modes):
        for z in out_modes[i + 1:]:
            P = kron(F.P[(x, z)], IG, U).add(kron(IF, G.P[(x, z)], U))
            for a in F.modes:
                for b in G.modes:
                    if W[x, z, a, b] != 0.0:
                        P.add(cc_FG[(a, b)], 2.0 * W[x, z, a, b])
            part.P[(x, z)] = P
    for x in out_modes:
        for z in out_modes:
            Q = kron(F.Q[(x, z)], IG, U).add(kron(IF, G.Q[(x, z)], U))
            for a in F.modes:
                for b in G.modes:
                    if W[x, a, z, b] != 0.0:
                        Q.add(cdc_FG[(a, b)], W[x, a, z, b])
            for a in G.modes:
                for b in F.modes:
                    if W[x, a, z, b] != 0.0:
                        Q.add(ccd_FG[(b, a)], -W[x, a, z, b])
            part.Q[(x, z)] = Q
    return part


def renormalize_part(part, T, newbasis):
    out = Part(newbasis, part.modes)
    out.H = renormalize(part.H, T, newbasis)
    for name in ("c", "S", "cc", "cdc", "P", "Q"):
        src = getattr(part, name)
        setattr(out, name, {k: renormalize(v, T, newbasis) for k, v in src.items()})
    return out


def basis_from_isometry(T):
    return Basis([(q, m.shape[1]) for q, m in T.items()])


class Window:
    """Two-site window (l, l+1): L. = L_l u site_l, .R = site_{l+1} u R_{l+2}."""

    def __init__(self, model, left, right, l):
        self.model = model
        self.l = l
        self.Ld = union(left, site_part(model, l), model, False,
                        model.allowed_left(l + 1))
        self.Rd = union(site_part(model, l + 1), right, model, True,
                        model.allowed_right(l + 1))
        self.terms = ([(self.Ld.H, self.Rd.ident(), 1.0),
                       (self.Ld.ident(), self.Rd.H, 1.0)]
                      + cross_terms(self.Ld, self.Rd, model))
        self.layout = []
        off = 0
        for qa, da in zip(self.Ld.basis.qns, self.Ld.basis.dims):
            qb = qsub(model.target, qa)
            db = self.Rd.basis.dim(qb)
            if db > 0:
                self.layout.append((qa, qb, off, da, db))
                off += da * db
        self.size = off
        self._qa = {x[0] for x in self.layout}

    def unpack(self, v):
        return {qa: v[o:o + da * db].reshape(da, db) for qa, qb, o, da, db in self.layout}

    def pack(self, blocks):
        v = np.zeros(self.size)
        for qa, qb, o, da, db in self.layout:
            if qa in blocks:
                v[o:o + da * db] = blocks[qa].ravel()
        return v

    def apply(self, v):
        """sigma = H_eff psi = sum_k coef_k (A_k x B_k) psi  (sector by sector)."""
        psi = self.unpack(v)
        sig = {qa: np.zeros((da, db)) for qa, qb, o, da, db in self.layout}
        for A, B, c in self.terms:
            for qa, qb, o, da, db in self.layout:
                a = A.blocks.get(qa)
                b = B.blocks.get(qb)
                if a is None or b is None:
                    continue
                qa2 = qadd(qa, A.shift)
                if qa2 not in sig:
                    continue
                sgn = -1.0 if (B.parity and (n_of(qa) & 1)) else 1.0
                sig[qa2] += (c * sgn) * (a @ psi[qa] @ b.T)
        return self.pack(sig)

    def solve(self, tol=1e-10, v0=None, seed=0):
        n = self.size
        if n <= 400:
            Hm = np.empty((n, n))
            eye = np.eye(n)
            for j in range(n):
                Hm[:, j] = self.apply(eye[:, j])
            w, V = np.linalg.eigh(0.5 * (Hm + Hm.T))
            return w[0], V[:, 0]
        op = spla.LinearOperator((n, n), matvec=self.apply, dtype=float)
        if v0 is None:
            v0 = np.random.default_rng(seed).standard_normal(n)
        w, V = spla.eigsh(op, k=1, which="SA", tol=tol, v0=v0, ncv=24)
        return w[0], V[:, 0]

    def truncate(self, v, D, side):
        """Keep the D largest Schmidt values over all sectors.

        Ties break by lower sector index, then lower in-sector index.
        side='left' returns the isometry L. -> L_{l+1}; 'right' .R -> R_{l+1}.
        Also returns the discarded weight and the block entropy.
        """
        psi = self.unpack(v)
        cand = []
        svd = {}
        for si, (qa, qb, o, da, db) in enumerate(self.layout):
            Uu, s, Vt = np.linalg.svd(psi[qa], full_matrices=False)
            svd[qa] = (Uu, s, Vt)
            for k, val in enumerate(s):
                cand.append((-val, si, k))
        cand.sort()
        keep = cand[:D]
        kept = {}
        for _, si, k in keep:
            kept.setdefault(si, []).append(k)
        T = {}
        for si, ks in kept.items():
            qa, qb, o, da, db = self.layout[si]
            Uu, s, Vt = svd[qa]
            ks = sorted(ks)
            if side == "left":
                T[qa] = Uu[:, ks]
            else:
                T[qb] = Vt[ks, :].T
        allw = np.array([c[0] ** 2 for c in cand])
        kw = np.array([c[0] ** 2 for c in keep])
        disc = float(allw.sum() - kw.sum())
        p = kw / kw.sum()
        p = p[p > 0]
        ent = float(-(p * np.log(p)).sum())
        return T, disc, ent


def left_blocks(model, left_iso, upto):
    """L_0 .. L_upto from left isometries left_iso[n]: L_{n-1}. -> L_n."""
    L = [vacuum_part(model)]
    for n in range(1, upto + 1):
        Ld = union(L[-1], site_part(model, n - 1), model, False, model.allowed_left(n))
        T = left_iso[n]
        L.append(renormalize_part(Ld, T, basis_from_isometry(T)))
    return L


def right_blocks(model, right_iso, downto):
    """R_N .. R_downto from right isometries right_iso[n]: .R_{n+1} -> R_n."""
    N = model.n_sites
    R = {N: vacuum_part(model)}
    for n in range(N - 1, downto - 1, -1):
        Rd = union(site_part(model, n), R[n + 1], model, True, model.allowed_right(n))
        T = right_iso[n]
        R[n] = renormalize_part(Rd, T, basis_from_isometry(T))
    return R


def window_from_mps(model, left_iso, right_iso, l):
    L = left_blocks(model, left_iso, l)
    R = right_blocks(model, right_iso, l + 2)
    return Window(model, L[l], R[l + 2], l)


def sweep(model, right_iso, D, n_sweeps, tol=1e-10, log=None):
    """Two-site DMRG sweeps from a right-canonical start.

    One sweep = windows l = 0..N-2 left to right (truncating to the left after
    each window except the last), then l = N-2..0 right to left (truncating to
    the right after each window except the last).  Returns per-sweep energies
    (energy of the final window of the sweep) and the per-window history.
    """
    N = model.n_sites
    R = right_blocks(model, right_iso, 2)
    L = {0: vacuum_part(model)}
    energies, hist = [], []
    for sw in range(n_sweeps):
        for l in range(0, N - 1):
            w = Window(model, L[l], R[l + 2], l)
            e, v = w.solve(tol=tol, seed=1000 * sw + l)
            hist.append((sw, "lr", l, e))
            if l < N - 2:
                T, disc, ent = w.truncate(v, D, "left")
                L[l + 1] = renormalize_part(w.Ld, T, basis_from_isometry(T))
        for l in range(N - 2, -1, -1):
            w = Window(model, L[l], R[l + 2], l)
            e, v = w.solve(tol=tol, seed=1000 * sw + 500 + l)
            hist.append((sw, "rl", l, e))
            if l > 0:
                T, disc, ent = w.truncate(v, D, "right")
                R[l + 1] = renormalize_part(w.Rd, T, basis_from_isometry(T))
        energies.append(e)
        if log:
            log(sw, e)
    return energies, hist
