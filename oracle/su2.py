"""U(1)xSU(2) spin adaptation, by exact expansion onto the U(1)xU(1) oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper runs its Hubbard calculations spin-adapted (Sec. IV, "Hubbard
model": non-Abelian U(1)xSU(2) symmetry, D counted in SU(2) multiplets, and
an equivalent U(1) dimension for comparison).  It does not write out the
spin-adapted algebra.  This module needs none of it: a spin-adapted basis is
a set of spin multiplets, and every multiplet state |beta J M> has an exact
image in the S_z (U(1)xU(1)) basis through Clebsch-Gordan coefficients.  With
E the isometric map from the multiplet basis of a window to the S_z basis of
the same window, the spin-adapted effective Hamiltonian has the plain
definition

    sigma = E^T  H_eff^{S_z}  E  psi,

where H_eff^{S_z} is the (separately pinned) U(1)xU(1) oracle's H_eff on the
expanded MPS.  H commutes with the total spin, so E psi (total S = 0) is
mapped into the S = 0 subspace and the projection E^T loses nothing.

Conventions (shared with the library's header):
  * SU(2) sectors (N, 2J); site multiplets {0} (N=0), {up, dn} (N=1,
    J=1/2; |1/2,+1/2> = c+_up|0>, |1/2,-1/2> = c+_dn|0>), {updn}
    (N=2, J=0; c+_up c+_dn |0>).
  * Coupling order follows the Jordan-Wigner order of the parts: left
    enlarged |(j_L j_s) J M>, right enlarged |(j_s j_R) J M>, window
    |(j_a j_b) S M>, each sum_m <j1 m1 j2 m2 | J M> |j1 m1>|j2 m2>.
  * Sectors are ordered by the (N_up, N_dn) of their highest-weight member.
    Enlarged-block rows run over pieces (site multiplet, block sector),
    ordered by site multiplet and then block sector, each piece holding all
    multiplets of its block sector.

Clebsch-Gordan coefficients use Racah's closed form (Racah 1942) evaluated in
exact rational arithmetic; arguments are doubled integers (tj = 2 j).
"""
import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

from . import dmrg as odmrg


def _fact(n):
    return math.factorial(n)


@lru_cache(maxsize=None)
def cg_exact(tj1, tm1, tj2, tm2, tJ, tM):
    """<j1 m1 j2 m2 | J M> as (sign, square) with square a Fraction.
    Doubled arguments.  Condon-Shortley phase convention."""
    if tm1 + tm2 != tM:
        return 0, Fraction(0)
    if tJ < abs(tj1 - tj2) or tJ > tj1 + tj2 or (tj1 + tj2 + tJ) % 2:
        return 0, Fraction(0)
    for tj, tm in ((tj1, tm1), (tj2, tm2), (tJ, tM)):
        if abs(tm) > tj or (tj + tm) % 2:
            return 0, Fraction(0)
    # half-integers as integers: a = j1 + j2 - J etc.
    a = (tj1 + tj2 - tJ) // 2
    b = (tj1 - tj2 + tJ) // 2
    c = (-tj1 + tj2 + tJ) // 2
    d = (tj1 + tj2 + tJ) // 2 + 1
    pref = Fraction((tJ + 1) * _fact(a) * _fact(b) * _fact(c), _fact(d))
    pref *= (_fact((tJ + tM) // 2) * _fact((tJ - tM) // 2) * _fact((tj1 - tm1) // 2)
             * _fact((tj1 + tm1) // 2) * _fact((tj2 - tm2) // 2) * _fact((tj2 + tm2) // 2))
    s = Fraction(0)
    for k in range(0, a + 1):
        den = [k, a - k, (tj1 - tm1) // 2 - k, (tj2 + tm2) // 2 - k,
               (tJ - tj2 + tm1) // 2 + k, (tJ - tj1 - tm2) // 2 + k]
        if min(den) < 0:
            continue
        p = 1
        for x in den:
            p *= _fact(x)
        s += Fraction((-1) ** k, p)
    if s == 0:
        return 0, Fraction(0)
    return (1 if s > 0 else -1), s * s * pref


def cg(tj1, tm1, tj2, tm2, tJ, tM):
    """<j1 m1 j2 m2 | J M> as a float (doubled arguments)."""
    sg, sq = cg_exact(tj1, tm1, tj2, tm2, tJ, tM)
    return sg * math.sqrt(sq) if sg else 0.0


def hw(q):
    """(N, 2J) -> S_z label (N_up, N_dn) of the highest-weight member; the
    sector order of spin-adapted bases."""
    return ((q[0] + q[1]) // 2, (q[0] - q[1]) // 2)


def sorted_sectors(qs):
    return sorted(qs, key=hw)


# site multiplets (N, 2J): {0}, {up, dn}, {updn}
SITE = [(0, 0), (1, 1), (2, 0)]


def couplings(tj1, tj2):
    return list(range(abs(tj1 - tj2), tj1 + tj2 + 1, 2))


def allowed(q, target, cap):
    """A part in sector q can be completed by `cap` sites to the total
    (N, 2S): the rest holds N - N_q particles, whose spin (at most
    min(n, 2 cap - n) / 2, of the parity of n) couples with J_q to S."""
    n_rest = target[0] - q[0]
    if n_rest < 0 or n_rest > 2 * cap:
        return False
    jmax2 = min(n_rest, 2 * cap - n_rest)
    return any(t <= jmax2 and (t - n_rest) % 2 == 0 for t in couplings(q[1], target[1]))


def enlarged_pieces(dims, target, cap):
    """{(N', 2J'): [(site multiplet, block sector, dim), ...]} in row order:
    by site multiplet, then block sector order."""
    out = {}
    for si, (ns, tjs) in enumerate(SITE):
        for q in sorted_sectors(dims):
            for tj in couplings(q[1], tjs):
                Q = (q[0] + ns, tj)
                if allowed(Q, target, cap):
                    out.setdefault(Q, []).append((si, q, dims[q]))
    return {Q: out[Q] for Q in sorted_sectors(out)}


# S_z site states of the U(1)xU(1) oracle, (N_up, N_dn): multiplet index, 2m
SITE_SZ = {(0, 0): (0, 0), (0, 1): (1, -1), (1, 0): (1, 1), (1, 1): (2, 0)}
SITE_OF_MULT = {}
for _q, (_s, _tm) in SITE_SZ.items():
    SITE_OF_MULT[(_s, _tm)] = _q


class MultBasis:
    """A block's multiplet basis together with its S_z image.

    sectors: {(N, 2J): number of multiplets}.  sz: {(N_up, N_dn): [(sector,
    multiplet index, 2M), ...]} -- the ordered S_z basis of the block the
    U(1)xU(1) oracle sees.  pos: (sector, beta, 2M) -> (S_z sector, index)."""

    def __init__(self, sectors, sz):
        self.sectors = dict(sectors)
        self.sz = sz
        self.pos = {}
        for Q, lst in sz.items():
            for i, key in enumerate(lst):
                self.pos[key] = (Q, i)

    def sz_dims(self):
        return {Q: len(v) for Q, v in self.sz.items()}


def vacuum_basis():
    return MultBasis({(0, 0): 1}, {(0, 0): [((0, 0), 0, 0)]})


def enlarged_images(X, target, cap, site_first):
    """S_z images of the multiplet states of an enlarged block X x site (or
    site x X): {(sector, row, 2M): {(S_z sector, S_z row): amplitude}}, with
    rows in the spin-adapted row order and S_z rows in the order of the
    U(1)xU(1) oracle's union basis (pieces by site state, f-major), plus the
    spin-adapted pieces."""
    pieces = enlarged_pieces(X.sectors, target, cap)
    # S_z enlarged basis, built like the U(1)xU(1) oracle's union_basis
    xdims = X.sz_dims()
    site_qs = sorted(SITE_SZ)
    zpieces = {}
    for qs in site_qs:
        for qx in sorted(xdims):
            Q = (qx[0] + qs[0], qx[1] + qs[1])
            zpieces.setdefault(Q, []).append((qs, qx))
    zoff = {}
    for Q, lst in zpieces.items():
        lst.sort(key=lambda p: p[0])            # by site state (stable)
        off = 0
        for qs, qx in lst:
            zoff[(Q, qs, qx)] = off
            off += xdims[qx]
    images = {}
    for Q, plist in pieces.items():
        row = 0
        for si, qb, d in plist:
            tjs = SITE[si][1]
            tj = qb[1]
            for beta in range(d):
                for tM in range(-Q[1], Q[1] + 1, 2):
                    img = {}
                    for tms in range(-tjs, tjs + 1, 2):
                        tmb = tM - tms
                        if abs(tmb) > tj:
                            continue
                        c = cg(tjs, tms, tj, tmb, Q[1], tM) if site_first else \
                            cg(tj, tmb, tjs, tms, Q[1], tM)
                        if c == 0.0:
                            continue
                        qsz_site = SITE_OF_MULT[(si, tms)]
                        zx, ix = X.pos[(qb, beta, tmb)]
                        Qz = (zx[0] + qsz_site[0], zx[1] + qsz_site[1])
                        r = zoff[(Qz, qsz_site, zx)] + ix
                        img[(Qz, r)] = img.get((Qz, r), 0.0) + c
                    images[(Q, row + beta, tM)] = img
            row += d
    return images, pieces


def expand_isometry(X, iso, target, cap, site_first):
    """Spin-adapted isometry {(N, 2J): rows x cols} of the enlarged block
    X x site -> (S_z isometry {(N_up, N_dn): matrix} in the U(1)xU(1)
    oracle's conventions, MultBasis of the new block)."""
    images, pieces = enlarged_images(X, target, cap, site_first)
    new_sz = {}
    for Q in sorted_sectors(iso):
        for tM in range(-Q[1], Q[1] + 1, 2):
            Qz = ((Q[0] + tM) // 2, (Q[0] - tM) // 2)
            for beta in range(iso[Q].shape[1]):
                new_sz.setdefault(Qz, []).append((Q, beta, tM))
    new_sz = {Qz: new_sz[Qz] for Qz in sorted(new_sz)}
    nb = MultBasis({Q: iso[Q].shape[1] for Q in iso}, new_sz)
    # S_z enlarged sector sizes
    zsize = {}
    for img in images.values():
        for (Qz, r) in img:
            zsize[Qz] = max(zsize.get(Qz, 0), r + 1)
    xdims = X.sz_dims()
    for qs in SITE_SZ:
        for qx, dx in xdims.items():
            Qz = (qx[0] + qs[0], qx[1] + qs[1])
            zsize.setdefault(Qz, 0)
    # exact S_z enlarged dimension: sum of pieces
    for Qz in zsize:
        zsize[Qz] = sum(xdims[qx] for qs in SITE_SZ for qx in xdims
                        if (qx[0] + qs[0], qx[1] + qs[1]) == Qz)
    out = {}
    for Qz, cols in new_sz.items():
        M = np.zeros((zsize[Qz], len(cols)))
        for c, (Q, beta, tM) in enumerate(cols):
            T = iso[Q]
            for r in range(T.shape[0]):
                if T[r, beta] == 0.0:
                    continue
                for (qz, zr), a in images[(Q, r, tM)].items():
                    assert qz == Qz
                    M[zr, c] += T[r, beta] * a
        out[Qz] = M
    return out, nb


def expand_mps(n_sites, target, left, right):
    """Spin-adapted left/right isometries -> S_z isometries (dicts n -> iso)
    and the MultBasis of every block."""
    lz, rz = {}, {}
    Lb = {0: vacuum_basis()}
    for n in sorted(left):
        lz[n], Lb[n] = expand_isometry(Lb[n - 1], left[n], target, n_sites - n, False)
    Rb = {n_sites: vacuum_basis()}
    for n in sorted(right, reverse=True):
        rz[n], Rb[n] = expand_isometry(Rb[n + 1], right[n], target, n, True)
    return lz, rz, Lb, Rb


class Su2Window:
    """Spin-adapted window (l, l+1) for total spin S = 0, through the
    U(1)xU(1) oracle.  layout: [(q_a, q_b, offset, dim_a, dim_b)] in (N, 2J)
    labels, blocks in the order of q_a's highest weight."""

    def __init__(self, model_sz, n_sites, target, left, right, l):
        if target[1] != 0:
            raise ValueError("spin-adapted windows are built for S = 0")
        self.target = target
        lz, rz, Lb, Rb = expand_mps(n_sites, target, {n: left[n] for n in left if n <= l},
                                    {n: right[n] for n in right if n >= l + 2})
        self.wz = odmrg.window_from_mps(model_sz, lz, rz, l)
        XL = Lb[l]
        XR = Rb[l + 2]
        self.imL, self.pL = enlarged_images(XL, target, n_sites - l - 1, False)
        self.imR, self.pR = enlarged_images(XR, target, l + 1, True)
        # S_z window: offsets of its (q_a, q_b) blocks
        self.zoff = {}
        for qa, qb, o, da, db in self.wz.layout:
            self.zoff[qa] = (o, da, db, qb)
        self.layout = []
        off = 0
        for qa, pa in self.pL.items():
            qb = (target[0] - qa[0], qa[1])
            if qb not in self.pR:
                continue
            da = sum(p[2] for p in pa)
            db = sum(p[2] for p in self.pR[qb])
            self.layout.append((qa, qb, off, da, db))
            off += da * db
        self.size = off
        self._build_embedding()

    def _build_embedding(self):
        """E as a sparse list: (spin-adapted index, S_z index, amplitude)."""
        rows, cols, vals = [], [], []
        for qa, qb, o, da, db in self.layout:
            tj = qa[1]
            for tm in range(-tj, tj + 1, 2):
                w = cg(tj, tm, tj, -tm, 0, 0)
                for ia in range(da):
                    ima = self.imL[(qa, ia, tm)]
                    for ib in range(db):
                        imb = self.imR[(qb, ib, -tm)]
                        for (za, ra), xa in ima.items():
                            zo, zda, zdb, zqb = self.zoff[za]
                            for (zb, rb), xb in imb.items():
                                assert zb == zqb
                                rows.append(o + ia * db + ib)
                                cols.append(zo + ra * zdb + rb)
                                vals.append(w * xa * xb)
        import scipy.sparse as sp
        self.E = sp.csr_matrix((vals, (cols, rows)), shape=(self.wz.size, self.size))

    def expand(self, psi):
        return self.E @ psi

    def project(self, v):
        return self.E.T @ v

    def apply(self, psi):
        """sigma = E^T H_eff^{S_z} E psi."""
        return self.project(self.wz.apply(self.expand(psi)))

    def solve(self, tol=1e-10, seed=0):
        import scipy.sparse.linalg as spla
        n = self.size
        if n <= 400:
            eye = np.eye(n)
            Hm = np.stack([self.apply(eye[:, j]) for j in range(n)], axis=1)
            w, V = np.linalg.eigh(0.5 * (Hm + Hm.T))
            return w[0], V[:, 0]
        op = spla.LinearOperator((n, n), matvec=self.apply, dtype=float)
        v0 = np.random.default_rng(seed).standard_normal(n)
        w, V = spla.eigsh(op, k=1, which="SA", tol=tol, v0=v0, ncv=24)
        return w[0], V[:, 0]
