"""Block-sparse operators over quantum-number sectors (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A quantum number (QN) is a tuple of ints: (N,) for the spinless model,
(N_up, N_dn) for the spinful one.  A Basis is a sorted list of sectors
(qn, dim).  An Op has a definite QN shift and fermion parity and stores one
dense block per input sector:  blocks[q_in] has shape (dim(q_in + shift),
dim(q_in)).

Two-part bases (the enlarged blocks L. = L x site, .R = site x R of two-site
DMRG, Sec. II and Eq. 4): the first part F precedes the second part G in the
Jordan-Wigner order.  A product state |f>|g> is (F creators)(G creators)|0>.
Within a union sector the pieces (one per site state) are ordered by the site
state's QN, and inside a piece the states are f-major.  The operator product
A_F B_G acts as
    (A_F B_G) |f>|g> = (-1)^(parity(B) * N(f)) (A_F|f>) (B_G|g>),
N(f) = particle number of the input F state.
"""
import numpy as np


def qadd(a, b):
    return tuple(x + y for x, y in zip(a, b))


def qsub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def qneg(a):
    return tuple(-x for x in a)


class Basis:
    def __init__(self, sectors):
        sectors = sorted((tuple(q), int(d)) for q, d in sectors if d > 0)
        self.qns = [q for q, _ in sectors]
        self.dims = [d for _, d in sectors]
        self.index = {q: k for k, q in enumerate(self.qns)}
        self.pieces = None          # set for two-part bases
        self.total = sum(self.dims)

    def dim(self, q):
        k = self.index.get(tuple(q))
        return 0 if k is None else self.dims[k]

    def has(self, q):
        return tuple(q) in self.index


class Op:
    def __init__(self, shift, parity, blocks=None):
        self.shift = tuple(shift)
        self.parity = int(parity) & 1
        self.blocks = {} if blocks is None else blocks

    def copy(self):
        return Op(self.shift, self.parity, {k: v.copy() for k, v in self.blocks.items()})

    def scaled(self, c):
        return Op(self.shift, self.parity, {k: c * v for k, v in self.blocks.items()})

    def add(self, other, c=1.0):
        """self += c * other (same shift)."""
        assert other.shift == self.shift and other.parity == self.parity
        for k, v in other.blocks.items():
            if k in self.blocks:
                self.blocks[k] = self.blocks[k] + c * v
            else:
                self.blocks[k] = c * v
        return self

    def dagger(self):
        """Hermitian conjugate = matrix transpose (real coefficients)."""
        nb = {qadd(q, self.shift): b.T.copy() for q, b in self.blocks.items()}
        return Op(qneg(self.shift), self.parity, nb)

    def dense(self, basis):
        """Full matrix on a Basis (rows/cols in sector order)."""
        offs = np.cumsum([0] + basis.dims)
        M = np.zeros((basis.total, basis.total))
        for q, b in self.blocks.items():
            qo = qadd(q, self.shift)
            i, j = basis.index[qo], basis.index[q]
            M[offs[i]:offs[i + 1], offs[j]:offs[j + 1]] += b
        return M


def zero_op(shift, parity):
    return Op(shift, parity, {})


def identity(basis):
    z = tuple(0 for _ in basis.qns[0])
    return Op(z, 0, {q: np.eye(d) for q, d in zip(basis.qns, basis.dims)})


def n_of(q):
    return sum(q)


def union_basis(F, G, site_is_first, allowed):
    """Two-part basis F x G restricted to allowed union QNs.

    pieces[Q] = list of (qf, qg, offset, dim_f, dim_g) ordered by the site
    state's QN (the site is F if site_is_first else G).
    """
    pieces = {}
    for qf, df in zip(F.qns, F.dims):
        for qg, dg in zip(G.qns, G.dims):
            Q = qadd(qf, qg)
            if not allowed(Q):
                continue
            pieces.setdefault(Q, []).append((qf, qg, df, dg))
    sectors = []
    final = {}
    for Q, lst in pieces.items():
        lst.sort(key=lambda p: p[0] if site_is_first else p[1])
        off = 0
        out = []
        for qf, qg, df, dg in lst:
            out.append((qf, qg, off, df, dg))
            off += df * dg
        final[Q] = out
        sectors.append((Q, off))
    B = Basis(sectors)
    B.pieces = final
    B.piece_index = {Q: {(p[0], p[1]): p for p in lst} for Q, lst in final.items()}
    return B


def kron(A, Bop, U):
    """Operator product A_F B_G on the two-part basis U (see module doc)."""
    shift = qadd(A.shift, Bop.shift)
    out = Op(shift, A.parity ^ Bop.parity, {})
    for Q, plist in U.pieces.items():
        Qo = qadd(Q, shift)
        if not U.has(Qo):
            continue
        dout, din = U.dim(Qo), U.dim(Q)
        blk = None
        for qf, qg, off, df, dg in plist:
            a = A.blocks.get(qf)
            b = Bop.blocks.get(qg)
            if a is None or b is None:
                continue
            qfo, qgo = qadd(qf, A.shift), qadd(qg, Bop.shift)
            po = U.piece_index[Qo].get((qfo, qgo))
            if po is None:
                continue
            sign = -1.0 if (Bop.parity and (n_of(qf) & 1)) else 1.0
            if blk is None:
                blk = np.zeros((dout, din))
            blk[po[2]:po[2] + po[3] * po[4], off:off + df * dg] += sign * np.kron(a, b)
        if blk is not None:
            out.blocks[Q] = blk
    return out


def renormalize(A, T, newbasis):
    """A' = T^T A T blockwise, T[Q] of shape (dim_U(Q), dim_new(Q))."""
    out = Op(A.shift, A.parity, {})
    for q, b in A.blocks.items():
        qo = qadd(q, A.shift)
        if q in T and qo in T and newbasis.has(q) and newbasis.has(qo):
            out.blocks[q] = T[qo].T @ b @ T[q]
    return out
