"""Exact diagonalisation of Eq. 1 in a fixed-particle-number Fock space (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Fock states |n> = prod_{p ascending} (c^+_p)^{n_p} |0> over M spin-orbitals;
the Jordan-Wigner sign of c_p is (-1)^(number of occupied modes below p).

The Hamiltonian is applied through one-body excitation operators
E_pq = c^+_p c_q, using the operator identity
    c^+_p c^+_q c_r c_s = delta_qr E_ps - E_pr E_qs,
so H v = sum_pq h_pq E_pq v + sum_ps (sum_q W_pqqs) E_ps v
         - sum_pr E_pr (sum_qs W_pqrs E_qs v).
This is a different route from the block-operator DMRG, which is what makes
it a check on it.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class FockSpace:
    """All occupation strings of M modes with exactly n_part particles."""

    def __init__(self, M, n_part):
        self.M = M
        self.n = n_part
        states = []
        for occ in itertools.combinations(range(M), n_part):
            s = 0
            for p in occ:
                s |= 1 << p
            states.append(s)
        self.states = np.array(sorted(states), dtype=np.int64)
        self.dim = len(self.states)
        self._E = {}

    def lookup(self, s):
        return np.searchsorted(self.states, s)

    def occ(self, p):
        return (self.states >> p) & 1

    def E(self, p, q):
        """Sparse matrix of c^+_p c_q on this space (cached)."""
        key = (p, q)
        if key in self._E:
            return self._E[key]
        st = self.states
        if p == q:
            m = sp.diags(self.occ(p).astype(float), format="csr")
            self._E[key] = m
            return m
        ok = (((st >> q) & 1) == 1) & (((st >> p) & 1) == 0)
        src = np.nonzero(ok)[0]
        s1 = st[src] & ~(1 << q)
        # sign of c_q on the source, then of c^+_p on the intermediate state
        sgn = np.ones(len(src))
        for b in range(q):
            sgn *= 1 - 2 * ((st[src] >> b) & 1)
        for b in range(p):
            sgn *= 1 - 2 * ((s1 >> b) & 1)
        s2 = s1 | (1 << p)
        dst = self.lookup(s2)
        m = sp.csr_matrix((sgn, (dst, src)), shape=(self.dim, self.dim))
        self._E[key] = m
        return m

    def apply_H(self, h, W, v):
        M = self.M
        out = np.zeros_like(v)
        oneb = h + np.einsum("pqqs->ps", W)
        for p in range(M):
            for q in range(M):
                c = oneb[p, q]
                if c != 0.0:
                    out += c * (self.E(p, q) @ v)
        U = np.empty((M * M, self.dim))
        for q in range(M):
            for s in range(M):
                U[q * M + s] = self.E(q, s) @ v
        Wm = W.transpose(0, 2, 1, 3).reshape(M * M, M * M)   # (p r), (q s)
        F = Wm @ U
        for p in range(M):
            for r in range(M):
                out -= self.E(p, r) @ F[p * M + r]
        return out

    def sector_mask(self, n_up=None):
        """States with a given number of up electrons (modes p = 2i)."""
        if n_up is None:
            return np.ones(self.dim, dtype=bool)
        cnt = np.zeros(self.dim, dtype=np.int64)
        for p in range(0, self.M, 2):
            cnt += (self.states >> p) & 1
        return cnt == n_up


def ground_energy(h, W, n_part, n_up=None, k=1, tol=1e-12, dense_max=3000):
    """Lowest eigenvalue(s) of Eq. 1 in the sector (n_part[, n_up])."""
    M = h.shape[0]
    fs = FockSpace(M, n_part)
    idx = np.nonzero(fs.sector_mask(n_up))[0]
    d = len(idx)

    def mv(x):
        full = np.zeros(fs.dim)
        full[idx] = x
        return fs.apply_H(h, W, full)[idx]

    if d <= dense_max:
        Hm = np.empty((d, d))
        eye = np.eye(d)
        for j in range(d):
            Hm[:, j] = mv(eye[:, j])
        return np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[:k]
    op = spla.LinearOperator((d, d), matvec=mv, dtype=float)
    rng = np.random.default_rng(12345)
    w = spla.eigsh(op, k=k, which="SA", tol=tol, v0=rng.standard_normal(d),
                   return_eigenvectors=False, ncv=max(20, 2 * k + 1))
    return np.sort(w)


def ground_state(h, W, n_part, n_up=None, tol=1e-13):
    """Lowest eigenpair in the sector: (E0, v on the whole fixed-n_part Fock
    space (zero outside the sector), FockSpace)."""
    M = h.shape[0]
    fs = FockSpace(M, n_part)
    idx = np.nonzero(fs.sector_mask(n_up))[0]
    d = len(idx)

    def mv(x):
        full = np.zeros(fs.dim)
        full[idx] = x
        return fs.apply_H(h, W, full)[idx]

    if d <= 3000:
        Hm = np.stack([mv(e) for e in np.eye(d)], axis=1)
        w, V = np.linalg.eigh(0.5 * (Hm + Hm.T))
        e0, x = w[0], V[:, 0]
    else:
        op = spla.LinearOperator((d, d), matvec=mv, dtype=float)
        rng = np.random.default_rng(12345)
        w, V = spla.eigsh(op, k=1, which="SA", tol=tol, v0=rng.standard_normal(d), ncv=24)
        e0, x = w[0], V[:, 0]
    v = np.zeros(fs.dim)
    v[idx] = x / np.linalg.norm(x)
    return e0, v, fs


def rdm1(fs, v):
    """Spin-orbital one-particle density matrix gamma[p, q] = <c+_q c_p>
    (the paper's gamma_{i,j} = <c+_j c_i>, Sec. II.B)."""
    M = fs.M
    g = np.empty((M, M))
    for p in range(M):
        for q in range(M):
            g[p, q] = v @ (fs.E(q, p) @ v)
    return g


def expectation(fs, h, W, v):
    """<v| H(h, W) |v> for an operator in the spin-orbital Eq. 1 form."""
    return float(v @ fs.apply_H(h, W, v))
