"""Spin-orbital form of the Eq. 1 Hamiltonian (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Mode (spin-orbital) numbering along the DMRG chain: spinless p = i;
spinful p = 2 i + a with a = 0 (up), 1 (down), so a site holds its up mode
before its down mode in the Jordan-Wigner order.

H = sum_pq h[p,q] c^+_p c_q + sum_pqrs W[p,q,r,s] c^+_p c^+_q c_r c_s, where W
is the Eq. 1 tensor antisymmetrised in (p,q) and in (r,s):
    W = (X - X^{qprs} - X^{pqsr} + X^{qpsr}) / 4,
which leaves the operator unchanged because c^+_p c^+_q = -c^+_q c^+_p and
c_r c_s = -c_s c_r.
"""
import numpy as np


def spin_orbital(T, V4, spinful):
    """Return (h, W) over spin-orbitals from spatial Eq. 1 parameters."""
    N = T.shape[0]
    if not spinful:
        X = V4.copy()
        h = T.copy()
    else:
        M = 2 * N
        h = np.zeros((M, M))
        for a in range(2):
            h[a::2, a::2] = T
        X = np.zeros((M, M, M, M))
        # X[(i a),(j b),(k b),(l a)] = V[i,j,k,l]
        for a in range(2):
            for b in range(2):
                X[a::2, b::2, b::2, a::2] += V4
    W = 0.25 * (X - X.transpose(1, 0, 2, 3) - X.transpose(0, 1, 3, 2)
                + X.transpose(1, 0, 3, 2))
    return h, W


def check_hermitian(h, W, tol=1e-12):
    """Hermiticity of Eq. 1 with real coefficients: h = h^T, W[pqrs] = W[srqp]."""
    e1 = np.max(np.abs(h - h.T)) if h.size else 0.0
    e2 = np.max(np.abs(W - W.transpose(3, 2, 1, 0))) if W.size else 0.0
    return max(e1, e2) <= tol * max(1.0, np.max(np.abs(W)) if W.size else 1.0)
