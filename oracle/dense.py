"""Explicit W^T H W projection for small systems (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The renormalised basis states of every block are written out as vectors in
the Fock space of the block's modes, following the isometries (Eq. 4 read as
a sequence of basis transformations).  For a window, W maps the L. x .R
basis into Fock space, and sigma_dense = W^T H W psi with H applied by the
exact-diagonalisation code (ed.py).  This is the plain definition of
H_eff psi that the block-operator route must reproduce.

Fock index of a state: bit p set <=> mode p occupied.  Because the modes of
the first part precede those of the second, the product state
(F creators)(G creators)|0> is the canonical ordered state: its Fock vector is
the outer product of the parts' vectors with no extra sign.
"""
import numpy as np

from .ed import FockSpace


def _site_states(model, i):
    k = len(model.site_modes(i))

    def qn(b):
        if not model.spinful:
            return (bin(b).count("1"),)
        return (b & 1, (b >> 1) & 1)
    order = sorted(range(2 ** k), key=qn)
    return [(qn(b), b) for b in order], k


def _enlarge_vectors(model, block_vecs, block_nmodes, i, first_is_site, allowed):
    """Fock vectors of the enlarged sectors, pieces ordered by site state."""
    sstates, k = _site_states(model, i)
    out = {}
    for qs, sb in sstates:
        for q, V in block_vecs.items():
            Q = tuple(a + b for a, b in zip(q, qs))
            if not allowed(Q):
                continue
            nb = V.shape[1]
            Vn = np.zeros((V.shape[0], 2 ** (block_nmodes + k)))
            if first_is_site:
                idx = sb + (np.arange(nb) << k)
            else:
                idx = np.arange(nb) + (sb << block_nmodes)
            Vn[:, idx] = V
            out.setdefault(Q, []).append(Vn)
    return {Q: np.vstack(lst) for Q, lst in sorted(out.items())}, block_nmodes + k


def left_vectors(model, left_iso, upto):
    vecs, nm = {model.zero(): np.ones((1, 1))}, 0
    for n in range(1, upto + 1):
        e, nm = _enlarge_vectors(model, vecs, nm, n - 1, False, model.allowed_left(n))
        T = left_iso[n]
        vecs = {Q: T[Q].T @ e[Q] for Q in T}
    return vecs, nm


def right_vectors(model, right_iso, downto):
    vecs, nm = {model.zero(): np.ones((1, 1))}, 0
    for n in range(model.n_sites - 1, downto - 1, -1):
        e, nm = _enlarge_vectors(model, vecs, nm, n, True, model.allowed_right(n))
        T = right_iso[n]
        vecs = {Q: T[Q].T @ e[Q] for Q in T}
    return vecs, nm


def dense_sigma(model, left_iso, right_iso, l, layout, psi):
    """sigma = W^T H W psi for window (l, l+1); layout as Window.layout."""
    Lv, nl = left_vectors(model, left_iso, l)
    Rv, nr = right_vectors(model, right_iso, l + 2)
    Ld, nld = _enlarge_vectors(model, Lv, nl, l, False, model.allowed_left(l + 1))
    Rd, nrd = _enlarge_vectors(model, Rv, nr, l + 1, True, model.allowed_right(l + 1))
    M = nld + nrd
    assert M == model.M
    fs = FockSpace(M, sum(model.target))
    phi = np.zeros((2 ** nld, 2 ** nrd))
    for qa, qb, o, da, db in layout:
        phi += Ld[qa].T @ psi[o:o + da * db].reshape(da, db) @ Rd[qb]
    full = phi.T.reshape(-1)             # index = a_bits + b_bits * 2^nld
    hv = fs.apply_H(model.h, model.W, full[fs.states])
    hfull = np.zeros(2 ** M)
    hfull[fs.states] = hv
    hm = hfull.reshape(2 ** nrd, 2 ** nld).T
    out = np.zeros_like(psi)
    for qa, qb, o, da, db in layout:
        out[o:o + da * db] = (Ld[qa] @ hm @ Rd[qb].T).ravel()
    return out
