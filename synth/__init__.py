"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and bench.

This module holds no arithmetic of the method: it draws random numbers and
does the quantum-number bookkeeping needed to give them the right shapes.

  * random isometries (a random left/right-canonical MPS basis, Eq. 4) with a
    prescribed distribution of states over sectors,
  * random wavefunctions psi for a two-site window,
  * the seeded Haar-orthogonal matrix Q used for the "optimized" mode basis
    stand-in (U = U_mom Q).

Conventions (shared format, see include/dmrg_b300.h):
  * QN = (N,) spinless or (N_up, N_dn) spinful; site states are ordered by QN.
  * Left isometry n maps the enlarged block L_{n-1} x site_{n-1} to L_n; right
    isometry n maps site_n x R_{n+1} to R_n.  For each QN Q it is a
    (dim_enlarged(Q), dim_new(Q)) matrix with orthonormal columns.  Rows of
    an enlarged sector run over pieces ordered by the site state's QN; each
    piece holds all states of the block sector Q - q(site state).
  * psi for window (l, l+1) has one block per L. sector q_a (ascending) paired
    with the .R sector target - q_a, row-major (dim_a, dim_b), concatenated.
"""
import math

import numpy as np


def site_qns(spinful):
    return [(0, 0), (0, 1), (1, 0), (1, 1)] if spinful else [(0,), (1,)]


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def _sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def _allowed(q, target, cap):
    return all(0 <= t - x <= cap for t, x in zip(target, q))


def _enlarged(dims, spinful, target, cap):
    out = {}
    for qs in site_qns(spinful):
        for q, d in dims.items():
            Q = _add(q, qs)
            if _allowed(Q, target, cap):
                out[Q] = out.get(Q, 0) + d
    return dict(sorted(out.items()))


def _distribute(edims, D, nbar, sigma, spinful):
    """Spread D states over sectors with Gaussian weights, capped by e(q)."""
    qs = list(edims)
    w = {}
    for q in qs:
        n = sum(q)
        ww = math.exp(-((n - nbar) ** 2) / (2 * sigma * sigma))
        if spinful:
            sz = 0.5 * (q[0] - q[1])
            ww *= math.exp(-sz * sz / 2)
        w[q] = ww
    d = {q: 0 for q in qs}
    free = set(qs)
    remaining = D
    while free and remaining > 0:
        tot = sum(w[q] for q in free)
        capped = [q for q in free if remaining * w[q] / tot >= edims[q]]
        if not capped:
            for q in free:
                d[q] = int(remaining * w[q] / tot)
            break
        for q in capped:
            d[q] = edims[q]
            remaining -= edims[q]
            free.discard(q)
    if sum(d.values()) == 0:
        d[max(qs, key=lambda x: w[x])] = 1
    return {q: v for q, v in d.items() if v > 0}


def _iso(rng, e, d):
    g = rng.standard_normal((e, d))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1
    return q * s


def random_left_isometries(n_sites, spinful, target, D, upto, seed, spread=None):
    """Isometries left[n], n = 1..upto (dict n -> {Q: matrix}).

    spread: width (in particles) of the Gaussian sector weights; default
    max(1, n_sites / 8).  A small spread puts D into fewer, wider sectors."""
    rng = np.random.default_rng(seed)
    dims = {tuple(0 for _ in target): 1}
    out = {}
    for n in range(1, upto + 1):
        e = _enlarged(dims, spinful, target, n_sites - n)
        nbar = sum(target) * n / n_sites
        dn = _distribute(e, D, nbar, spread or max(1.0, n_sites / 8), spinful)
        out[n] = {Q: _iso(rng, e[Q], dn[Q]) for Q in dn}
        dims = dn
    return out


def random_right_isometries(n_sites, spinful, target, D, downto, seed, spread=None):
    """Isometries right[n], n = n_sites-1 .. downto (dict n -> {Q: matrix});
    spread as for random_left_isometries."""
    rng = np.random.default_rng(seed)
    dims = {tuple(0 for _ in target): 1}
    out = {}
    for n in range(n_sites - 1, downto - 1, -1):
        e = _enlarged(dims, spinful, target, n)
        nbar = sum(target) * (n_sites - n) / n_sites
        dn = _distribute(e, D, nbar, spread or max(1.0, n_sites / 8), spinful)
        out[n] = {Q: _iso(rng, e[Q], dn[Q]) for Q in dn}
        dims = dn
    return out


def block_dims(iso):
    return {Q: m.shape[1] for Q, m in iso.items()}


def window_layout(n_sites, spinful, target, left_dims, right_dims, l):
    """[(q_a, q_b, dim_a, dim_b)] for window (l, l+1) given dims of L_l, R_{l+2}."""
    Ld = _enlarged(left_dims, spinful, target, n_sites - l - 1)
    Rd = {}
    for qs in site_qns(spinful):
        for q, d in right_dims.items():
            Q = _add(q, qs)
            if _allowed(Q, target, l + 1):
                Rd[Q] = Rd.get(Q, 0) + d
    out = []
    for qa in sorted(Ld):
        qb = _sub(target, qa)
        if qb in Rd:
            out.append((qa, qb, Ld[qa], Rd[qb]))
    return out


def random_psi(layout, seed):
    rng = np.random.default_rng(seed)
    n = sum(da * db for _, _, da, db in layout)
    return rng.standard_normal(n)


def haar_rotation(N, seed):
    """Q factor of a seeded N x N standard-normal matrix, diag(R) > 0."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((N, N))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))


# ---------------------------------------------------------------------------
# U(1)xSU(2) bookkeeping (spin-adapted MPS basis: D counts multiplets).
#
# A sector is (N, 2J): particle number and twice the spin of its multiplets.
# Sectors are ordered by the (N_up, N_dn) of their highest-weight member,
# ((N + 2J) / 2, (N - 2J) / 2), ascending.  The site multiplets are
# {0} (N=0, J=0), {up, dn} (N=1, J=1/2), {updn} (N=2, J=0), in that order.
# An enlarged block (block x site or site x block) has sectors (N', 2J')
# for every coupling J' of the block's J with the site's j; its rows run over
# pieces (site multiplet, block sector) ordered by site multiplet, then block
# sector order, each piece holding all multiplets of the block sector.
# ---------------------------------------------------------------------------

SU2_SITE = [(0, 0), (1, 1), (2, 0)]


def su2_key(q):
    """Sort key of an SU(2) sector (N, 2J): its highest weight (N_up, N_dn)."""
    n, tj = q
    return ((n + tj) // 2, (n - tj) // 2)


def su2_sorted(qs):
    return sorted(qs, key=su2_key)


def su2_couplings(tj1, tj2):
    """Twice the spins that j1 x j2 couples to."""
    return list(range(abs(tj1 - tj2), tj1 + tj2 + 1, 2))


def su2_allowed(q, target, cap):
    """Can a part with sector q be completed by `cap` more sites to the total
    (N, 2S) = target?"""
    n_rest = target[0] - q[0]
    if n_rest < 0 or n_rest > 2 * cap:
        return False
    jmax2 = min(n_rest, 2 * cap - n_rest)
    for tjr in su2_couplings(q[1], target[1]):
        if tjr <= jmax2 and (tjr - n_rest) % 2 == 0:
            return True
    return False


def su2_enlarged_pieces(dims, target, cap, site_first):
    """Enlarged sectors of a block with sectors dims {(N, 2J): d} and one site:
    {(N', 2J'): [(site multiplet index, block sector, d), ...]} in row order."""
    out = {}
    for si, (ns, tjs) in enumerate(SU2_SITE):
        for q in su2_sorted(dims):
            for tj in su2_couplings(q[1], tjs):
                Q = (q[0] + ns, tj)
                if su2_allowed(Q, target, cap):
                    out.setdefault(Q, []).append((si, q, dims[q]))
    return {Q: out[Q] for Q in su2_sorted(out)}


def _su2_distribute(edims, D, nbar, sigma):
    qs = list(edims)
    w = {q: math.exp(-((q[0] - nbar) ** 2) / (2 * sigma * sigma)) * math.exp(-(q[1] / 2) ** 2 / 2)
         for q in qs}
    d = {q: 0 for q in qs}
    free = set(qs)
    remaining = D
    while free and remaining > 0:
        tot = sum(w[q] for q in free)
        capped = [q for q in free if remaining * w[q] / tot >= edims[q]]
        if not capped:
            for q in free:
                d[q] = int(remaining * w[q] / tot)
            break
        for q in capped:
            d[q] = edims[q]
            remaining -= edims[q]
            free.discard(q)
    if sum(d.values()) == 0:
        d[max(qs, key=lambda x: w[x])] = 1
    return {q: v for q, v in d.items() if v > 0}


def random_left_isometries_su2(n_sites, target, D, upto, seed, spread=None):
    """Spin-adapted left isometries left[n], n = 1..upto: {n: {(N, 2J): matrix}}
    (D multiplets per block; target = (N, 2S))."""
    rng = np.random.default_rng(seed)
    dims = {(0, 0): 1}
    out = {}
    for n in range(1, upto + 1):
        pieces = su2_enlarged_pieces(dims, target, n_sites - n, False)
        e = {Q: sum(p[2] for p in v) for Q, v in pieces.items()}
        nbar = target[0] * n / n_sites
        dn = _su2_distribute(e, D, nbar, spread or max(1.0, n_sites / 8))
        out[n] = {Q: _iso(rng, e[Q], dn[Q]) for Q in su2_sorted(dn)}
        dims = dn
    return out


def random_right_isometries_su2(n_sites, target, D, downto, seed, spread=None):
    """Spin-adapted right isometries right[n], n = n_sites-1 .. downto."""
    rng = np.random.default_rng(seed)
    dims = {(0, 0): 1}
    out = {}
    for n in range(n_sites - 1, downto - 1, -1):
        pieces = su2_enlarged_pieces(dims, target, n, True)
        e = {Q: sum(p[2] for p in v) for Q, v in pieces.items()}
        nbar = target[0] * (n_sites - n) / n_sites
        dn = _su2_distribute(e, D, nbar, spread or max(1.0, n_sites / 8))
        out[n] = {Q: _iso(rng, e[Q], dn[Q]) for Q in su2_sorted(dn)}
        dims = dn
    return out


def su2_window_layout(n_sites, target, left_dims, right_dims, l):
    """[(q_a, q_b, dim_a, dim_b)] of window (l, l+1) for total spin S = 0:
    L. sector q_a = (N_a, 2J) pairs with .R sector (N - N_a, 2J)."""
    if target[1] != 0:
        raise ValueError("spin-adapted windows are laid out for S = 0")
    Lp = su2_enlarged_pieces(left_dims, target, n_sites - l - 1, False)
    Rp = su2_enlarged_pieces(right_dims, target, l + 1, True)
    out = []
    for qa, pa in Lp.items():
        qb = (target[0] - qa[0], qa[1])
        if qb in Rp:
            out.append((qa, qb, sum(p[2] for p in pa), sum(p[2] for p in Rp[qb])))
    return out
