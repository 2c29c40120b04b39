"""Lattice Hamiltonians and the one-particle mode rotation (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (readings of the paper where it is ambiguous or garbled):
  * site index i = y * Lx + x on an Lx x Ly torus (periodic in both directions,
    Sec. II.A "torus geometry").
  * hopping enters as -t (c^+_i c_j + h.c.) per bond; Eq. 2 / Eq. 3 print +t,
    which on the even tori used here is isospectral by the gauge
    c_i -> (-1)^(x+y) c_i.
  * the Hubbard interaction of Eq. 2 is read as U sum_i n_{i up} n_{i dn}.
  * Eq. 1 coefficient order: V[i,j,k,l] multiplies c^+_i c^+_j c_k c_l, with no
    prefactor.  For spinful models the spatial V is spin-independent:
    sum_{ab} V[i,j,k,l] c^+_{i a} c^+_{j b} c_{k b} c_{l a}.
"""
import numpy as np


def torus_bonds(Lx, Ly, kind="nn"):
    """Bonds of the torus, each listed once (Sec. II.A, torus geometry).

    kind='nn': (r, r+x) and (r, r+y) for every site r -> 2N bonds.
    kind='nnn': (r, r+x+y) and (r, r+x-y) for every site r -> 2N bonds.
    Requires Lx, Ly >= 3 so that no bond is listed twice.
    """
    if Lx < 3 or Ly < 3:
        raise ValueError("torus bonds need Lx, Ly >= 3")
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            r = y * Lx + x
            if kind == "nn":
                bonds.append((r, y * Lx + (x + 1) % Lx))
                bonds.append((r, ((y + 1) % Ly) * Lx + x))
            elif kind == "nnn":
                bonds.append((r, ((y + 1) % Ly) * Lx + (x + 1) % Lx))
                bonds.append((r, ((y - 1) % Ly) * Lx + (x + 1) % Lx))
            else:
                raise ValueError(kind)
    return bonds


def spinless_tV(Lx, Ly, t=1.0, tp=0.0, V=1.0):
    """Eq. 3: spinless t-t'-V model on the torus, as (T, V) in Eq. 1 form.

    T[i,j] = -t on NN bonds, -t' on NNN bonds (both orientations).
    V n_i n_j = V c^+_i c^+_j c_j c_i for i != j, so V4[i,j,j,i] += V once per
    NN bond.
    """
    N = Lx * Ly
    T = np.zeros((N, N))
    V4 = np.zeros((N, N, N, N))
    for i, j in torus_bonds(Lx, Ly, "nn"):
        T[i, j] += -t
        T[j, i] += -t
        V4[i, j, j, i] += V
    if tp != 0.0:
        for i, j in torus_bonds(Lx, Ly, "nnn"):
            T[i, j] += -tp
            T[j, i] += -tp
    return T, V4


def hubbard(Lx, Ly, t=1.0, U=4.0):
    """Eq. 2 (read as U n_up n_dn on site) in spatial Eq. 1 form.

    With the spinful convention above, V4[i,i,i,i] = U/2 gives
    (U/2) sum_{ab} c^+_{ia} c^+_{ib} c_{ib} c_{ia} = U n_{i up} n_{i dn}.
    """
    N = Lx * Ly
    T = np.zeros((N, N))
    V4 = np.zeros((N, N, N, N))
    for i, j in torus_bonds(Lx, Ly, "nn"):
        T[i, j] += -t
        T[j, i] += -t
    for i in range(N):
        V4[i, i, i, i] = U / 2.0
    return T, V4


def momentum_levels(Lx, Ly, t=1.0):
    """Single-particle energies -2t(cos kx + cos ky), k = 2 pi n / L."""
    out = []
    for ny in range(Ly):
        for nx in range(Lx):
            kx, ky = 2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly
            out.append(-2 * t * (np.cos(kx) + np.cos(ky)))
    return np.array(out)


def momentum_basis(Lx, Ly):
    """Real standing-wave momentum modes (reading of Sec. II.B's mode basis).

    For each pair {k, -k} with k != -k (mod 2 pi): sqrt(2/N) cos(k.r) and
    sqrt(2/N) sin(k.r); for self-conjugate k: sqrt(1/N) cos(k.r).  The pair's
    representative is the member with the smaller (nx, ny).  Modes are ordered
    by (eps_k, nx, ny, cos before sin) with eps_k = -2(cos kx + cos ky).
    Returns U with U[i, m] = amplitude of mode m on site i, so c_i = sum_m
    U[i,m] d_m.
    """
    N = Lx * Ly
    xs = np.array([i % Lx for i in range(N)], dtype=float)
    ys = np.array([i // Lx for i in range(N)], dtype=float)
    seen = set()
    modes = []
    for ny in range(Ly):
        for nx in range(Lx):
            if (nx, ny) in seen:
                continue
            mx, my = (-nx) % Lx, (-ny) % Ly
            seen.add((nx, ny))
            seen.add((mx, my))
            rep = min((nx, ny), (mx, my))
            kx, ky = 2 * np.pi * rep[0] / Lx, 2 * np.pi * rep[1] / Ly
            eps = round(-2.0 * (np.cos(kx) + np.cos(ky)), 12)
            phase = kx * xs + ky * ys
            if (mx, my) == (nx, ny):
                modes.append(((eps, rep[0], rep[1], 0), np.sqrt(1.0 / N) * np.cos(phase)))
            else:
                modes.append(((eps, rep[0], rep[1], 0), np.sqrt(2.0 / N) * np.cos(phase)))
                modes.append(((eps, rep[0], rep[1], 1), np.sqrt(2.0 / N) * np.sin(phase)))
    modes.sort(key=lambda m: m[0])
    return np.stack([m[1] for m in modes], axis=1)


def rotate(T, V4, U):
    """H(U): rotate the Eq. 1 parameters instead of the operators (Sec. II.B).

    T'[a,b] = sum_ij U[i,a] T[i,j] U[j,b];
    V'[a,b,c,d] = sum_ijkl V[i,j,k,l] U[i,a] U[j,b] U[k,c] U[l,d],
    done as four quarter transforms (real U).
    """
    Tp = U.T @ T @ U
    W = np.tensordot(U, V4, axes=([0], [0]))          # a j k l
    W = np.tensordot(W, U, axes=([1], [0]))           # a k l b
    W = W.transpose(0, 3, 1, 2)                       # a b k l
    W = np.tensordot(W, U, axes=([2], [0]))           # a b l c
    W = W.transpose(0, 1, 3, 2)                       # a b c l
    W = np.tensordot(W, U, axes=([3], [0]))           # a b c d
    return Tp, W


def cdw_square(Lx, Ly):
    """(n_even - n_odd)^2 in Eq. 1 form, real space (the operator of the CDW
    order parameter C_CDW = <(n_even - n_odd)^2> / N^2, Sec. III.C).

    With s_i = +1 on sites with x + y even and -1 otherwise,
    (sum_i s_i n_i)^2 = sum_i n_i + sum_ij s_i s_j c^+_i c^+_j c_j c_i
    (n_i n_j = delta_ij n_i + c^+_i c^+_j c_j c_i, s_i^2 = 1): T = identity,
    V[i, j, j, i] = s_i s_j; in the spinful convention the a = b terms of
    sum_ab V_iiii c^+_ia c^+_ib c_ib c_ia vanish, so the same (T, V) holds.
    """
    N = Lx * Ly
    s = np.array([1.0 - 2.0 * (((i % Lx) + (i // Lx)) % 2) for i in range(N)])
    T = np.eye(N)
    V4 = np.zeros((N, N, N, N))
    for i in range(N):
        for j in range(N):
            V4[i, j, j, i] = s[i] * s[j]
    return T, V4
