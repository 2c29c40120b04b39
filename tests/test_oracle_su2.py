"""Pins for the spin-adapted (U(1)xSU(2)) oracle.

The spin-adapted H_eff is defined through the exact Clebsch-Gordan expansion
of the multiplet basis onto the S_z basis of the U(1)xU(1) oracle.  Its parts
are pinned against things other than themselves:
  * Clebsch-Gordan coefficients: orthogonality, the j = 0 closed forms, and a
    library implementation (sympy) on sample values;
  * the expansion: an isometry, with orthonormal expanded MPS columns, and
    sector bookkeeping equal to the shared input bookkeeping;
  * H_eff: hermitian, and at full bond dimension its lowest eigenvalue is the
    exact-diagonalisation ground energy over the whole S_z = 0 sector (the
    3x3 Hubbard torus with 8 electrons has a singlet ground state, which the
    test confirms by reaching the ED value).
"""
import numpy as np
import pytest

import synth
from oracle import dmrg as odmrg
from oracle import ed, hamiltonian, lattice, su2


def test_cg_orthogonality_and_closed_forms():
    for tj1 in range(0, 5):
        for tj2 in range(0, 5):
            for tM in range(-(tj1 + tj2), tj1 + tj2 + 1, 2):
                Js = [tJ for tJ in su2.couplings(tj1, tj2) if abs(tM) <= tJ]
                for tJ in Js:
                    for tK in Js:
                        s = sum(su2.cg(tj1, m, tj2, tM - m, tJ, tM) * su2.cg(tj1, m, tj2, tM - m, tK, tM)
                                for m in range(-tj1, tj1 + 1, 2))
                        assert abs(s - (tJ == tK)) < 1e-14
    for tj in range(0, 7):
        for tm in range(-tj, tj + 1, 2):
            # coupling with spin 0 is the identity
            assert su2.cg(tj, tm, 0, 0, tj, tm) == pytest.approx(1.0, abs=1e-15)
            # the singlet: <j m j -m | 0 0> = (-1)^(j - m) / sqrt(2j + 1)
            assert su2.cg(tj, tm, tj, -tm, 0, 0) == pytest.approx(
                (-1) ** ((tj - tm) // 2) / np.sqrt(tj + 1), abs=1e-15)


def test_cg_matches_library():
    sympy = pytest.importorskip("sympy")
    from sympy.physics.quantum.cg import CG
    rng = np.random.default_rng(0)
    n = 0
    while n < 40:
        tj1, tj2 = (int(x) for x in rng.integers(0, 7, 2))
        tJ = int(rng.choice(su2.couplings(tj1, tj2)))
        tm1 = int(rng.choice(range(-tj1, tj1 + 1, 2)))
        tM = int(rng.choice(range(-tJ, tJ + 1, 2)))
        if abs(tM - tm1) > tj2:
            continue
        h = sympy.Rational(1, 2)
        ref = float(CG(tj1 * h, tm1 * h, tj2 * h, (tM - tm1) * h, tJ * h, tM * h).doit())
        assert su2.cg(tj1, tm1, tj2, tM - tm1, tJ, tM) == pytest.approx(ref, abs=1e-14)
        n += 1


def _hubbard_3x3():
    T, V4 = lattice.hubbard(3, 3, 1.0, 4.0)
    T, V4 = lattice.rotate(T, V4, lattice.momentum_basis(3, 3))
    h, W = hamiltonian.spin_orbital(T, V4, True)
    return odmrg.Model(h, W, True, (4, 4)), h, W


def test_sector_bookkeeping_matches_inputs():
    li = synth.random_left_isometries_su2(16, (16, 0), 48, 7, 5)
    for n in range(1, 8):
        prev = {(0, 0): 1} if n == 1 else synth.block_dims(li[n - 1])
        mine = su2.enlarged_pieces(prev, (16, 0), 16 - n)
        theirs = synth.su2_enlarged_pieces(prev, (16, 0), 16 - n, False)
        assert mine == theirs
        assert all(li[n][Q].shape[0] == sum(p[2] for p in mine[Q]) for Q in li[n])


@pytest.mark.parametrize("l", [1, 3])
def test_expansion_is_isometric(l):
    m, h, W = _hubbard_3x3()
    li = synth.random_left_isometries_su2(9, (8, 0), 12, l, 5)
    ri = synth.random_right_isometries_su2(9, (8, 0), 12, l + 2, 6)
    lz, rz, Lb, Rb = su2.expand_mps(9, (8, 0), li, ri)
    for iso in list(lz.values()) + list(rz.values()):
        for M in iso.values():
            assert np.abs(M.T @ M - np.eye(M.shape[1])).max() < 1e-13
    w = su2.Su2Window(m, 9, (8, 0), li, ri, l)
    EtE = (w.E.T @ w.E).toarray()
    assert np.abs(EtE - np.eye(w.size)).max() < 1e-13
    lay = synth.su2_window_layout(9, (8, 0), synth.block_dims(li[l]), synth.block_dims(ri[l + 2]), l)
    assert [(a, b, da, db) for a, b, _, da, db in w.layout] == lay
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(w.size), rng.standard_normal(w.size)
    hy, hx = w.apply(y), w.apply(x)
    assert abs(x @ hy - y @ hx) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(hy)


def test_full_bond_dimension_matches_ed():
    """Hubbard 3x3 torus, U = 4, 8 electrons, momentum basis: window 3 with
    complete (untruncated) multiplet bases spans the whole S = 0 space; its
    lowest eigenvalue is the ED ground energy over all 15876 S_z = 0 states."""
    m, h, W = _hubbard_3x3()
    e_ed = ed.ground_energy(h, W, 8, n_up=4)[0]
    li = synth.random_left_isometries_su2(9, (8, 0), 400, 3, 5)
    ri = synth.random_right_isometries_su2(9, (8, 0), 400, 5, 6)
    w = su2.Su2Window(m, 9, (8, 0), li, ri, 3)
    assert w.wz.size == 126 * 126
    e, v = w.solve(tol=1e-12)
    assert e == pytest.approx(e_ed, abs=1e-10)
