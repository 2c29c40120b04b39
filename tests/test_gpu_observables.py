"""Observables of a converged sweep against exact diagonalisation.

At a bond dimension where nothing is truncated the sweep's final state is the
ED ground state (non-degenerate cases), so its one-particle reduced density
matrix (dmrg_rdm1, mode basis; back-rotated to real space) and expectation
values of Eq. 1 operators (the CDW order parameter of Sec. III.C) must agree
with the ED ones.  ED works in the Fock space of the oracle, independently of
the block-operator algebra.
"""
import numpy as np
import pytest

import synth
from oracle import ed, hamiltonian, lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402
from paper_2311_14106_b300 import observables as obs  # noqa: E402


def generic(N, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((N, N))
    T = T + T.T
    X = rng.standard_normal((N,) * 4) * scale
    return T, X + X.transpose(3, 2, 1, 0)


def spatial(g):
    """Spin-summed spatial 1-RDM from a spin-orbital one (p = 2 i + spin)."""
    return g[0::2, 0::2] + g[1::2, 1::2]


def ed_state(T, V, U, spinful, n, n_up=None):
    if U is not None:
        T, V = lattice.rotate(T, V, U)
    h, W = hamiltonian.spin_orbital(T, V, spinful)
    return ed.ground_state(h, W, n, n_up=n_up)


def test_rdm1_spinless_generic():
    N, n = 8, 4
    T, V = generic(N, 21)
    e0, v, fs = ed_state(T, V, None, False, n)
    g = lib.Dmrg(N, n, d_max=70, davidson_tol=1e-11)
    g.set_hamiltonian(T, V, None)
    g.set_mps(right=synth.random_right_isometries(N, False, (n,), 70, 1, 0))
    E = g.sweep(2)
    assert abs(E[-1] - e0) <= 1e-9 * abs(e0)
    gam = obs.rdm1_final(g)
    assert np.abs(gam - ed.rdm1(fs, v)).max() <= 1e-8
    g.close()


@pytest.mark.parametrize("su2", [False, True])
def test_rdm1_spinful_generic(su2):
    N = 4
    T, V = generic(N, 5)
    e0, v, fs = ed_state(T, V, None, True, 4, n_up=2)
    # the S_z = 1 sector lies higher: the ground state is a singlet
    e1 = ed_state(T, V, None, True, 4, n_up=3)[0]
    assert e1 > e0 + 1e-6
    if su2:
        g = lib.Dmrg(N, 4, su2=True, d_max=64, davidson_tol=1e-11)
        g.set_hamiltonian(T, V, None)
        g.set_mps(right=synth.random_right_isometries_su2(N, (4, 0), 64, 1, 0))
    else:
        g = lib.Dmrg(N, 2, 2, spinful=True, d_max=64, davidson_tol=1e-11)
        g.set_hamiltonian(T, V, None)
        g.set_mps(right=synth.random_right_isometries(N, True, (2, 2), 64, 1, 0))
    E = g.sweep(2)
    assert abs(E[-1] - e0) <= 1e-9 * abs(e0)
    gam = obs.rdm1_final(g)
    ref = spatial(ed.rdm1(fs, v))
    assert np.abs(gam - ref).max() <= 1e-8, np.abs(gam - ref).max()
    g.close()


def test_rdm1_back_rotation_to_real_space():
    """A run in a rotated mode basis (Haar factor): U gamma U^T equals the 1-RDM
    of the real-space ED ground state."""
    N, n = 6, 3
    T, V = generic(N, 8)
    U = synth.haar_rotation(N, 3)
    e0, v, fs = ed_state(T, V, None, False, n)       # real space
    g = lib.Dmrg(N, n, d_max=20, davidson_tol=1e-11)
    g.set_hamiltonian(T, V, U)
    g.set_mps(right=synth.random_right_isometries(N, False, (n,), 20, 1, 0))
    E = g.sweep(2)
    assert abs(E[-1] - e0) <= 1e-9 * abs(e0)
    real = obs.back_rotate(obs.rdm1_final(g), U)
    assert np.abs(real - ed.rdm1(fs, v)).max() <= 1e-8
    g.close()


def test_cdw_order_parameter_c1_lattice():
    """Config C1's lattice (4x4 spinless t-V, 8 particles, V = 1) in the
    momentum basis at D = 256 (exact): C_CDW from the library against the ED
    value of <(n_even - n_odd)^2> / N^2 in real space (12870 states)."""
    T, V = lattice.spinless_tV(4, 4, 1.0, 0.0, 1.0)
    e0, v, fs = ed_state(T, V, None, False, 8)
    To, Vo = lattice.cdw_square(4, 4)
    ho, Wo = hamiltonian.spin_orbital(To, Vo, False)
    c_ed = ed.expectation(fs, ho, Wo, v) / 16.0 ** 2
    Tg, Vg = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, 4, 4, 1.0, 0.0, 1.0)
    U = lib.momentum_basis(4, 4)
    g = lib.Dmrg(16, 8, d_max=256, davidson_tol=1e-10)
    g.set_hamiltonian(Tg, Vg, U)
    g.set_mps(right=synth.random_right_isometries(16, False, (8,), 256, 1, 0))
    E = g.sweep(3)
    assert abs(E[-1] - e0) <= 1e-9 * abs(e0)
    c = obs.cdw_order_parameter(g, 4, 4, U)
    assert abs(c - c_ed) <= 1e-8 * abs(c_ed), (c, c_ed)
    g.close()


def test_cdw_and_rdm1_spin_adapted_hubbard_3x3():
    """Hubbard 3x3, U = 4, 8 electrons (non-degenerate singlet ground state),
    momentum basis, spin-adapted at D = 400 multiplets (exact): the
    spin-summed 1-RDM (back-rotated) and <(sum_i s_i n_i)^2> against ED."""
    T, V = lattice.hubbard(3, 3, 1.0, 4.0)
    e0, v, fs = ed_state(T, V, None, True, 8, n_up=4)
    To, Vo = lattice.cdw_square(3, 3)
    ho, Wo = hamiltonian.spin_orbital(To, Vo, True)
    o_ed = ed.expectation(fs, ho, Wo, v)
    U = lib.momentum_basis(3, 3)
    Tg, Vg = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 3, 3, 1.0, 0.0, 4.0)
    g = lib.Dmrg(9, 8, su2=True, d_max=400, davidson_tol=1e-11)
    g.set_hamiltonian(Tg, Vg, U)
    g.set_mps(right=synth.random_right_isometries_su2(9, (8, 0), 400, 1, 0))
    E = g.sweep(2)
    assert abs(E[-1] - e0) <= 1e-9 * abs(e0)
    real = obs.back_rotate(obs.rdm1_final(g), U)
    assert np.abs(real - spatial(ed.rdm1(fs, v))).max() <= 1e-8
    Tc, Vc = obs.cdw_operator(3, 3)
    o = obs.expectation(g, Tc, Vc, U)
    assert abs(o - o_ed) <= 1e-8 * abs(o_ed), (o, o_ed)
    g.close()
