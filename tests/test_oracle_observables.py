"""Pins of the oracle's observables: ED ground-state 1-RDM and expectation
values, and the CDW operator (Sec. III.C), against closed forms."""
import numpy as np
import pytest

from oracle import ed, hamiltonian, lattice


def _free(N, n, seed):
    """Random real one-body t (non-degenerate levels), no interaction."""
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((N, N))
    return T + T.T


def test_rdm1_of_a_slater_determinant_is_the_occupied_projector():
    """V = 0: the ground state fills the n lowest one-body levels, so
    gamma = sum_occupied phi phi^T (closed form)."""
    N, n = 7, 3
    T = _free(N, n, 4)
    h, W = hamiltonian.spin_orbital(T, np.zeros((N,) * 4), False)
    e0, v, fs = ed.ground_state(h, W, n)
    g = ed.rdm1(fs, v)
    w, phi = np.linalg.eigh(T)
    P = phi[:, :n] @ phi[:, :n].T
    assert np.abs(g - P).max() < 1e-10
    assert e0 == pytest.approx(w[:n].sum(), abs=1e-10)
    assert ed.expectation(fs, h, W, v) == pytest.approx(e0, abs=1e-10)


def test_rdm1_invariants_interacting():
    T, V4 = lattice.spinless_tV(3, 3, 1.0, 0.3, 1.7)
    h, W = hamiltonian.spin_orbital(T, V4, False)
    e0, v, fs = ed.ground_state(h, W, 4)
    g = ed.rdm1(fs, v)
    assert np.trace(g) == pytest.approx(4.0, abs=1e-10)
    assert np.abs(g - g.T).max() < 1e-12
    lam = np.linalg.eigvalsh(g)
    assert lam.min() > -1e-10 and lam.max() < 1 + 1e-10


def test_cdw_square_wick_and_classical_limits():
    """<(n_even - n_odd)^2> of a Slater determinant by Wick's theorem,
    sum_i g_ii + sum_{i != j} s_i s_j (g_ii g_jj - g_ij g_ji), against the ED
    expectation of the Eq. 1 operator; and a classical configuration (the
    t = 0, V > 0 ground state of a 4x4 torus at half filling is the
    checkerboard, (n_even - n_odd)^2 = N^2)."""
    Lx, Ly, n = 4, 3, 5
    N = Lx * Ly
    T = _free(N, n, 9)
    h, W = hamiltonian.spin_orbital(T, np.zeros((N,) * 4), False)
    e0, v, fs = ed.ground_state(h, W, n)
    g = ed.rdm1(fs, v)
    To, Vo = lattice.cdw_square(Lx, Ly)
    ho, Wo = hamiltonian.spin_orbital(To, Vo, False)
    s = np.array([1.0 - 2.0 * (((i % Lx) + (i // Lx)) % 2) for i in range(N)])
    wick = np.trace(g) + sum(s[i] * s[j] * (g[i, i] * g[j, j] - g[i, j] * g[j, i])
                             for i in range(N) for j in range(N) if i != j)
    assert ed.expectation(fs, ho, Wo, v) == pytest.approx(wick, abs=1e-9)
    # classical limit: 4x4 checkerboard
    T4, V4 = lattice.spinless_tV(4, 4, 0.0, 0.0, 1.0)
    h4, W4 = hamiltonian.spin_orbital(T4, V4, False)
    e4, v4, fs4 = ed.ground_state(h4, W4, 8)
    assert e4 == pytest.approx(0.0, abs=1e-10)
    To4, Vo4 = lattice.cdw_square(4, 4)
    ho4, Wo4 = hamiltonian.spin_orbital(To4, Vo4, False)
    # the two checkerboards are degenerate: any ground state has |n_e - n_o| = 8
    assert ed.expectation(fs4, ho4, Wo4, v4) == pytest.approx(64.0, abs=1e-8)
