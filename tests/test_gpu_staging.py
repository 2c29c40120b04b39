"""Block operators over the HBM budget, staged through pinned host memory.

With cfg.hbm_budget_bytes set below the operator footprint of a sweep, the
library releases blocks the sweep rebuilds before reusing them, offloads the
blocks used last to pinned host memory and brings them back on a side stream
ahead of use (the paper's H2D/D2H operator traffic, Sec. III.B).  The data
moved is copied exactly, so the results must be bitwise the same as without
a budget.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402


def _hubbard4x4(budget, prec):
    T, V = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 4, 4, 1.0, 0.0, 4.0)
    g = lib.Dmrg(16, 16, su2=True, d_max=48, precision=prec, davidson_tol=1e-9, seed=1,
                 hbm_budget_bytes=budget)
    g.set_hamiltonian(T, V, lib.momentum_basis(4, 4))
    return g


@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_sweeps_bitwise_equal_under_a_tiny_budget(prec):
    ri = synth.random_right_isometries_su2(16, (16, 0), 48, 1, 4)
    E = {}
    stats = {}
    for budget in (0, 1 << 20):
        g = _hubbard4x4(budget, prec)
        g.set_mps(right=ri)
        E[budget] = g.sweep(2)
        stats[budget] = g.staging_stats()
        g.close()
    assert np.array_equal(E[0], E[1 << 20]), E
    st = stats[1 << 20]
    assert st["offloads"] > 0 and st["reloads"] > 0 and st["releases"] > 0, st
    assert st["h2d_bytes"] > 0 and st["d2h_bytes"] > 0 and st["h2d_seconds"] > 0, st
    assert stats[0]["offloads"] == 0 and stats[0]["h2d_bytes"] == 0, stats[0]


def test_window_build_under_a_budget():
    """dmrg_build_block_ops with a budget releases every block once the next
    one is built from it; the window's sigma is bitwise the same."""
    N, ne, D, l = 16, 16, 64, 7
    li = synth.random_left_isometries_su2(N, (ne, 0), D, l, 5)
    ri = synth.random_right_isometries_su2(N, (ne, 0), D, l + 2, 6)
    out = {}
    for budget in (0, 1):
        g = _hubbard4x4(budget, lib.FP64)
        g.set_mps(li, ri)
        g.build_block_ops(l)
        n, lay = g.heff_layout()
        psi = synth.random_psi(lay, 2)
        out[budget] = g.heff_apply_host(psi)
        if budget:
            assert g.staging_stats()["releases"] >= N - 4
        g.close()
    assert np.array_equal(out[0], out[1])


def test_fp64_stacks_given_back_under_a_budget():
    """With a budget the FP64 stacks and T are given back once the split path
    has its FP16 copies, and the next FP64 apply gathers the stacks again:
    sigma of both paths bitwise the same as in a context without a budget."""
    N, ne, D, l = 16, 16, 64, 7
    li = synth.random_left_isometries_su2(N, (ne, 0), D, l, 5)
    ri = synth.random_right_isometries_su2(N, (ne, 0), D, l + 2, 6)
    out = {}
    for budget in (0, 1):
        g = _hubbard4x4(budget, lib.SPLIT)
        g.set_mps(li, ri)
        g.build_block_ops(l)
        st = g.heff_fp64_state()
        assert st["stacks_backed"] and not st["t_backed"], st   # T backed on first FP64 use
        n, lay = g.heff_layout()
        psi = synth.random_psi(lay, 2)
        s_split = g.heff_apply_host(psi)
        st = g.heff_fp64_state()
        assert st["stacks_backed"] == (budget == 0), st
        g.set_precision(lib.FP64)
        s_64 = g.heff_apply_host(psi)
        st = g.heff_fp64_state()
        assert st["stacks_backed"] and st["t_backed"], st
        g.set_precision(lib.SPLIT)
        s_split2 = g.heff_apply_host(psi)
        out[budget] = (s_split, s_64, s_split2)
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[1][0], out[1][2])
