"""Several H_eff*psi products in one pass of the split kernels.

dmrg_heff_apply_batch runs nv vectors through one plan whose work items are
the single-vector items once per vector; each vector sees the same tiles, K
ranges and partial-sum order, so its sigma must be bitwise the single-vector
result, and that one is pinned to the oracle in test_gpu_heff.py /
test_gpu_su2.py (checked here once more against the oracle).
"""
import numpy as np
import pytest

import synth
from oracle import dmrg as odmrg
from oracle import hamiltonian, lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402


def _window(su2):
    if su2:
        N, ne, D, l = 16, 16, 96, 7
        T, V = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 4, 4, 1.0, 0.0, 4.0)
        g = lib.Dmrg(N, ne, su2=True, d_max=D, precision=lib.SPLIT)
        g.set_hamiltonian(T, V, lib.momentum_basis(4, 4))
        g.set_mps(synth.random_left_isometries_su2(N, (ne, 0), D, l, 5, spread=0.7),
                  synth.random_right_isometries_su2(N, (ne, 0), D, l + 2, 6, spread=0.7))
    else:
        N, D, l = 16, 128, 7
        T, V = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, 4, 4, 1.0, 0.0, 1.0)
        g = lib.Dmrg(N, 8, d_max=D, precision=lib.SPLIT)
        g.set_hamiltonian(T, V, lib.momentum_basis(4, 4))
        g.set_mps(synth.random_left_isometries(N, False, (8,), D, l, 5),
                  synth.random_right_isometries(N, False, (8,), D, l + 2, 6))
    g.build_block_ops(l)
    return g


@pytest.mark.parametrize("su2", [False, True])
@pytest.mark.parametrize("nv", [2, 5])
def test_batch_equals_single_applies_bitwise(su2, nv):
    g = _window(su2)
    n, lay = g.heff_layout()
    rng = np.random.default_rng(nv)
    psi = torch.tensor(rng.standard_normal((nv, n)), device="cuda")
    sig = torch.empty_like(psi)
    g.heff_apply_batch(psi, sig)
    for rep in range(2):   # the second pass replays the captured graph
        if rep:
            sig.zero_()
            g.heff_apply_batch(psi, sig)
        g.sync()
        for v in range(nv):
            one = torch.empty(n, dtype=torch.float64, device="cuda")
            g.heff_apply(psi[v].contiguous(), one)
            g.sync()
            assert torch.equal(one, sig[v]), (v, rep)
    g.close()


def test_batch_vs_oracle_spinless():
    Lx = Ly = 4
    N, D, l = 16, 128, 7
    T, V = lattice.spinless_tV(Lx, Ly, 1.0, 0.0, 1.0)
    T, V = lattice.rotate(T, V, lattice.momentum_basis(Lx, Ly))
    h, W = hamiltonian.spin_orbital(T, V, False)
    model = odmrg.Model(h, W, False, (8,))
    w = odmrg.window_from_mps(model, synth.random_left_isometries(N, False, (8,), D, l, 5),
                              synth.random_right_isometries(N, False, (8,), D, l + 2, 6), l)
    g = _window(False)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((3, w.size))
    sig = torch.empty(3, w.size, dtype=torch.float64, device="cuda")
    g.heff_apply_batch(torch.tensor(X, device="cuda"), sig)
    g.sync()
    S = sig.cpu().numpy()
    for v in range(3):
        ref = w.apply(X[v])
        assert np.linalg.norm(S[v] - ref) <= 2e-5 * np.linalg.norm(ref)
    g.close()
