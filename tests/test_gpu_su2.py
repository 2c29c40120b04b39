"""GPU parity of the spin-adapted (U(1)xSU(2)) path against the oracle.

The library builds spin-adapted block operators (reduced matrix elements
between spin multiplets, D counting multiplets, Sec. IV) and runs the same
tcgen05 / FP64 H_eff*psi kernels on them; the oracle defines the spin-adapted
sigma as E^T H_eff^{S_z} E psi through the exact Clebsch-Gordan expansion of
the multiplet basis (oracle/su2.py).  Both get the same seeded inputs (the
multiplet isometries of synth, psi) and build everything else themselves.

Tolerances as for the S_z path: FP64 sigma <= 1e-12 relative 2-norm (and per
block), split <= 2e-5 (per block <= 2e-4, floor 1e-6 of |sigma|).
"""
import numpy as np
import pytest

import synth
from oracle import dmrg as odmrg
from oracle import ed, hamiltonian, lattice, su2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402

TOL64 = 1e-12
TOL_SPLIT = 2e-5


def generic(N, seed):
    """Random real Hermitian Eq. 1 coefficients (V[ijkl] = V[lkji])."""
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((N, N))
    T = T + T.T
    X = rng.standard_normal((N,) * 4) * 0.3
    return T, X + X.transpose(3, 2, 1, 0), None


def hubbard(Lx, Ly, U=4.0, rot_seed=None):
    T, V = lattice.hubbard(Lx, Ly, 1.0, U)
    Um = lattice.momentum_basis(Lx, Ly)
    if rot_seed is not None:
        Um = Um @ synth.haar_rotation(Lx * Ly, rot_seed)
    return T, V, Um


def oracle_model(ham, ne):
    T, V, Um = ham
    if Um is not None:
        T, V = lattice.rotate(T, V, Um)
    h, W = hamiltonian.spin_orbital(T, V, True)
    return odmrg.Model(h, W, True, (ne // 2, ne // 2)), h, W


def library(N, ne, ham, D, **kw):
    T, V, Um = ham
    g = lib.Dmrg(N, ne, su2=True, d_max=D, **kw)
    g.set_hamiltonian(T, V, Um)
    return g


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def block_errors(s, ref, layout, floor_rel=1e-6):
    floor = floor_rel * np.linalg.norm(ref)
    out, o = [], 0
    for _, _, da, db in layout:
        r, x = ref[o:o + da * db], s[o:o + da * db]
        out.append(np.linalg.norm(x - r) / max(np.linalg.norm(r), floor))
        o += da * db
    return np.array(out)


def window(N, ne, ham, D, l, spread=None, seed=5):
    model, h, W = oracle_model(ham, ne)
    li = synth.random_left_isometries_su2(N, (ne, 0), D, l, seed, spread=spread)
    ri = synth.random_right_isometries_su2(N, (ne, 0), D, l + 2, seed + 1, spread=spread)
    w = su2.Su2Window(model, N, (ne, 0), li, ri, l)
    g = library(N, ne, ham, D)
    g.set_mps(li, ri)
    g.build_block_ops(l)
    n, lay = g.heff_layout()
    assert n == w.size
    assert lay == [(a, b, da, db) for a, b, _, da, db in w.layout]
    return w, g, lay


GEN4 = generic(4, 3)
CASES = ([("gen4", 4, 4, GEN4, 8, l, None) for l in range(3)]
         + [("hub3", 9, 8, hubbard(3, 3), 12, l, None) for l in (0, 3, 5, 7)]
         + [("hub3q", 9, 8, hubbard(3, 3, rot_seed=2), 16, 4, None),
            ("hub4", 16, 16, hubbard(4, 4, rot_seed=2), 64, 7, None)])


@pytest.mark.parametrize("name,N,ne,ham,D,l,spread", CASES)
def test_su2_heff_vs_oracle(name, N, ne, ham, D, l, spread):
    w, g, lay = window(N, ne, ham, D, l, spread)
    psi = synth.random_psi(lay, 11)
    ref = w.apply(psi)
    g.set_precision(lib.FP64)
    s64 = g.heff_apply_host(psi)
    assert rel(s64, ref) <= TOL64, rel(s64, ref)
    assert block_errors(s64, ref, lay).max() <= 1e-11
    g.set_precision(lib.SPLIT)
    s32 = g.heff_apply_host(psi)
    assert rel(s32, ref) <= TOL_SPLIT, rel(s32, ref)
    assert block_errors(s32, ref, lay).max() <= 10 * TOL_SPLIT
    g.close()


def test_su2_full_size_paths_vs_oracle():
    """Hubbard 4x4, 16 electrons, S = 0, momentum basis with a Haar factor,
    D = 220 multiplets concentrated in few sectors: psi blocks up to 173
    multiplets on a side (two MMA tiles), long split-K ranges and packed
    small blocks in the split plan."""
    w, g, lay = window(16, 16, hubbard(4, 4, rot_seed=2), 220, 7, spread=0.5)
    psi = synth.random_psi(lay, 11)
    ref = w.apply(psi)
    g.set_precision(lib.FP64)
    s64 = g.heff_apply_host(psi)
    assert rel(s64, ref) <= TOL64, rel(s64, ref)
    assert block_errors(s64, ref, lay).max() <= 1e-11
    g.set_precision(lib.SPLIT)
    s32 = g.heff_apply_host(psi)
    assert rel(s32, ref) <= TOL_SPLIT, rel(s32, ref)
    assert block_errors(s32, ref, lay).max() <= 10 * TOL_SPLIT
    paths = g.heff_split_paths()
    assert paths["wide_blocks"] > 0 and paths["extra_tiles"] > 0, paths
    assert paths["multi_part_blocks"] > 0, paths
    assert paths["packed_r2"] + paths["packed_r4"] > 0, paths
    g.close()


def test_su2_davidson_energy_vs_oracle():
    w, g, lay = window(9, 8, hubbard(3, 3, rot_seed=2), 16, 4)
    e_ref, _ = w.solve(tol=1e-12)
    for prec in (lib.FP64, lib.SPLIT):
        g.set_precision(prec)
        x = torch.zeros(w.size, dtype=torch.float64, device="cuda")
        e, it, conv = g.davidson(x)
        assert conv
        assert abs(e - e_ref) <= 1e-9 * abs(e_ref), (prec, e, e_ref)
    g.close()


@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_su2_sweep_exact_at_full_D(prec):
    """Hubbard 3x3 torus, U = 4, 8 electrons (singlet ground state), momentum
    basis: with D = 400 multiplets nothing is truncated and two sweeps reach
    the ED ground energy over the 15876-state S_z = 0 sector.  The second
    sweep starts every window from the transformed previous state, so it
    needs few matvecs."""
    ham = hubbard(3, 3)
    model, h, W = oracle_model(ham, 8)
    e_ed = ed.ground_energy(h, W, 8, n_up=4)[0]
    g = library(9, 8, ham, 400, davidson_tol=1e-10, precision=prec)
    g.set_mps(right=synth.random_right_isometries_su2(9, (8, 0), 400, 1, 0))
    E = g.sweep(2)
    assert g.sweep_converged
    assert abs(E[-1] - e_ed) <= 1e-9 * abs(e_ed), (E, e_ed)
    g.close()


def test_su2_split_sweeps_match_fp64_at_truncated_D():
    """Hubbard 4x4, U = 4, half filling, momentum basis, D = 48 multiplets,
    two sweeps from the same random MPS: the split path with its FP64
    refinement ends within 1e-9 relative of the FP64 path at every sweep.
    (D counts multiplets, so no truncation splits a multiplet.)  The window
    solves converge to a residual of 1e-10: the residual left in early
    windows reaches the final energy to first order through the truncations
    of the first sweep (with 1e-9 the first-sweep energies differed by 2e-9)."""
    ham = hubbard(4, 4)
    E = {}
    for prec in (lib.FP64, lib.SPLIT):
        g = library(16, 16, ham, 48, davidson_tol=1e-10, precision=prec, seed=3)
        g.set_mps(right=synth.random_right_isometries_su2(16, (16, 0), 48, 1, 7))
        E[prec] = g.sweep(2)
        g.close()
    for a, b in zip(E[lib.SPLIT], E[lib.FP64]):
        assert abs(a - b) <= 1e-9 * abs(b), E


@pytest.mark.parametrize("steps", [8, 20])
def test_su2_split_sweeps_with_correction_equation_refinement(steps):
    """The same two sweeps with the refinement's correction-equation steps
    forced on every window (dmrg_set_refinement with no flop threshold): the
    split path still ends within 1e-9 relative of the FP64 path."""
    ham = hubbard(4, 4)
    E = {}
    for prec in (lib.FP64, lib.SPLIT):
        g = library(16, 16, ham, 48, davidson_tol=1e-10, precision=prec, seed=3)
        g.set_refinement(steps, 0.0)
        g.set_mps(right=synth.random_right_isometries_su2(16, (16, 0), 48, 1, 7))
        E[prec] = g.sweep(2)
        g.close()
    for a, b in zip(E[lib.SPLIT], E[lib.FP64]):
        assert abs(a - b) <= 1e-9 * abs(b), E


def test_su2_sweep_from_library_random_start():
    """dmrg_random_start in multiplet sectors: Hubbard 3x3, 8 electrons, full
    D, two sweeps reach the ED ground energy."""
    ham = hubbard(3, 3)
    model, h, W = oracle_model(ham, 8)
    e_ed = ed.ground_energy(h, W, 8, n_up=4)[0]
    g = library(9, 8, ham, 400, davidson_tol=1e-10)
    g.random_start(5)
    E = g.sweep(2)
    assert abs(E[-1] - e_ed) <= 1e-9 * abs(e_ed), (E, e_ed)
    g.close()
