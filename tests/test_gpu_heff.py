"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Both sides get the same seeded inputs (lattice parameters, the Haar factor
of the mode rotation, random isometries, random psi) and build everything
else -- lattice Hamiltonian, momentum basis, rotation, block operators --
with their own code.

Tolerances
  * FP64 path: relative 2-norm error of sigma <= 1e-12.
  * split path (FP16 hi + lo with per-block power-of-two scales, three
    products, FP32 accumulation): relative 2-norm error of sigma <= 2e-5.
    Operands carry ~22 significant bits and the accumulation is FP32, so
    the expected error is a few 1e-7 times sqrt(K) for K up to ~4e3.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg as odmrg
from oracle import ed, hamiltonian, lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402

TOL64 = 1e-12
TOL_SPLIT = 2e-5


def problem(Lx, Ly, spinful, target, rot_seed=2, V=1.0, U=4.0, tp=0.0):
    N = Lx * Ly
    Q = synth.haar_rotation(N, rot_seed) if rot_seed is not None else np.eye(N)
    # oracle side
    if spinful:
        To, Vo = lattice.hubbard(Lx, Ly, 1.0, U)
    else:
        To, Vo = lattice.spinless_tV(Lx, Ly, 1.0, tp, V)
    Uo = lattice.momentum_basis(Lx, Ly) @ Q
    To, Vo = lattice.rotate(To, Vo, Uo)
    h, W = hamiltonian.spin_orbital(To, Vo, spinful)
    model = odmrg.Model(h, W, spinful, target)
    # library side (its own lattice and momentum basis)
    if spinful:
        Tg, Vg = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, Lx, Ly, 1.0, 0.0, U)
    else:
        Tg, Vg = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, Lx, Ly, 1.0, tp, V)
    Ug = lib.momentum_basis(Lx, Ly) @ Q
    return model, (Tg, Vg, Ug), h, W


def make_gpu(n_sites, target, spinful, ham, **kw):
    d = lib.Dmrg(n_sites, target[0], target[1] if spinful else 0, spinful=spinful, **kw)
    d.set_hamiltonian(*ham)
    return d


def window_case(Lx, Ly, spinful, target, D, l, seed=5, spread=None):
    model, ham, h, W = problem(Lx, Ly, spinful, target)
    N = Lx * Ly
    li = synth.random_left_isometries(N, spinful, target, D, l, seed, spread=spread)
    ri = synth.random_right_isometries(N, spinful, target, D, l + 2, seed + 1, spread=spread)
    w = odmrg.window_from_mps(model, li, ri, l)
    g = make_gpu(N, target, spinful, ham, d_max=D)
    g.set_mps(li, ri)
    g.build_block_ops(l)
    n, lay = g.heff_layout()
    assert n == w.size
    assert lay == [(a, b, da, db) for a, b, _, da, db in w.layout]
    return w, g


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = ([("s3", 3, 3, False, (4,), 8, l) for l in range(8)]
         + [("h3", 3, 3, True, (5, 4), 16, l) for l in (0, 4, 7)]
         + [("s4", 4, 4, False, (8,), 64, 7), ("s4b", 4, 4, False, (8,), 128, 5)])


@pytest.mark.parametrize("name,Lx,Ly,spinful,target,D,l", CASES)
def test_heff_fp64_and_split_vs_oracle(name, Lx, Ly, spinful, target, D, l):
    w, g = window_case(Lx, Ly, spinful, target, D, l)
    psi = synth.random_psi([(a, b, da, db) for a, b, _, da, db in w.layout], 11)
    ref = w.apply(psi)
    g.set_precision(lib.FP64)
    s64 = g.heff_apply_host(psi)
    assert rel(s64, ref) <= TOL64, rel(s64, ref)
    g.set_precision(lib.SPLIT)
    s32 = g.heff_apply_host(psi)
    assert rel(s32, ref) <= TOL_SPLIT, rel(s32, ref)
    # repeated applies (graph replay) are bitwise reproducible
    assert np.array_equal(g.heff_apply_host(psi), s32)
    # device-pointer entry point agrees with the host one
    x = torch.tensor(psi, device="cuda")
    y = torch.empty_like(x)
    g.set_precision(lib.FP64)
    g.heff_apply(x, y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), s64)


def block_errors(s, ref, layout, floor_rel=1e-6):
    """Relative error of every sigma block (norms below floor_rel of the
    whole sigma are judged against that floor)."""
    floor = floor_rel * np.linalg.norm(ref)
    out, o = [], 0
    for _, _, da, db in layout:
        r, x = ref[o:o + da * db], s[o:o + da * db]
        out.append(np.linalg.norm(x - r) / max(np.linalg.norm(r), floor))
        o += da * db
    return np.array(out)


# Windows whose split plan reaches every code path of the tcgen05 kernels:
# sigma blocks longer than 128 on a side (two MMA tiles), several split-K
# partial tiles per block, and the R = 2 and R = 4 packing of small blocks.
# The MPS sectors are concentrated (spread) so that D = 200-256 gives blocks
# of up to 150-165 rows while the oracle still builds the window in under a
# minute.
FULL_CASES = [("h4_D256", 4, 4, True, (8, 8), 256, 7, 0.6),
              ("s6_D200", 6, 6, False, (18,), 200, 17, 0.8)]


@pytest.mark.parametrize("name,Lx,Ly,spinful,target,D,l,spread", FULL_CASES)
def test_full_size_paths_vs_oracle(name, Lx, Ly, spinful, target, D, l, spread):
    w, g = window_case(Lx, Ly, spinful, target, D, l, spread=spread)
    n, layout = g.heff_layout()
    psi = synth.random_psi(layout, 11)
    ref = w.apply(psi)
    g.set_precision(lib.FP64)
    s64 = g.heff_apply_host(psi)
    assert rel(s64, ref) <= TOL64, rel(s64, ref)
    e64 = block_errors(s64, ref, layout)
    assert e64.max() <= 1e-11, (e64.max(), int(e64.argmax()))
    g.set_precision(lib.SPLIT)
    s32 = g.heff_apply_host(psi)
    assert rel(s32, ref) <= TOL_SPLIT, rel(s32, ref)
    e32 = block_errors(s32, ref, layout)
    assert e32.max() <= 10 * TOL_SPLIT, (e32.max(), int(e32.argmax()), layout[int(e32.argmax())])
    paths = g.heff_split_paths()
    assert paths["wide_blocks"] > 0, paths
    assert paths["extra_tiles"] > 0, paths
    assert paths["multi_part_blocks"] > 0 and paths["max_parts"] >= 3, paths
    if name == "h4_D256":
        assert paths["packed_r2"] > 0 and paths["packed_r4"] > 0, paths
    g.close()


def test_heff_flops_matches_layout_count():
    w, g = window_case(4, 4, False, (8,), 64, 7)
    f = g.heff_flops()
    assert f > 0
    # every term contributes 2 (m'mn + m'nn') per nonzero sector block; the
    # oracle's term list includes identity factors exactly as the library's
    assert f >= 2 * sum(da * da * db for _, _, _, da, db in w.layout)


def test_davidson_energy_vs_oracle():
    w, g = window_case(4, 4, False, (8,), 64, 7)
    e_ref, _ = w.solve(tol=1e-12)
    for prec in (lib.FP64, lib.SPLIT):
        g.set_precision(prec)
        x = torch.zeros(w.size, dtype=torch.float64, device="cuda")
        e, it, conv = g.davidson(x)
        assert conv
        assert abs(e - e_ref) <= 1e-9 * abs(e_ref), (prec, e, e_ref)
        v = x.cpu().numpy()
        assert abs(np.linalg.norm(v) - 1) < 1e-10


def test_sweep_matches_ed_spinless_3x3():
    model, ham, h, W = problem(3, 3, False, (4,))
    e_ed = ed.ground_energy(h, W, 4)[0]
    g = make_gpu(9, (4,), False, ham, d_max=20, davidson_tol=1e-9)
    g.set_mps(right=synth.random_right_isometries(9, False, (4,), 20, 1, 0))
    E = g.sweep(2)
    assert abs(E[-1] - e_ed) <= 1e-9 * abs(e_ed), (E, e_ed)


def test_sweep_split_matches_ed_spinless_3x3():
    model, ham, h, W = problem(3, 3, False, (4,))
    e_ed = ed.ground_energy(h, W, 4)[0]
    g = make_gpu(9, (4,), False, ham, d_max=20, davidson_tol=1e-9, precision=lib.SPLIT)
    g.set_mps(right=synth.random_right_isometries(9, False, (4,), 20, 1, 0))
    E = g.sweep(2)
    assert abs(E[-1] - e_ed) <= 1e-9 * abs(e_ed), (E, e_ed)


def test_split_min_flops_solves_small_windows_in_fp64():
    """dmrg_set_split_min_flops above every window's flops: a split context
    sweeps exactly as an FP64 one (bitwise equal energies)."""
    model, ham, h, W = problem(3, 3, False, (4,))
    E = {}
    for prec in (lib.FP64, lib.SPLIT):
        g = make_gpu(9, (4,), False, ham, d_max=20, davidson_tol=1e-9, precision=prec)
        g.set_split_min_flops(1e30)
        g.set_mps(right=synth.random_right_isometries(9, False, (4,), 20, 1, 0))
        E[prec] = g.sweep(2)
        g.close()
    assert np.array_equal(E[lib.FP64], E[lib.SPLIT]), E


# Hubbard runs in U(1)xU(1) sectors: the members of a spin multiplet have
# exactly equal Schmidt weights in different S_z sectors, so where the cut at
# D falls inside a multiplet, which members are kept is decided by rounding
# noise, and two correct runs can keep different ones.  Their energies then
# differ at the level of the truncation error, not 1e-9; the 1e-9 criterion
# is checked on spinless runs (no spin) and on U(1)xSU(2) runs (D counts
# multiplets).
TOL_U1U1_SWEEP = 1e-6


@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_sweep_hubbard_3x3_variational_and_matches_oracle(prec):
    """Identical D and sweep schedule from the same MPS: the energy of both
    precisions against the oracle's (the split path through its FP64
    refinement), within TOL_U1U1_SWEEP."""
    model, ham, h, W = problem(3, 3, True, (5, 4), rot_seed=None)
    e_ed = ed.ground_energy(h, W, 9, n_up=5)[0]
    ri = synth.random_right_isometries(9, True, (5, 4), 16, 1, 0)
    g = make_gpu(9, (5, 4), True, ham, d_max=16, davidson_tol=1e-10, precision=prec)
    g.set_mps(right=ri)
    E = g.sweep(1)
    Eo, hist = odmrg.sweep(model, {n: ri[n] for n in ri if n >= 2}, 16, 1, tol=1e-12)
    assert E[-1] >= e_ed - 1e-9
    assert abs(E[-1] - Eo[-1]) <= TOL_U1U1_SWEEP * abs(e_ed), (E, Eo)


_ORACLE_SWEEPS = {}


def oracle_sweep_spinless_4x4():
    if not _ORACLE_SWEEPS:
        model, ham, h, W = problem(4, 4, False, (8,))
        ri = synth.random_right_isometries(16, False, (8,), 48, 1, 3)
        Eo, _ = odmrg.sweep(model, {n: ri[n] for n in ri if n >= 2}, 48, 2, tol=1e-12)
        _ORACLE_SWEEPS["s4"] = (ham, ri, Eo)
    return _ORACLE_SWEEPS["s4"]


@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_sweeps_match_oracle_spinless_4x4(prec):
    """C1-type lattice (4x4 spinless t-V, momentum basis with a Haar factor),
    D = 48, two sweeps from the same MPS: energies within 1e-9 relative of
    the oracle's at every sweep."""
    ham, ri, Eo = oracle_sweep_spinless_4x4()
    g = make_gpu(16, (8,), False, ham, d_max=48, davidson_tol=1e-10, precision=prec)
    g.set_mps(right=ri)
    E = g.sweep(2)
    for a, b in zip(E, Eo):
        assert abs(a - b) <= 1e-9 * abs(b), (E, Eo)
    g.close()


@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_sweep_4x4_full_D_exact_and_D128_gap(prec):
    """4x4 spinless model at the paper's Fig. 1 parameters (t'=0.4, V=0.8, half
    filling), momentum basis, vs ED over all 12870 states.  At D = 256 (the
    largest Schmidt rank of the middle cut) the sweep is exact.  Sec. III.A
    reports exactness already at D = 128 in its optimized basis; in the
    momentum basis the D = 128 result must be variational and close (gap
    reported in the assertion message)."""
    model, ham, h, W = problem(4, 4, False, (8,), rot_seed=None, V=0.8, tp=0.4)
    e_ed = ed.ground_energy(h, W, 8)[0]
    for D, nsw, tol in ((256, 3, 1e-9), (128, 3, 1e-4)):
        g = make_gpu(16, (8,), False, ham, d_max=D, davidson_tol=1e-9, precision=prec)
        g.set_mps(right=synth.random_right_isometries(16, False, (8,), D, 1, 0))
        E = g.sweep(nsw)
        assert E[-1] >= e_ed - 1e-9 * abs(e_ed), (D, E, e_ed)
        assert abs(E[-1] - e_ed) <= tol * abs(e_ed), (D, E, e_ed, g.profile())
        g.close()


def test_split_sweeps_follow_fp64_hubbard_4x4():
    """Hubbard 4x4 (U = 4, half filling, momentum basis), D = 128 states, two
    sweeps from the same random MPS: the split path (with its FP64
    refinement) ends where the FP64 path does, within TOL_U1U1_SWEEP (see
    there).  From this start an early window has an excited state that
    converges before the ground state appears; a Davidson that stopped at
    the split noise floor kept it and ended 0.7 % higher."""
    T, V = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 4, 4, 1.0, 0.0, 4.0)
    U = lib.momentum_basis(4, 4)
    E = {}
    for prec in (lib.FP64, lib.SPLIT):
        g = lib.Dmrg(16, 8, 8, spinful=True, d_max=128, precision=prec, davidson_tol=1e-9, seed=7)
        g.set_hamiltonian(T, V, U)
        g.set_mps(right=synth.random_right_isometries(16, True, (8, 8), 128, 1, 7))
        E[prec] = g.sweep(2)
        g.close()
    for a, b in zip(E[lib.SPLIT], E[lib.FP64]):
        assert abs(a - b) <= TOL_U1U1_SWEEP * abs(b), E


@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_window_rebuild_while_apply_in_flight(prec):
    """The window is rebuilt (new couplings, same sizes) while an H_eff*psi
    enqueued on another stream has not started yet.  The old window's
    buffers go back to the memory pool without a device synchronisation, but
    only after that apply, so it still computes the old operator exactly."""
    w, g = window_case(4, 4, False, (8,), 64, 7)
    g.set_precision(prec)
    psi = torch.tensor(np.random.default_rng(3).standard_normal(w.size), device="cuda")
    ref = torch.empty_like(psi)
    g.heff_apply(psi, ref)
    torch.cuda.synchronize()
    side, other = torch.cuda.Stream(), torch.cuda.Stream()
    sig = torch.zeros_like(psi)
    with torch.cuda.stream(side):
        torch.cuda._sleep(200_000_000)   # about 0.1 s: the apply below waits behind it
    g.heff_apply(psi, sig, stream=side)
    _, ham, _, _ = problem(4, 4, False, (8,), V=2.5)
    g.set_hamiltonian(*ham)
    g.build_block_ops(7, stream=other)
    side.synchronize()
    assert torch.equal(sig, ref)
    new = torch.empty_like(psi)
    g.heff_apply(psi, new, stream=other)
    other.synchronize()
    assert rel(new.cpu().numpy(), ref.cpu().numpy()) > 1e-3
    g.close()


def test_graph_cache_many_buffer_pairs():
    """The split apply replays a captured graph per (psi, sigma) pointer pair
    and keeps at most 64 of them per window: 70 different output buffers
    (the cache is flushed once on the way) all give the same sigma."""
    w, g = window_case(4, 4, False, (8,), 64, 7)
    g.set_precision(lib.SPLIT)
    psi = torch.tensor(np.random.default_rng(4).standard_normal(w.size), device="cuda")
    ref = torch.empty_like(psi)
    g.heff_apply(psi, ref)
    outs = [torch.empty_like(psi) for _ in range(70)]
    for o in outs:
        g.heff_apply(psi, o)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)
    g.close()


def test_sweep_from_library_random_start_matches_ed():
    """dmrg_random_start (the library's own seeded start, used by serving):
    spinless 3x3, two sweeps at D = 20 reach the ED ground energy."""
    model, ham, h, W = problem(3, 3, False, (4,))
    e_ed = ed.ground_energy(h, W, 4)[0]
    g = make_gpu(9, (4,), False, ham, d_max=20, davidson_tol=1e-10)
    g.random_start(11)
    E = g.sweep(2)
    assert abs(E[-1] - e_ed) <= 1e-9 * abs(e_ed), (E, e_ed)
    g.close()
