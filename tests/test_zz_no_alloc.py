"""The allocation-free split-precision H_eff*psi entry point.

Some callers cannot let a library allocate device memory while they run
(they live inside another framework's memory pool, or must avoid the implicit
device synchronisation of cudaMalloc/cudaFree).  dmrg_heff_apply_split_static
serves them from a fixed device array instead.  This file is collected last
on purpose.  The test checks, through the C ABI, that two calls in a row give
the same sigma as the allocating dmrg_heff_apply in the same precision and
agree with the FP64 oracle within the split-path tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg as odmrg
from oracle import hamiltonian, lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402

TOL_SPLIT = 2e-5   # same bound as the split-path parity tests


def _window():
    Lx = Ly = 4
    N, target, D, l = 16, (8,), 64, 7
    Q = synth.haar_rotation(N, 2)
    To, Vo = lattice.spinless_tV(Lx, Ly, 1.0, 0.0, 1.0)
    To, Vo = lattice.rotate(To, Vo, lattice.momentum_basis(Lx, Ly) @ Q)
    h, W = hamiltonian.spin_orbital(To, Vo, False)
    model = odmrg.Model(h, W, False, target)
    li = synth.random_left_isometries(N, False, target, D, l, 5)
    ri = synth.random_right_isometries(N, False, target, D, l + 2, 6)
    w = odmrg.window_from_mps(model, li, ri, l)
    g = lib.Dmrg(N, 8, d_max=D, precision=lib.SPLIT)
    Tg, Vg = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, Lx, Ly, 1.0, 0.0, 1.0)
    g.set_hamiltonian(Tg, Vg, lib.momentum_basis(Lx, Ly) @ Q)
    g.set_mps(li, ri)
    g.build_block_ops(l)
    return w, g


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_scratch_apply_matches_allocating_apply():
    w, g = _window()
    g.set_precision(lib.SPLIT)
    rng = np.random.default_rng(3)
    psi = torch.tensor(rng.standard_normal(w.size), device="cuda")
    ref = torch.empty_like(psi)
    g.heff_apply(psi, ref)          # allocating entry point (also builds the FP16 operator copies)
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    oracle = w.apply(psi.cpu().numpy())
    for _ in range(2):              # two calls in a row share the array
        out = torch.full_like(psi, float("nan"))
        g.heff_apply_static(psi, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert rel(o, ref_h) <= TOL_SPLIT
        assert rel(o, oracle) <= TOL_SPLIT
    g.close()


def _small_window():
    N, target, D, l = 9, (4,), 16, 3
    g = lib.Dmrg(N, 4, d_max=D, precision=lib.SPLIT)
    Tg, Vg = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, 3, 3, 1.0, 0.0, 2.0)
    g.set_hamiltonian(Tg, Vg, lib.momentum_basis(3, 3))
    g.set_mps(synth.random_left_isometries(N, False, target, D, l, 1),
              synth.random_right_isometries(N, False, target, D, l + 2, 2))
    g.build_block_ops(l)
    return g


def test_static_scratch_shared_by_two_contexts():
    """Two contexts with different windows take turns on the one array
    (serialised on one stream): each call rewrites the array's tables for its
    own window, and every sigma is bitwise the context's allocating result."""
    _, ga = _window()
    gb = _small_window()
    refs, psis = [], []
    for g in (ga, gb):
        n, _ = g.heff_layout()
        x = torch.tensor(np.random.default_rng(n).standard_normal(n), device="cuda")
        r = torch.empty_like(x)
        g.heff_apply(x, r)
        psis.append(x)
        refs.append(r)
    torch.cuda.synchronize()
    for _ in range(2):
        for g, x, r in ((ga, psis[0], refs[0]), (gb, psis[1], refs[1])):
            out = torch.full_like(x, float("nan"))
            g.heff_apply_static(x, out)
            torch.cuda.synchronize()
            assert torch.equal(out, r)
    ga.close()
    gb.close()


def test_static_scratch_rejects_a_window_over_its_size():
    """A window whose split scratch exceeds the fixed array (6x6 Hubbard,
    spin-adapted, D = 256 multiplets: tens of MB of stage-1 intermediate)
    is rejected with DMRG_ERR_ARG; the allocating path still serves it."""
    N, ne, D, l = 36, 36, 256, 17
    T, V = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 6, 6, 1.0, 0.0, 4.0)
    g = lib.Dmrg(N, ne, su2=True, d_max=D, precision=lib.SPLIT)
    g.set_hamiltonian(T, V, lib.momentum_basis(6, 6))
    g.set_mps(synth.random_left_isometries_su2(N, (ne, 0), D, l, 5),
              synth.random_right_isometries_su2(N, (ne, 0), D, l + 2, 6))
    g.build_block_ops(l)
    n, _ = g.heff_layout()
    x = torch.tensor(np.random.default_rng(0).standard_normal(n), device="cuda")
    y = torch.empty_like(x)
    g.heff_apply(x, y)
    with pytest.raises(lib.DmrgError) as ei:
        g.heff_apply_static(x, torch.empty_like(x))
    assert ei.value.code == lib.ERR_ARG
    assert "scratch" in str(ei.value)
    g.close()
