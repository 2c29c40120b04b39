"""Full-size check of the split path in the configuration bench.py times.

At the 6x6 Hubbard, D = 1024 window the FP64 oracle cannot build the block
operators in reasonable time, so the reference here is the library's own
FP64 path (pinned to the oracle at <= 1e-12 on the smaller windows of
test_gpu_heff.py).  The window has sigma blocks wider than 128 (two MMA
tiles per block), long split-K ranges and all packing classes of stage 2,
which the small windows do not all reach.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402

TOL_SPLIT = 2e-5


def build(D):
    N, nu, nd, U = 36, 18, 18, 4.0
    T, V = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 6, 6, 1.0, 0.0, U)
    g = lib.Dmrg(N, nu, nd, spinful=True, d_max=D, davidson_tol=1e-6)
    g.set_hamiltonian(T, V, lib.momentum_basis(6, 6))
    l = N // 2 - 1
    g.set_mps(synth.random_left_isometries(N, True, (nu, nd), D, l, 5),
              synth.random_right_isometries(N, True, (nu, nd), D, l + 2, 6))
    g.build_block_ops(l)
    return g


@pytest.mark.parametrize("D", [1024])
def test_split_path_vs_fp64_full_size(D):
    g = build(D)
    n, layout = g.heff_layout()
    assert max(max(da, db) for _, _, da, db in layout) > 128
    psi = synth.random_psi(layout, 1)
    g.set_precision(lib.FP64)
    ref = g.heff_apply_host(psi)
    g.set_precision(lib.SPLIT)
    s = g.heff_apply_host(psi)      # raises if a kernel recorded an error
    err = np.linalg.norm(s - ref) / np.linalg.norm(ref)
    assert err <= TOL_SPLIT, err
    # the sampled elements of the largest block agree elementwise too
    big = max(range(len(layout)), key=lambda i: layout[i][2] * layout[i][3])
    off = sum(da * db for _, _, da, db in layout[:big])
    blk = slice(off, off + layout[big][2] * layout[big][3])
    scale = np.abs(ref).max()
    assert np.abs(s[blk] - ref[blk]).max() <= 1e-4 * scale
    g.close()
