"""C-ABI checks that need no GPU: the library loads, exports every function
the header declares, and its host-side lattice / momentum-basis helpers (a1,
a2) agree with the oracle's independent implementation."""
import os
import re

import numpy as np
import pytest

import paper_2311_14106_b300 as lib
from oracle import lattice

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "dmrg_b300.h")


def test_header_symbols_exported():
    src = open(HEADER).read()
    declared = set(re.findall(r"^\s*(?:\w+\s+)+\**\s*(dmrg_\w+)\s*\(", src, re.M))
    assert declared, "no declarations parsed"
    assert declared == set(lib.HEADER_FUNCTIONS)
    for name in declared:
        assert hasattr(lib._lib, name), name


@pytest.mark.parametrize("model", ["spinless", "hubbard"])
def test_lattice_matches_oracle(model):
    if model == "spinless":
        T, V = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, 4, 4, 1.0, 0.4, 0.8)
        To, Vo = lattice.spinless_tV(4, 4, 1.0, 0.4, 0.8)
    else:
        T, V = lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 3, 4, 1.0, 0.0, 4.0)
        To, Vo = lattice.hubbard(3, 4, 1.0, 4.0)
    assert np.array_equal(T, To)
    assert np.array_equal(V, Vo)


@pytest.mark.parametrize("L", [(3, 3), (4, 4), (6, 6), (4, 6)])
def test_momentum_basis_matches_oracle(L):
    U = lib.momentum_basis(*L)
    Uo = lattice.momentum_basis(*L)
    assert np.abs(U - Uo).max() < 1e-13


def test_bad_arguments_rejected():
    with pytest.raises(lib.DmrgError):
        lib.lattice_hamiltonian(lib.MODEL_HUBBARD, 2, 4)
    assert lib._lib.dmrg_create(None, None) == lib.ERR_ARG
    assert lib._lib.dmrg_destroy(None) == lib.OK
    assert lib._lib.dmrg_error_string(lib.ERR_TIMEOUT).decode().startswith("bounded")


def test_staging_policy_matches_sweep_walk():
    """The staging policy's next-use distances against a walk of the sweep:
    window l uses L_l and R_{l+2}; truncation after window l builds L_{l+1}
    (left to right) or R_{l+1} (right to left), which makes the old block of
    that name stale."""
    N = 7
    order = [(0, l) for l in range(N - 1)] + [(1, l) for l in range(N - 2, -1, -1)]
    order = order * 3
    for start, (pass_, l) in enumerate(order[:len(order) // 3]):
        for left in (1, 0):
            for n in range(0, N + 1):
                # walk forward: first event on this block name
                want = -1
                for k, (p2, l2) in enumerate(order[start:]):
                    uses = (l2 == n) if left else (l2 + 2 == n)
                    if uses:
                        want = k
                        break
                    # after window l2 the truncation rebuilds one block
                    rebuilt = (left and p2 == 0 and l2 < N - 2 and l2 + 1 == n) or \
                              (not left and p2 == 1 and l2 > 0 and l2 + 1 == n)
                    if rebuilt:
                        break
                if (left and n > N - 2) or (not left and (n < 2 or n > N)):
                    continue
                got = lib._lib.dmrg_sweep_next_use(N, pass_, l, left, n)
                assert got == want, (pass_, l, left, n, got, want)
    assert lib._lib.dmrg_sweep_next_use(1, 0, 0, 1, 0) == -2


def test_fp64_gemm_tile_choice():
    """The grouped FP64 GEMM's tile plan (pure host function): tiny operator
    blocks that share an operand are folded into one tall or wide problem,
    large blocks keep square tiles, square_only never folds, and the choice
    never issues much more work than any candidate shape."""
    import math
    shapes = [(16, 16), (32, 32), (64, 64), (64, 16), (16, 64)]

    def issued(M, N, b, tm, tn, fold):
        Mt, Nt = (b * M if fold == 1 else M), (b * N if fold == 2 else N)
        return math.ceil(Mt / tm) * math.ceil(Nt / tn) * (1 if fold else b) * tm * tn

    assert lib.gemm_tile_choice(10, 5, 4000, fold_rows_ok=True) == (64, 16, 1)
    assert lib.gemm_tile_choice(5, 10, 4000, fold_cols_ok=True) == (16, 64, 2)
    tm, tn, f = lib.gemm_tile_choice(10, 5, 4000, True, True, square_only=True)
    assert f == 0 and tm == tn
    assert lib.gemm_tile_choice(500, 500, 1)[2] == 0
    for M, N, b, f1, f2 in [(3, 7, 50, True, False), (130, 129, 1, False, False),
                            (64, 8, 200, False, True), (17, 200, 9, True, True)]:
        tm, tn, f = lib.gemm_tile_choice(M, N, b, f1, f2)
        assert (tm, tn) in shapes and (f != 1 or f1) and (f != 2 or f2)
        mine = issued(M, N, b, tm, tn, f)
        for (a, c) in shapes:
            for g in [0] + ([1] if f1 else []) + ([2] if f2 else []):
                assert mine <= 1.5 * issued(M, N, b, a, c, g)
    with pytest.raises(lib.DmrgError):
        lib.gemm_tile_choice(0, 4, 1)
