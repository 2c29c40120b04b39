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
    declared = set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dmrg_\w+)\s*\(", src, re.M))
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
