"""FP64 CPU oracle for two-site ab initio DMRG (arXiv 2311.14106).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: it exists so that tests, the smoke check and
the CPU-baseline leg of the benchmark can compare the CUDA path against a
plain, slow, obviously checkable restatement of the method.  It shares no
code, tables or constants with the CUDA path.

Modules
  lattice      Eq. 2 / Eq. 3 lattice Hamiltonians on a torus, momentum basis,
               one-particle mode rotation (Sec. II.B).
  hamiltonian  spin-orbital form of Eq. 1 (antisymmetrised two-body tensor).
  ed           exact diagonalisation in a fixed particle-number sector.
  blocks       block-sparse operators over quantum-number sectors.
  dmrg         two-site DMRG with normal / complementary block operators:
               enlarged blocks, H_eff * psi, Davidson, truncation, sweeps.
  dense        explicit W^T H W projection of the Fock-space Hamiltonian.
  su2          spin-adapted (U(1)xSU(2)) windows: exact Clebsch-Gordan
               expansion of multiplet bases onto the S_z basis, sigma =
               E^T H_eff E psi through the U(1)xU(1) window.

Every function is pinned by tests against something other than itself
(closed forms, brute force, invariants); see tests/test_oracle.py.
"""
