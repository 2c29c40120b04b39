"""Observables of a converged state (the paper's Sec. II.B and its discussion of
Fig. 11): the one-particle reduced density matrix, its back-rotation to the
real-space basis, and expectation values of any operator written in the form
of Eq. 1, among them the charge-density-wave order parameter
    C_CDW = < (n_even - n_odd)^2 > / N^2,
n_even/odd the particle number on the two sublattices of the torus.

Every number is computed by the library: the 1-RDM by dmrg_rdm1 on the final
window of a sweep, an expectation value by building the block operators of
the operator itself (its t_ij, V_ijkl rotated into the run's mode basis like
the Hamiltonian) on the sweep's final MPS and applying them to the final
psi.  This module only sets up those calls.
"""
import numpy as np

from . import Dmrg


def back_rotate(gamma, U):
    """Real-space 1-RDM from the mode-basis one: with c_i = sum_m U[i, m] d_m,
    <c+_j c_i> = sum_mn U[i, m] U[j, n] <d+_n d_m>, i.e. U gamma U^T."""
    U = np.asarray(U, dtype=float)
    return U @ np.asarray(gamma, dtype=float) @ U.T


def sublattice_signs(Lx, Ly):
    """+1 on the even, -1 on the odd sublattice (site i = y * Lx + x)."""
    return np.array([1.0 if ((i % Lx) + (i // Lx)) % 2 == 0 else -1.0 for i in range(Lx * Ly)])


def cdw_operator(Lx, Ly):
    """(n_even - n_odd)^2 = sum_ij e_i e_j n_i n_j in Eq. 1 form (real space):
    n_i n_j = delta_ij n_i + c+_i c+_j c_j c_i, so t = identity and
    V[i, j, j, i] = e_i e_j.  The same (t, V) serves the spinful models with
    the spin-independent convention sum_ab V_ijkl c+_ia c+_jb c_kb c_la."""
    e = sublattice_signs(Lx, Ly)
    N = e.size
    T = np.eye(N)
    V = np.zeros((N, N, N, N))
    for i in range(N):
        for j in range(N):
            V[i, j, j, i] = e[i] * e[j]
    return T, V


def expectation(dmrg, T, V, U=None, stream=None):
    """<psi| O |psi> of an Eq. 1 operator O = (T, V) (real space, rotated by U
    like the Hamiltonian) in the final state of dmrg's last sweep."""
    right, l, psi = dmrg.get_mps()
    twin = Dmrg(**dmrg.kwargs)
    try:
        twin.set_hamiltonian(T, V, U)
        twin.set_mps(right=right)
        twin.build_block_ops(l, stream)
        return float(psi @ twin.heff_apply_host(psi, stream))
    finally:
        twin.close()


def cdw_order_parameter(dmrg, Lx, Ly, U=None, stream=None):
    """C_CDW = <(n_even - n_odd)^2> / N^2 of dmrg's final state."""
    T, V = cdw_operator(Lx, Ly)
    return expectation(dmrg, T, V, U, stream) / float(Lx * Ly) ** 2


def rdm1_final(dmrg, stream=None):
    """1-RDM (mode basis) of the final state of dmrg's last sweep (its window
    is the sweep's final window)."""
    import torch
    _, _, psi = dmrg.get_mps()
    x = torch.tensor(psi, dtype=torch.float64, device="cuda")
    return dmrg.rdm1(x, stream)
