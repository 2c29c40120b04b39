"""Error reporting through the C ABI, exercised without a fault.

* A bounded pipeline wait that gives up inside a stream-ordered H_eff*psi
  call must reach the caller: the context's next call (once the failed call's
  status has reached the host) or dmrg_sync returns DMRG_ERR_TIMEOUT, once.
  dmrg_selftest_timeout_report sets the error word exactly as such a wait does
  (the wait runs out on a barrier nothing completes; about one second).
* A sweep whose window solves hit the Davidson iteration limit says so.
* dmrg_get_mps / dmrg_get_center return the state a sweep ended with.
"""
import numpy as np
import pytest

import synth
from oracle import dmrg as odmrg
from oracle import hamiltonian, lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402


def _window(prec=lib.SPLIT, D=16, l=3):
    N, target = 9, (4,)
    Q = synth.haar_rotation(N, 2)
    To, Vo = lattice.spinless_tV(3, 3, 1.0, 0.0, 1.0)
    To, Vo = lattice.rotate(To, Vo, lattice.momentum_basis(3, 3) @ Q)
    h, W = hamiltonian.spin_orbital(To, Vo, False)
    model = odmrg.Model(h, W, False, target)
    li = synth.random_left_isometries(N, False, target, D, l, 5)
    ri = synth.random_right_isometries(N, False, target, D, l + 2, 6)
    w = odmrg.window_from_mps(model, li, ri, l)
    g = lib.Dmrg(N, 4, d_max=D, precision=prec)
    Tg, Vg = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, 3, 3, 1.0, 0.0, 1.0)
    g.set_hamiltonian(Tg, Vg, lib.momentum_basis(3, 3) @ Q)
    g.set_mps(li, ri)
    g.build_block_ops(l)
    return w, g


def test_timeout_reported_once_by_next_apply():
    w, g = _window()
    psi = torch.tensor(np.random.default_rng(1).standard_normal(w.size), device="cuda")
    ref = torch.empty_like(psi)
    g.heff_apply(psi, ref)
    g.sync()
    g.selftest_timeout_report(0)
    torch.cuda.synchronize()            # the status copy has landed
    out = torch.empty_like(psi)
    with pytest.raises(lib.DmrgError) as ei:
        g.heff_apply(psi, out)
    assert ei.value.code == lib.ERR_TIMEOUT
    g.heff_apply(psi, out)              # reported once; the context stays usable
    g.sync()
    assert torch.equal(out, ref)
    g.close()


def test_timeout_reported_by_sync():
    w, g = _window()
    psi = torch.tensor(np.random.default_rng(2).standard_normal(w.size), device="cuda")
    out = torch.empty_like(psi)
    g.heff_apply(psi, out)
    g.selftest_timeout_report(0)
    with pytest.raises(lib.DmrgError) as ei:
        g.sync()
    assert ei.value.code == lib.ERR_TIMEOUT
    g.sync()
    g.close()


def test_static_path_timeout_reported_and_cleared():
    w, g = _window()
    psi = torch.tensor(np.random.default_rng(3).standard_normal(w.size), device="cuda")
    ref = torch.empty_like(psi)
    g.heff_apply(psi, ref)
    out = torch.empty_like(psi)
    g.heff_apply_static(psi, out)
    g.sync()
    g.selftest_timeout_report(1)
    torch.cuda.synchronize()
    with pytest.raises(lib.DmrgError) as ei:
        g.heff_apply_static(psi, out)
    assert ei.value.code == lib.ERR_TIMEOUT
    g.heff_apply_static(psi, out)       # the word was cleared when read
    g.sync()
    assert torch.equal(out, ref)
    g.close()


def test_sweep_reports_unconverged_windows():
    T, V = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, 3, 3, 1.0, 0.0, 1.0)
    g = lib.Dmrg(9, 4, d_max=16, davidson_tol=1e-12, davidson_max_iter=2)
    g.set_hamiltonian(T, V, lib.momentum_basis(3, 3))
    g.set_mps(right=synth.random_right_isometries(9, False, (4,), 16, 1, 0))
    E = g.sweep(1)
    assert not g.sweep_converged
    assert np.all(np.isfinite(E))
    g.close()


@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_get_mps_returns_the_final_state(prec):
    """After two sweeps the returned right isometries and center psi rebuild
    the final state: in a fresh context its energy <psi|H_eff|psi> at window
    0 is the sweep energy."""
    T, V = lib.lattice_hamiltonian(lib.MODEL_SPINLESS_TV, 3, 3, 1.0, 0.0, 1.0)
    U = lib.momentum_basis(3, 3)
    g = lib.Dmrg(9, 4, d_max=12, davidson_tol=1e-10, precision=prec)
    g.set_hamiltonian(T, V, U)
    g.set_mps(right=synth.random_right_isometries(9, False, (4,), 12, 1, 0))
    E = g.sweep(2)
    right, l, psi = g.get_mps()
    assert l == 0 and abs(np.linalg.norm(psi) - 1) < 1e-12
    for n, iso in right.items():
        for m in iso.values():
            assert np.abs(m.T @ m - np.eye(m.shape[1])).max() < 1e-12
    h = lib.Dmrg(9, 4, d_max=12)
    h.set_hamiltonian(T, V, U)
    h.set_mps(right=right)
    h.build_block_ops(0)
    n, _ = h.heff_layout()
    assert n == psi.size
    e = float(psi @ h.heff_apply_host(psi))
    assert abs(e - E[-1]) <= 1e-10 * abs(E[-1]), (e, E)
    g.close()
    h.close()
