"""Failure detection of the tcgen05 kernels, made without a fault.

Every pipeline wait in the H_eff*psi kernels is bounded: after about one
second it records an error code, raises the CTA's abort flag and returns, and
the host reports DMRG_ERR_TIMEOUT.  The self-test runs the same wait on a
shared-memory barrier that nothing completes (a flag nothing sets) and
checks the status; the context must stay usable afterwards.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2311_14106_b300 as lib  # noqa: E402


def test_bounded_wait_gives_up_and_reports():
    t0 = time.perf_counter()
    rc = lib.selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert rc == lib.ERR_TIMEOUT, rc
    assert 0.2 < dt < 10.0, dt
    # the device is still usable
    x = torch.arange(1000, dtype=torch.float64, device="cuda")
    assert float(x.sum()) == 499500.0
    assert np.isfinite(dt)
