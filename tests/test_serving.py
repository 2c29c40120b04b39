"""Serving loop: admission by slots and HBM footprint (host logic, CPU) and,
on the GPU, that each solve gives the same energy alone and in the mix."""
import threading
import time

import numpy as np
import pytest

import paper_2311_14106_b300 as lib
from paper_2311_14106_b300 import serving


def test_admission_respects_slots_and_budget(monkeypatch):
    state = {"active": 0, "peak": 0, "bytes": 0.0, "peak_bytes": 0.0}
    lk = threading.Lock()

    def fake_run(req, precision, stream=None, davidson_tol=1e-7):
        fp = serving.estimate_bytes(req)
        with lk:
            state["active"] += 1
            state["bytes"] += fp
            state["peak"] = max(state["peak"], state["active"])
            state["peak_bytes"] = max(state["peak_bytes"], state["bytes"])
        time.sleep(0.02 + 0.01 * (req.rid % 3))
        with lk:
            state["active"] -= 1
            state["bytes"] -= fp
        return np.array([-1.0 - req.rid]), {}

    monkeypatch.setattr(serving, "run_one", fake_run)

    class FakeStream:
        pass

    import sys
    import types
    fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Stream=FakeStream))
    monkeypatch.setitem(sys.modules, "torch", fake_torch)
    mix = [("spinless", 4, 4, (0.0, 4.0), [64, 128]), ("hubbard", 4, 4, (0.0, 8.0), [64])]
    reqs = serving.poisson_stream(24, 0.005, 3, mix)
    budget = 2.5 * max(serving.estimate_bytes(r) for r in reqs)
    srv = serving.Server(slots=3, hbm_budget=budget)
    out = srv.run(reqs)
    assert out["solves"] == 24 and out["errors"] == 0
    assert state["peak"] <= 3
    assert state["peak_bytes"] <= budget
    assert out["p99_latency_s"] >= out["p50_latency_s"] > 0
    assert sorted(r.rid for r in srv.results) == list(range(24))


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [lib.FP64, lib.SPLIT])
def test_same_result_alone_and_in_the_mix(prec):
    pytest.importorskip("torch")
    mix = [("spinless", 3, 3, (0.5, 2.0), [16, 24]), ("hubbard", 3, 3, (2.0, 6.0), [16])]
    reqs = serving.poisson_stream(6, 0.02, 11, mix, sweeps=2)
    for r in reqs:
        if r.model == "hubbard":
            # S_z = 1/2 runs in U(1)xU(1) sectors, S = 0 spin-adapted
            r.filling = (5, 4) if r.rid % 2 else (4, 4)
    assert {r.filling for r in reqs if r.model == "hubbard"} == {(5, 4), (4, 4)}
    srv = serving.Server(precision=prec, slots=3, hbm_budget=50e9, davidson_tol=1e-9)
    out = srv.run(reqs)
    assert out["solves"] == len(reqs) and out["errors"] == 0, srv.errors
    mixed = {r.rid: r.energy for r in srv.results}
    for r in reqs:
        E, _ = serving.run_one(r, prec, None, 1e-9)
        assert abs(E[-1] - mixed[r.rid]) <= 1e-9 * abs(E[-1]), (r, E[-1], mixed[r.rid])


@pytest.mark.gpu
@pytest.mark.parametrize("model,L,D", [("spinless", 4, 128), ("hubbard", 4, 128),
                                        ("spinless", 6, 64), ("hubbard", 6, 64)])
def test_footprint_estimate_bounds_the_measured_footprint(model, L, D):
    """Admission uses serving.estimate_bytes: it must not undercount what a
    solve holds on the device (the most memory in use at any window build of
    the solve, dmrg_memory_stats, above what was in use before it)."""
    torch = pytest.importorskip("torch")
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    req = serving.Request(0, model, L, L, 4.0 if model == "hubbard" else 2.0, D, 1, 0.0, seed=5)
    E, prof = serving.run_one(req, lib.SPLIT, torch.cuda.Stream())
    used = prof["memory"]["device_in_use"] - (total - free0)
    assert used > 0
    assert serving.estimate_bytes(req) >= used, (serving.estimate_bytes(req), used)
