"""Continuous-admission serving of independent DMRG ground-state solves.

Requests (lattice, coupling, bond dimension, sweeps) arrive over time.  A
request is admitted as soon as a slot is free and its estimated device
footprint fits the HBM budget; admitted solves run concurrently, each with
its own library context (block operators and Davidson state stay on the
device) and its own CUDA stream, so their kernels overlap on the GPU.  The
library's C calls release the Python GIL, so one host thread per active solve
is enough to keep the device fed.  Results are deterministic per request: a
solve computes the same energy alone and in the mix.

This is the serving pattern of phase-diagram scans (many solves over a grid
of couplings) run on one B300.
"""
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import (FP64, MODEL_HUBBARD, MODEL_SPINLESS_TV, SPLIT, Dmrg,
               lattice_hamiltonian, momentum_basis)


@dataclass
class Request:
    rid: int
    model: str            # "spinless" or "hubbard"
    Lx: int
    Ly: int
    coupling: float       # V (spinless) or U (hubbard)
    D: int
    n_sweeps: int
    arrival: float        # seconds after the stream starts
    seed: int = 0
    filling: tuple = None  # (n_up, n_dn); default half filling / S_z = 0
    su2: bool = True       # hubbard: spin-adapted sectors, D counts multiplets


@dataclass
class Result:
    rid: int
    energy: float
    energies: list
    arrival: float
    start: float
    finish: float
    footprint: float
    profile: dict = field(default_factory=dict)

    @property
    def latency(self):
        return self.finish - self.arrival


def target_of(req):
    N = req.Lx * req.Ly
    if req.filling is not None:
        return req.filling
    if req.model == "hubbard":
        return (N // 2, N // 2)
    return (N // 2, 0)


def estimate_bytes(req):
    """Rough device footprint of one solve: operators of all stored blocks.

    Every block keeps O(M^2) operators (normal and complementary pairs) with
    about D^2 / n_sectors elements each; the window adds the enlarged blocks
    (d^2 larger) and the H_eff stacks.  Used only for admission.
    """
    N = req.Lx * req.Ly
    M = 2 * N if req.model == "hubbard" else N
    d = 4 if req.model == "hubbard" else 2
    nsec = max(4.0, (M / 4.0) ** (2 if req.model == "hubbard" else 1))
    per_op = 8.0 * req.D * req.D / nsec
    if req.model == "hubbard" and req.su2:
        # multiplet blocks: fewer sectors, and half the tensors of the
        # spin-orbital operator set
        per_op = 8.0 * req.D * req.D / max(4.0, M / 4.0) / 2.0
    blocks = N * 2.0 * M * M * per_op
    window = 6.0 * d * d * M * M * per_op
    # 2.3: measured device footprints (dmrg_memory_stats) of 4x4 and 6x6
    # solves at D = 128-256 stay below this bound (tests/test_serving.py)
    return 2.3 * (blocks + window) + 256e6


def run_one(req, precision, stream=None, davidson_tol=1e-7, rng_iso=None):
    """Solve one request synchronously; returns (energies, profile)."""
    spinful = req.model == "hubbard"
    N = req.Lx * req.Ly
    tgt = target_of(req)
    if spinful:
        T, V = lattice_hamiltonian(MODEL_HUBBARD, req.Lx, req.Ly, 1.0, 0.0, req.coupling)
    else:
        T, V = lattice_hamiltonian(MODEL_SPINLESS_TV, req.Lx, req.Ly, 1.0, 0.0, req.coupling)
    su2 = spinful and req.su2 and tgt[0] == tgt[1]
    if su2:
        g = Dmrg(N, tgt[0] + tgt[1], su2=True, d_max=req.D, precision=precision,
                 davidson_tol=davidson_tol, seed=req.seed)
    else:
        g = Dmrg(N, tgt[0], tgt[1] if spinful else 0, spinful=spinful, d_max=req.D,
                 precision=precision, davidson_tol=davidson_tol, seed=req.seed)
    # Concurrent solves launch directly: a CUDA-graph capture in one thread can
    # be invalidated by device-synchronising calls (allocation, stream
    # creation) made by the other solves' threads.
    g.set_graphs(False)
    try:
        g.set_hamiltonian(T, V, momentum_basis(req.Lx, req.Ly))
        g.random_start(req.seed)
        E = g.sweep(req.n_sweeps, stream=stream)
        prof = g.profile()
        prof["memory"] = g.memory_stats()
    finally:
        g.close()
    return E, prof


class Server:
    """Admits requests by slots and HBM footprint; runs them concurrently."""

    def __init__(self, precision=SPLIT, slots=4, hbm_budget=200e9, davidson_tol=1e-7):
        self.precision = precision
        self.slots = slots
        self.hbm_budget = hbm_budget
        self.davidson_tol = davidson_tol
        self.lock = threading.Condition()
        self.active = 0
        self.used = 0.0
        self.results = []
        self.errors = []

    def _fits(self, fp):
        return self.active < self.slots and (self.used + fp <= self.hbm_budget or self.active == 0)

    def _worker(self, req, fp, t0):
        import torch
        start = time.perf_counter() - t0
        try:
            stream = torch.cuda.Stream()
            E, prof = run_one(req, self.precision, stream, self.davidson_tol)
            res = Result(req.rid, float(E[-1]), E.tolist(), req.arrival, start,
                         time.perf_counter() - t0, fp, prof)
            with self.lock:
                self.results.append(res)
        except Exception as e:   # recorded, the stream goes on
            with self.lock:
                self.errors.append((req.rid, repr(e)))
        finally:
            with self.lock:
                self.active -= 1
                self.used -= fp
                self.lock.notify_all()

    def run(self, requests):
        """Serve a stream of requests (arrival times relative to now)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        threads = []
        for req in reqs:
            wait = req.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            fp = estimate_bytes(req)
            with self.lock:
                while not self._fits(fp):
                    self.lock.wait()
                self.active += 1
                self.used += fp
            th = threading.Thread(target=self._worker, args=(req, fp, t0), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        return self.summary(wall)

    def summary(self, wall):
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        return {"solves": len(self.results), "errors": len(self.errors), "wall_s": wall,
                "solves_per_s": len(self.results) / wall if wall > 0 else 0.0,
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "slots": self.slots, "error_messages": [m for _, m in self.errors[:3]]}


def poisson_stream(n, mean_interval, seed, mix, sweeps=2):
    """n requests with exponential inter-arrival times; mix = list of
    (model, Lx, Ly, (cmin, cmax), [D choices])."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(mean_interval)
        model, Lx, Ly, (c0, c1), Ds = mix[rng.integers(len(mix))]
        out.append(Request(i, model, Lx, Ly, float(rng.uniform(c0, c1)),
                           int(Ds[rng.integers(len(Ds))]), sweeps, t, seed=int(rng.integers(1 << 30))))
    return out
