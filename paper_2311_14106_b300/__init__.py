"""Python binding of libdmrgb300 (B300 two-site DMRG hot path, arXiv 2311.14106).

Argument marshalling only: every step runs in the CUDA library through its
C ABI (include/dmrg_b300.h).  PyTorch tensors are accepted for device
buffers (psi, sigma) and streams.  There is no CPU fallback: if the shared
library is missing or cannot be loaded, importing this module fails.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdmrgb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} not built; run paper_2311_14106_b300/build.py")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_TIMEOUT, ERR_NOT_CONVERGED = 0, -1, -2, -3, -4, -5, -6
U1, U1U1, U1SU2 = 1, 2, 3
FP64, SPLIT = 0, 1
MODEL_SPINLESS_TV, MODEL_HUBBARD = 1, 2

HEADER_FUNCTIONS = [
    "dmrg_error_string", "dmrg_last_error", "dmrg_create", "dmrg_destroy",
    "dmrg_lattice_hamiltonian", "dmrg_momentum_basis", "dmrg_set_hamiltonian",
    "dmrg_set_isometry", "dmrg_build_block_ops", "dmrg_heff_layout",
    "dmrg_set_precision", "dmrg_heff_apply", "dmrg_heff_apply_host",
    "dmrg_heff_flops", "dmrg_davidson", "dmrg_truncate", "dmrg_sweep",
    "dmrg_heff_stage_info", "dmrg_heff_timing", "dmrg_profile",
    "dmrg_heff_apply_split_static", "dmrg_heff_tuning", "dmrg_set_graphs",
    "dmrg_heff_split_plan", "dmrg_heff_entries", "dmrg_selftest_bounded_wait",
    "dmrg_sync", "dmrg_get_mps", "dmrg_get_center", "dmrg_heff_split_paths",
    "dmrg_selftest_timeout_report", "dmrg_staging_stats", "dmrg_sweep_next_use",
    "dmrg_rdm1", "dmrg_heff_apply_batch", "dmrg_random_start", "dmrg_heff_fp64_state",
    "dmrg_memory_stats", "dmrg_set_refinement", "dmrg_set_split_min_flops",
    "dmrg_gemm_tile_choice",
]


class Config(ctypes.Structure):
    _fields_ = [
        ("sym", ctypes.c_int), ("n_sites", ctypes.c_int), ("n_up", ctypes.c_int),
        ("n_dn", ctypes.c_int), ("d_max", ctypes.c_int), ("precision", ctypes.c_int),
        ("davidson_tol", ctypes.c_double), ("davidson_max_sub", ctypes.c_int),
        ("davidson_max_iter", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t),
        ("seed", ctypes.c_uint64), ("twice_s", ctypes.c_int),
    ]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_sig = {
    "dmrg_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dmrg_last_error": (ctypes.c_char_p, [_P]),
    "dmrg_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Config)]),
    "dmrg_destroy": (ctypes.c_int, [_P]),
    "dmrg_lattice_hamiltonian": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, _D, _D]),
    "dmrg_momentum_basis": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _D]),
    "dmrg_set_hamiltonian": (ctypes.c_int, [_P, _D, _D, _D]),
    "dmrg_set_isometry": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         _I, _I, _I, _D]),
    "dmrg_build_block_ops": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "dmrg_heff_layout": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong), _I, _I]),
    "dmrg_set_precision": (ctypes.c_int, [_P, ctypes.c_int]),
    "dmrg_heff_apply": (ctypes.c_int, [_P, _P, _P, _P]),
    "dmrg_heff_apply_host": (ctypes.c_int, [_P, _D, _D, _P]),
    "dmrg_heff_apply_split_static": (ctypes.c_int, [_P, _P, _P, _P]),
    "dmrg_heff_flops": (ctypes.c_int, [_P, _D]),
    "dmrg_davidson": (ctypes.c_int, [_P, _P, _D, _I, _P]),
    "dmrg_truncate": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _D, _D, _P]),
    "dmrg_sweep": (ctypes.c_int, [_P, ctypes.c_int, _I, _D, _P]),
    "dmrg_heff_stage_info": (ctypes.c_int, [_P, _D]),
    "dmrg_heff_timing": (ctypes.c_int, [_P, ctypes.c_int, _D]),
    "dmrg_profile": (ctypes.c_int, [_P, _D]),
    "dmrg_heff_tuning": (ctypes.c_int, [_P, _D, ctypes.c_int, _I]),
    "dmrg_set_graphs": (ctypes.c_int, [_P, ctypes.c_int]),
    "dmrg_heff_split_plan": (ctypes.c_int, [_P, _D]),
    "dmrg_heff_entries": (ctypes.c_int, [_P, _I, ctypes.c_int, _I]),
    "dmrg_selftest_bounded_wait": (ctypes.c_int, [_P]),
    "dmrg_sync": (ctypes.c_int, [_P, _P]),
    "dmrg_get_mps": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _I,
                                    ctypes.POINTER(ctypes.c_longlong), _I, _I, _I, _D]),
    "dmrg_get_center": (ctypes.c_int, [_P, _I, ctypes.POINTER(ctypes.c_longlong), _D]),
    "dmrg_heff_split_paths": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "dmrg_selftest_timeout_report": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "dmrg_staging_stats": (ctypes.c_int, [_P, _D]),
    "dmrg_sweep_next_use": (ctypes.c_longlong, [ctypes.c_int] * 5),
    "dmrg_rdm1": (ctypes.c_int, [_P, _P, _D, _P]),
    "dmrg_heff_apply_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "dmrg_random_start": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "dmrg_heff_fp64_state": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "dmrg_memory_stats": (ctypes.c_int, [_P, _D]),
    "dmrg_set_refinement": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "dmrg_set_split_min_flops": (ctypes.c_int, [_P, ctypes.c_double]),
    "dmrg_gemm_tile_choice": (ctypes.c_int, [ctypes.c_int] * 6 + [_I]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class DmrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_lib.dmrg_error_string(code).decode()} ({code}): {msg}")
        self.code = code


def _dptr(a):
    return a.ctypes.data_as(_D)


def _iptr(a):
    return a.ctypes.data_as(_I)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _tensor_ptr(t):
    if hasattr(t, "data_ptr"):
        if t.dtype.__repr__() != "torch.float64" or not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous float64 CUDA tensor")
        return t.data_ptr()
    return int(t)


def selftest_bounded_wait(stream=None):
    """Status of the bounded-wait self-test (ERR_TIMEOUT is the expected,
    passing result: the device wait gave up after about a second)."""
    return _lib.dmrg_selftest_bounded_wait(_stream_ptr(stream))


def lattice_hamiltonian(model, Lx, Ly, t=1.0, tp=0.0, v=1.0):
    """a1: Eq. 2 / Eq. 3 on an Lx x Ly torus -> (T[N,N], V[N,N,N,N])."""
    N = Lx * Ly
    T = np.zeros((N, N))
    V = np.zeros((N, N, N, N))
    rc = _lib.dmrg_lattice_hamiltonian(model, Lx, Ly, t, tp, v, _dptr(T), _dptr(V))
    if rc != OK:
        raise DmrgError(rc, "lattice_hamiltonian")
    return T, V


def momentum_basis(Lx, Ly):
    """a2 helper: real standing-wave momentum modes, U[site, mode]."""
    U = np.zeros((Lx * Ly, Lx * Ly))
    rc = _lib.dmrg_momentum_basis(Lx, Ly, _dptr(U))
    if rc != OK:
        raise DmrgError(rc, "momentum_basis")
    return U


def gemm_tile_choice(M, N, batch, fold_rows_ok=False, fold_cols_ok=False, square_only=False):
    """(tile rows, tile columns, fold) of the grouped FP64 GEMM (see the header)."""
    out = np.zeros(3, dtype=np.int32)
    rc = _lib.dmrg_gemm_tile_choice(M, N, batch, int(fold_rows_ok), int(fold_cols_ok),
                                    int(square_only), _iptr(out))
    if rc != OK:
        raise DmrgError(rc, "gemm_tile_choice")
    return tuple(int(x) for x in out)


class Dmrg:
    """One library context (one problem: Hamiltonian, MPS basis, window)."""

    def __init__(self, n_sites, n_up, n_dn=0, spinful=False, d_max=128, precision=FP64,
                 davidson_tol=1e-8, davidson_max_sub=20, davidson_max_iter=200, seed=0,
                 su2=False, twice_s=0, hbm_budget_bytes=0):
        """su2=True: spin-adapted (U(1)xSU(2)) sectors (N, 2J); n_up is then
        the total particle number and D counts multiplets."""
        sym = U1SU2 if su2 else (U1U1 if spinful else U1)
        cfg = Config(sym, n_sites, n_up, n_dn, d_max, precision,
                     davidson_tol, davidson_max_sub, davidson_max_iter, hbm_budget_bytes, seed,
                     twice_s)
        spinful = spinful or su2
        h = _P()
        rc = _lib.dmrg_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != OK:
            raise DmrgError(rc, "dmrg_create")
        self._h = h
        self.kwargs = dict(n_sites=n_sites, n_up=n_up, n_dn=n_dn, spinful=spinful, d_max=d_max,
                           su2=su2, twice_s=twice_s)
        self.spinful = spinful
        self.nq = 2 if spinful else 1
        self.n_sites = n_sites

    def close(self):
        if getattr(self, "_h", None):
            _lib.dmrg_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, rc, what):
        if rc != OK:
            raise DmrgError(rc, f"{what}: {_lib.dmrg_last_error(self._h).decode()}")
        return rc

    def set_hamiltonian(self, T, V, U=None):
        T = np.ascontiguousarray(T, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        Up = None if U is None else _dptr(np.ascontiguousarray(U, dtype=np.float64))
        self._check(_lib.dmrg_set_hamiltonian(self._h, _dptr(T), _dptr(V), Up), "set_hamiltonian")

    def set_isometry(self, side, site, iso):
        """iso: {qn tuple: (rows, cols) ndarray}; side 0 left, 1 right."""
        qs = sorted(iso)
        qn = np.array([x for q in qs for x in q[: self.nq]], dtype=np.int32)
        rows = np.array([iso[q].shape[0] for q in qs], dtype=np.int32)
        cols = np.array([iso[q].shape[1] for q in qs], dtype=np.int32)
        data = np.concatenate([np.ascontiguousarray(iso[q], dtype=np.float64).ravel() for q in qs])
        self._check(_lib.dmrg_set_isometry(self._h, side, site, len(qs), _iptr(qn), _iptr(rows),
                                           _iptr(cols), _dptr(data)), "set_isometry")

    def set_mps(self, left=None, right=None):
        for n, iso in (left or {}).items():
            self.set_isometry(0, n, iso)
        for n, iso in (right or {}).items():
            self.set_isometry(1, n, iso)

    def random_start(self, seed):
        """A seeded random right-canonical MPS basis made by the library."""
        self._check(_lib.dmrg_random_start(self._h, seed), "random_start")

    def build_block_ops(self, l, stream=None):
        self._check(_lib.dmrg_build_block_ops(self._h, l, _stream_ptr(stream)), "build_block_ops")

    def heff_layout(self):
        n = ctypes.c_longlong()
        nb = ctypes.c_int()
        self._check(_lib.dmrg_heff_layout(self._h, ctypes.byref(n), ctypes.byref(nb), None),
                    "heff_layout")
        blocks = np.zeros((nb.value, 2 * self.nq + 2), dtype=np.int32)
        self._check(_lib.dmrg_heff_layout(self._h, None, None, _iptr(blocks)), "heff_layout")
        out = []
        for b in blocks:
            qa = tuple(int(x) for x in b[: self.nq])
            qb = tuple(int(x) for x in b[self.nq: 2 * self.nq])
            out.append((qa, qb, int(b[-2]), int(b[-1])))
        return n.value, out

    def set_refinement(self, inner_steps, min_window_flops):
        """Split-precision correction steps of the FP64 refinement (see the header)."""
        self._check(_lib.dmrg_set_refinement(self._h, inner_steps, min_window_flops),
                    "set_refinement")

    def set_split_min_flops(self, min_window_flops):
        """Windows below this many flops per product solve in FP64 (see the header)."""
        self._check(_lib.dmrg_set_split_min_flops(self._h, min_window_flops),
                    "set_split_min_flops")

    def set_precision(self, p):
        self._check(_lib.dmrg_set_precision(self._h, p), "set_precision")

    def heff_apply(self, psi, sigma, stream=None):
        """a5: sigma = H_eff psi on device buffers (torch float64 CUDA tensors)."""
        self._check(_lib.dmrg_heff_apply(self._h, _tensor_ptr(psi), _tensor_ptr(sigma),
                                         _stream_ptr(stream)), "heff_apply")

    def heff_apply_batch(self, psi, sigma, stream=None):
        """sigma[v] = H_eff psi[v] for the rows of a contiguous (nv, psi_len)
        float64 CUDA tensor, in one batched pass on the split path."""
        nv = psi.shape[0] if psi.dim() == 2 else 1
        self._check(_lib.dmrg_heff_apply_batch(self._h, nv, _tensor_ptr(psi), _tensor_ptr(sigma),
                                               _stream_ptr(stream)), "heff_apply_batch")

    def heff_apply_static(self, psi, sigma, stream=None):
        """Split-precision H_eff psi that allocates no device memory: its
        scratch is the library's fixed 64 MiB device array (see the header)."""
        self._check(_lib.dmrg_heff_apply_split_static(self._h, _tensor_ptr(psi), _tensor_ptr(sigma),
                                                     _stream_ptr(stream)), "heff_apply_split_static")

    def heff_apply_host(self, psi, stream=None):
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.zeros_like(psi)
        self._check(_lib.dmrg_heff_apply_host(self._h, _dptr(psi), _dptr(out),
                                              _stream_ptr(stream)), "heff_apply_host")
        return out

    def heff_flops(self):
        f = ctypes.c_double()
        self._check(_lib.dmrg_heff_flops(self._h, ctypes.byref(f)), "heff_flops")
        return f.value

    def davidson(self, psi, stream=None):
        """a6: lowest eigenpair; psi (device tensor) is start vector and result."""
        e = ctypes.c_double()
        it = ctypes.c_int()
        rc = _lib.dmrg_davidson(self._h, _tensor_ptr(psi), ctypes.byref(e), ctypes.byref(it),
                                _stream_ptr(stream))
        if rc not in (OK, ERR_NOT_CONVERGED):
            self._check(rc, "davidson")
        return e.value, it.value, rc == OK

    def truncate(self, psi, side, d_max, stream=None):
        disc = ctypes.c_double()
        ent = ctypes.c_double()
        self._check(_lib.dmrg_truncate(self._h, _tensor_ptr(psi), side, d_max, ctypes.byref(disc),
                                       ctypes.byref(ent), _stream_ptr(stream)), "truncate")
        return disc.value, ent.value

    def sweep(self, n_sweeps, d_schedule=None, stream=None):
        """a6-a8: two-site sweeps; returns the per-sweep energies.  A window
        whose Davidson hit its iteration limit does not raise: the energies
        are returned and self.sweep_converged is False."""
        E = np.zeros(n_sweeps)
        ds = None
        if d_schedule is not None:
            ds = np.ascontiguousarray(d_schedule, dtype=np.int32)
        rc = _lib.dmrg_sweep(self._h, n_sweeps, None if ds is None else _iptr(ds), _dptr(E),
                             _stream_ptr(stream))
        self.sweep_converged = rc == OK
        if rc not in (OK, ERR_NOT_CONVERGED):
            self._check(rc, "sweep")
        return E

    def sync(self, stream=None):
        """Synchronise the stream; raises DmrgError (ERR_TIMEOUT) if a bounded
        device wait of an earlier H_eff*psi gave up."""
        self._check(_lib.dmrg_sync(self._h, _stream_ptr(stream)), "sync")

    def get_isometry(self, side, site):
        """One isometry of the current MPS basis: {qn tuple: (rows, cols) ndarray}."""
        ns = ctypes.c_int()
        ne = ctypes.c_longlong()
        self._check(_lib.dmrg_get_mps(self._h, side, site, ctypes.byref(ns), ctypes.byref(ne),
                                      None, None, None, None), "get_mps")
        qn = np.zeros(max(ns.value, 1) * self.nq, dtype=np.int32)
        rows = np.zeros(max(ns.value, 1), dtype=np.int32)
        cols = np.zeros(max(ns.value, 1), dtype=np.int32)
        data = np.zeros(max(ne.value, 1))
        self._check(_lib.dmrg_get_mps(self._h, side, site, ctypes.byref(ns), ctypes.byref(ne),
                                      _iptr(qn), _iptr(rows), _iptr(cols), _dptr(data)), "get_mps")
        out, off = {}, 0
        for k in range(ns.value):
            q = tuple(int(x) for x in qn[k * self.nq:(k + 1) * self.nq])
            r, c = int(rows[k]), int(cols[k])
            out[q] = data[off:off + r * c].reshape(r, c).copy()
            off += r * c
        return out

    def get_mps(self):
        """The MPS after dmrg_sweep: (right isometries {n: iso} for n = 2..N-1,
        window l of the center, center psi as a host array)."""
        l = ctypes.c_int()
        n = ctypes.c_longlong()
        self._check(_lib.dmrg_get_center(self._h, ctypes.byref(l), ctypes.byref(n), None),
                    "get_center")
        psi = np.zeros(max(n.value, 1))
        self._check(_lib.dmrg_get_center(self._h, ctypes.byref(l), ctypes.byref(n), _dptr(psi)),
                    "get_center")
        right = {k: self.get_isometry(1, k) for k in range(l.value + 2, self.n_sites)}
        return right, l.value, psi[:n.value]

    def selftest_timeout_report(self, which, stream=None):
        """Set this context's error word (0 window, 1 static path) the way a
        pipeline wait that gave up does (about one second, no fault)."""
        self._check(_lib.dmrg_selftest_timeout_report(self._h, which, _stream_ptr(stream)),
                    "selftest_timeout_report")

    def rdm1(self, psi, stream=None):
        """One-particle reduced density matrix of psi (device tensor, this
        window's layout): gamma[i, j] = sum_s <c+_{j s} c_{i s}>, rotated
        mode basis."""
        g = np.zeros((self.n_sites, self.n_sites))
        self._check(_lib.dmrg_rdm1(self._h, _tensor_ptr(psi), _dptr(g), _stream_ptr(stream)),
                    "rdm1")
        return g

    def staging_stats(self):
        """Block-operator staging under hbm_budget_bytes (see the header)."""
        out = np.zeros(8)
        self._check(_lib.dmrg_staging_stats(self._h, _dptr(out)), "staging_stats")
        keys = ["h2d_bytes", "h2d_seconds", "d2h_bytes", "peak_resident_bytes", "offloads",
                "reloads", "releases", "budget"]
        return dict(zip(keys, out.tolist()))

    def heff_fp64_state(self):
        """Physical memory of the window's FP64 path (see dmrg_heff_fp64_state)."""
        out = (ctypes.c_longlong * 4)()
        self._check(_lib.dmrg_heff_fp64_state(self._h, out), "heff_fp64_state")
        return {"stacks_backed": bool(out[0]), "t_backed": bool(out[1]),
                "stack_bytes": int(out[2]), "t_bytes": int(out[3])}

    def heff_split_paths(self):
        """Code paths of the split plan (see dmrg_heff_split_paths)."""
        out = (ctypes.c_longlong * 8)()
        self._check(_lib.dmrg_heff_split_paths(self._h, out), "heff_split_paths")
        keys = ["items1", "items2", "wide_blocks", "packed_r2", "packed_r4", "max_parts",
                "multi_part_blocks", "extra_tiles"]
        return dict(zip(keys, list(out)))

    def heff_stage_info(self):
        """Per-stage work: flops1, flops2, A/B/T stack elements, psi_len."""
        out = np.zeros(6)
        self._check(_lib.dmrg_heff_stage_info(self._h, _dptr(out)), "heff_stage_info")
        keys = ["flops1", "flops2", "nA", "nB", "nT", "psi_len"]
        return dict(zip(keys, out.tolist()))

    def heff_entries(self):
        """H_eff term structure: int array of (psi block in, psi block out, terms)."""
        n = ctypes.c_int(0)
        self._check(_lib.dmrg_heff_entries(self._h, None, 0, ctypes.byref(n)), "heff_entries")
        out = np.zeros(3 * max(n.value, 1), dtype=np.int32)
        self._check(_lib.dmrg_heff_entries(self._h, out.ctypes.data_as(_I), n.value,
                                           ctypes.byref(n)), "heff_entries")
        return out[:3 * n.value].reshape(-1, 3)

    def heff_split_plan(self):
        """Split-precision plan: launches per apply, stage-1 / stage-2 tiles, split-K range."""
        out = np.zeros(4)
        self._check(_lib.dmrg_heff_split_plan(self._h, _dptr(out)), "heff_split_plan")
        return {"launches": int(out[0]), "tiles1": int(out[1]), "tiles2": int(out[2]),
                "ksub": int(out[3])}

    def heff_timing(self, enable):
        """Start (1) / stop (0) per-kernel event timing; returns accumulated
        [split_ms, stage1_ms, stage2_ms, partial_sum_ms, n_applies]."""
        out = np.zeros(5)
        self._check(_lib.dmrg_heff_timing(self._h, enable, _dptr(out)), "heff_timing")
        return out

    def heff_tuning(self):
        """Autotuner record: [(candidate, ms per apply), ...]; candidates below
        100000 are stage-2 split-K ranges, 100000 + 10 cap + order stage-1
        schedules (see the header)."""
        n = ctypes.c_int()
        self._check(_lib.dmrg_heff_tuning(self._h, None, 0, ctypes.byref(n)), "heff_tuning")
        out = np.zeros(2 * max(n.value, 1))
        self._check(_lib.dmrg_heff_tuning(self._h, _dptr(out), n.value, ctypes.byref(n)),
                    "heff_tuning")
        return [(int(out[2 * i]), float(out[2 * i + 1])) for i in range(n.value)]

    def set_graphs(self, enable):
        self._check(_lib.dmrg_set_graphs(self._h, int(enable)), "set_graphs")

    def memory_stats(self):
        """Largest device objects so far (bytes; see dmrg_memory_stats)."""
        out = np.zeros(6)
        self._check(_lib.dmrg_memory_stats(self._h, _dptr(out)), "memory_stats")
        keys = ["block", "enlarged_block", "ren_temp", "fp64_stacks", "split_copies",
                "device_in_use"]
        return dict(zip(keys, out.tolist()))

    def profile(self):
        out = np.zeros(7)
        self._check(_lib.dmrg_profile(self._h, _dptr(out)), "profile")
        keys = ["Diag_H", "Ren", "Tables", "Diag_D", "StVec", "Other", "n_matvec"]
        return dict(zip(keys, out.tolist()))
