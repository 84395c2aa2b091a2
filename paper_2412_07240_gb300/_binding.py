"""ctypes binding of libpmf (include/pmf.h): argument marshalling only.

Every step of the filter runs in the library's CUDA kernels; this module
converts Python/numpy arguments into the C structs, passes torch's current
CUDA stream, and turns return codes into exceptions.  It raises on import of
the library if libpmf.so has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_NX = 4
MAX_NZ = 3
MEAS_NPARAM = 24

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DEGENERATE, ERR_TIMEOUT, ERR_ADMISSION, ERR_UNSUPPORTED = range(8)
PREC = {"fp64": 0, "tf32": 1, "bf16x3": 3, "fp16x3": 4, "bf16x6": 5}
PSI = {"euler": 0, "exact": 1}
REALIGN = {"multilinear": 0, "shear": 1}
TRANSFORM = {"auto": 0, "gemm": 1, "fft": 2}
MEAS = {"linear": 0, "range": 1, "bearing_linear3": 2, "terrain_gm": 3}
ERRNAMES = {1: "PMF_ERR_ARG", 2: "PMF_ERR_OOM", 3: "PMF_ERR_CUDA", 4: "PMF_ERR_DEGENERATE",
            5: "PMF_ERR_TIMEOUT", 6: "PMF_ERR_ADMISSION", 7: "PMF_ERR_UNSUPPORTED"}


class PmfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Degenerate(PmfError):
    pass


class Unsupported(PmfError):
    pass


class PmfConfig(C.Structure):
    _fields_ = [("nx", C.c_int), ("N", C.c_int * MAX_NX), ("A", C.c_double * (MAX_NX * MAX_NX)),
                ("Q", C.c_double * (MAX_NX * MAX_NX)), ("m0", C.c_double * MAX_NX),
                ("P0", C.c_double * (MAX_NX * MAX_NX)), ("span_sigma", C.c_double),
                ("dt_sub", C.c_double), ("realign_rho", C.c_double), ("precision", C.c_int),
                ("psi_mode", C.c_int), ("realign_mode", C.c_int), ("transform", C.c_int)]


class PmfMeas(C.Structure):
    _fields_ = [("kind", C.c_int), ("nz", C.c_int), ("z", C.c_double * MAX_NZ),
                ("R", C.c_double * (MAX_NZ * MAX_NZ)), ("H", C.c_double * (MAX_NZ * MAX_NX)),
                ("p", C.c_double * MEAS_NPARAM)]


# (name, restype, argtypes) of every entry point declared in include/pmf.h
SIGNATURES = [
    ("pmf_config_defaults", None, [C.POINTER(PmfConfig)]),
    ("pmf_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(PmfConfig), C.c_void_p]),
    ("pmf_time_update", C.c_int, [C.c_void_p, C.c_double]),
    ("pmf_meas_update", C.c_int, [C.c_void_p, C.POINTER(PmfMeas)]),
    ("pmf_step", C.c_int, [C.c_void_p, C.POINTER(PmfMeas), C.c_double]),
    ("pmf_moments", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("pmf_get_pdf", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                              C.POINTER(C.c_double)]),
    ("pmf_sync", C.c_int, [C.c_void_p]),
    ("pmf_num_points", C.c_longlong, [C.c_void_p]),
    ("pmf_path", C.c_int, [C.c_void_p]),
    ("pmf_launch_count", C.c_longlong, [C.c_void_p]),
    ("pmf_last_error", C.c_char_p, [C.c_void_p]),
    ("pmf_destroy", None, [C.c_void_p]),
    ("pmf_batch_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(PmfConfig), C.POINTER(PmfMeas), C.c_int,
                                   C.c_size_t, C.c_void_p]),
    ("pmf_batch_step", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_int),
                                 C.POINTER(C.c_double), C.c_int]),
    ("pmf_batch_moments", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    ("pmf_batch_status", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
    ("pmf_batch_get_pdf", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    ("pmf_batch_bytes", C.c_longlong, [C.c_void_p]),
    ("pmf_batch_launch_count", C.c_longlong, [C.c_void_p]),
    ("pmf_batch_destroy", None, [C.c_void_p]),
    ("pmf_fdm_transition", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                     C.c_double, C.c_double, C.c_int, C.c_double, C.c_void_p]),
    ("pmf_server_create", C.c_int, [C.POINTER(C.c_void_p), C.c_size_t, C.c_int, C.c_int]),
    ("pmf_server_admit", C.c_int, [C.c_void_p, C.POINTER(PmfConfig), C.POINTER(PmfMeas), C.POINTER(C.c_int)]),
    ("pmf_server_evict", C.c_int, [C.c_void_p, C.c_int]),
    ("pmf_server_bytes", C.c_longlong, [C.c_void_p]),
    ("pmf_server_replay", C.c_int, [C.c_void_p, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    ("pmf_server_moments", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("pmf_server_get_pdf", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    ("pmf_server_last_error", C.c_char_p, [C.c_void_p]),
    ("pmf_server_destroy", None, [C.c_void_p]),
    ("pmf_moments_noalloc", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.c_void_p, C.c_void_p]),
    ("pmf_selftest_bounded_wait", C.c_int, [C.c_longlong, C.c_int, C.c_void_p]),
]
SERVE_NSTATS = 6

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpmf.so (building it first if allowed); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise ImportError(f"libpmf.so not built at {_build.LIB}")
        _build.build()
    lib = C.CDLL(_build.LIB)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _fill(dst, a, n):
    """Copy the first n values of a (flattened row-major) into the ctypes array dst."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())
    if a.size < n:
        raise ValueError(f"expected {n} values, got {a.size}")
    for i in range(n):
        dst[i] = float(a[i])


def _stream_handle(stream):
    if stream is not None:
        return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return C.c_void_p(0)


def make_config(cfg, precision="fp64", psi_mode="euler", transform="auto") -> PmfConfig:
    """Marshal a filter configuration (nx, N, A, Q, m0, P0, span, dt_sub, realign_rho)."""
    lib = load()
    c = PmfConfig()
    lib.pmf_config_defaults(C.byref(c))
    n = int(cfg.nx)
    c.nx = n
    for a in range(n):
        c.N[a] = int(cfg.N[a])
    _fill(c.A, cfg.A, n * n)
    _fill(c.Q, cfg.Q, n * n)
    _fill(c.m0, cfg.m0, n)
    _fill(c.P0, cfg.P0, n * n)
    c.span_sigma = float(getattr(cfg, "span", 6.0))
    c.dt_sub = float(getattr(cfg, "dt_sub", 0.01))
    c.realign_rho = float(getattr(cfg, "realign_rho", 0.5))
    c.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    c.psi_mode = PSI[psi_mode] if isinstance(psi_mode, str) else int(psi_mode)
    c.realign_mode = REALIGN[getattr(cfg, "realign_mode", "multilinear")]
    c.transform = TRANSFORM[transform] if isinstance(transform, str) else int(transform)
    return c


def make_meas(meas, z, nx) -> PmfMeas:
    """Marshal a measurement (kind, R, H) and its value z."""
    m = PmfMeas()
    m.kind = MEAS[meas.kind]
    R = np.asarray(meas.R, dtype=np.float64)
    nz = R.shape[0]
    m.nz = nz
    _fill(m.z, z, nz)
    _fill(m.R, R, nz * nz)
    if meas.H is not None:
        _fill(m.H, meas.H, nz * nx)
    params = getattr(meas, "params", None)
    if params is not None:
        _fill(m.p, params, len(np.ravel(params)))
    return m


def moments_noalloc(weights, N, c, M, out, stream=None) -> None:
    """pmf_moments_noalloc on device tensors ``weights`` (float64, prod N) and
    ``out`` (float64, 1 + nx + nx^2): {S0, mean, cov} without any allocation."""
    lib = load()
    nx = len(N)
    Na = (C.c_int * nx)(*[int(v) for v in N])
    ca = (C.c_double * nx)()
    Ma = (C.c_double * (nx * nx))()
    _fill(ca, c, nx)
    _fill(Ma, M, nx * nx)
    rc = lib.pmf_moments_noalloc(C.c_void_p(int(weights.data_ptr())), nx, Na, ca, Ma,
                                 C.c_void_p(int(out.data_ptr())), _stream_handle(stream))
    if rc != OK:
        raise PmfError(rc, "pmf_moments_noalloc failed")


def selftest_bounded_wait(polls: int, arrive: bool, stream=None) -> int:
    """pmf_selftest_bounded_wait: the return code of a bounded mbarrier wait
    (OK when the arrival happened, ERR_TIMEOUT when it gave up)."""
    return int(load().pmf_selftest_bounded_wait(int(polls), 1 if arrive else 0, _stream_handle(stream)))


class Filter:
    """One spectral point-mass filter resident on the GPU (a pmf_ctx)."""

    def __init__(self, cfg, precision="fp64", psi_mode="euler", stream=None, transform="auto"):
        self._lib = load()
        self.nx = int(cfg.nx)
        self.N = tuple(int(v) for v in cfg.N[: self.nx])
        self._cfg = make_config(cfg, precision, psi_mode, transform)
        self._stream = _stream_handle(stream)
        h = C.c_void_p()
        rc = self._lib.pmf_create(C.byref(h), C.byref(self._cfg), self._stream)
        if rc != OK:
            cls = Unsupported if rc == ERR_UNSUPPORTED else PmfError
            raise cls(rc, "pmf_create failed")
        self._h = h

    def _check(self, rc):
        if rc == OK:
            return
        msg = self._lib.pmf_last_error(self._h).decode(errors="replace")
        if rc == ERR_DEGENERATE:
            raise Degenerate(rc, msg)
        raise PmfError(rc, msg)

    def time_update(self, tau: float) -> None:
        self._check(self._lib.pmf_time_update(self._h, float(tau)))

    def meas_update(self, meas, z) -> None:
        m = make_meas(meas, z, self.nx)
        self._check(self._lib.pmf_meas_update(self._h, C.byref(m)))

    def step(self, meas, z, tau: float) -> None:
        m = make_meas(meas, z, self.nx)
        self._check(self._lib.pmf_step(self._h, C.byref(m), float(tau)))

    def sync(self) -> None:
        self._check(self._lib.pmf_sync(self._h))

    def moments(self):
        n = self.nx
        m = (C.c_double * n)()
        P = (C.c_double * (n * n))()
        self._check(self._lib.pmf_moments(self._h, m, P))
        return np.array(m[:]), np.array(P[:]).reshape(n, n)

    def pdf(self):
        n = self.nx
        out = np.empty(int(np.prod(self.N)), dtype=np.float64)
        c = (C.c_double * n)()
        M = (C.c_double * (n * n))()
        self._check(self._lib.pmf_get_pdf(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), c, M))
        return out.reshape(self.N), np.array(c[:]), np.array(M[:]).reshape(n, n)

    @property
    def path(self) -> int:
        return self._lib.pmf_path(self._h)

    @property
    def num_points(self) -> int:
        return int(self._lib.pmf_num_points(self._h))

    @property
    def launches(self) -> int:
        return int(self._lib.pmf_launch_count(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.pmf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class Batch:
    """Many independent 2-D filters resident on the GPU (a pmf_batch)."""

    def __init__(self, cfgs, models, precision="fp16x3", psi_mode="euler", hbm_budget=0, stream=None,
                 transform="auto"):
        self._lib = load()
        n = len(cfgs)
        self.count = n
        self.N = [tuple(int(v) for v in c.N[:2]) for c in cfgs]
        carr = (PmfConfig * n)()
        marr = (PmfMeas * n)()
        for i, (c, m) in enumerate(zip(cfgs, models)):
            carr[i] = make_config(c, precision, psi_mode, transform)
            marr[i] = make_meas(m, np.zeros(np.asarray(m.R).shape[0]), 2)
        self._stream = _stream_handle(stream)
        h = C.c_void_p()
        rc = self._lib.pmf_batch_create(C.byref(h), carr, marr, n, int(hbm_budget), self._stream)
        if rc != OK:
            cls = Unsupported if rc == ERR_UNSUPPORTED else PmfError
            raise cls(rc, "pmf_batch_create failed")
        self._h = h

    def step(self, ids, z, taus, do_meas=None) -> None:
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        k = ids.size
        zz = np.zeros((k, MAX_NZ))
        if z is not None:
            z = np.asarray(z, dtype=np.float64).reshape(k, -1)
            for j in range(z.shape[1]):   # column by column: a third of one strided 2-D copy
                zz[:, j] = z[:, j]
        t = np.asarray(taus, dtype=np.float64)
        taus = np.full(k, float(t)) if t.ndim == 0 else np.ascontiguousarray(np.broadcast_to(t, (k,)))
        dm = None if do_meas is None else np.ascontiguousarray(do_meas, dtype=np.int32)
        rc = self._lib.pmf_batch_step(self._h, _iptr(ids), _dptr(zz), None if dm is None else _iptr(dm),
                                      _dptr(taus), k)
        if rc != OK:
            raise PmfError(rc, "pmf_batch_step failed")

    def moments(self, ids=None, strict=True):
        """Means and covariances; with strict=False a filter that reported a
        degenerate normaliser does not raise (see status())."""
        ids = np.arange(self.count, dtype=np.int32) if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        k = ids.size
        m = np.empty((k, 2))
        P = np.empty((k, 2, 2))
        rc = self._lib.pmf_batch_moments(self._h, _iptr(ids), k, _dptr(m), _dptr(P))
        if rc == ERR_DEGENERATE:
            if not strict:
                return m, P
            raise Degenerate(rc, "degenerate normaliser in the batch")
        if rc != OK:
            raise PmfError(rc, "pmf_batch_moments failed")
        return m, P

    def status(self, ids=None):
        """Per-filter status words (0 = OK), cleared after reading."""
        ids = np.arange(self.count, dtype=np.int32) if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        st = np.empty(ids.size, dtype=np.int32)
        rc = self._lib.pmf_batch_status(self._h, _iptr(ids), ids.size, _iptr(st))
        if rc != OK:
            raise PmfError(rc, "pmf_batch_status failed")
        return st

    def pdf(self, i):
        out = np.empty(int(np.prod(self.N[i])))
        c = np.empty(2)
        M = np.empty(4)
        rc = self._lib.pmf_batch_get_pdf(self._h, int(i), _dptr(out), _dptr(c), _dptr(M))
        if rc != OK:
            raise PmfError(rc, "pmf_batch_get_pdf failed")
        return out.reshape(self.N[i]), c, M.reshape(2, 2)

    @property
    def bytes(self) -> int:
        return int(self._lib.pmf_batch_bytes(self._h))

    @property
    def launches(self) -> int:
        return int(self._lib.pmf_batch_launch_count(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.pmf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Resident filters of mixed dimension served by continuous batching (a pmf_server)."""

    def __init__(self, max_filters, precision="fp16x3", hbm_budget=0):
        self._lib = load()
        h = C.c_void_p()
        rc = self._lib.pmf_server_create(C.byref(h), int(hbm_budget), int(max_filters), PREC[precision])
        if rc != OK:
            raise PmfError(rc, "pmf_server_create failed")
        self._h = h
        self.nx = {}
        self.N = {}

    def _err(self, rc, what):
        msg = self._lib.pmf_server_last_error(self._h)
        msg = msg.decode() if msg else ""
        cls = Degenerate if rc == ERR_DEGENERATE else Unsupported if rc == ERR_UNSUPPORTED else PmfError
        return cls(rc, f"{what}: {msg}")

    def admit(self, cfg, model) -> int:
        """Admit a filter; returns its id (PmfError with code ERR_ADMISSION over the budget)."""
        nx = int(cfg.nx)
        c = make_config(cfg, "fp16x3")
        m = make_meas(model, np.zeros(np.asarray(model.R).shape[0]), nx)
        fid = C.c_int(-1)
        rc = self._lib.pmf_server_admit(self._h, C.byref(c), C.byref(m), C.byref(fid))
        if rc != OK:
            raise self._err(rc, "pmf_server_admit")
        self.nx[fid.value] = nx
        self.N[fid.value] = tuple(int(v) for v in cfg.N[:nx])
        return fid.value

    def evict(self, fid) -> None:
        rc = self._lib.pmf_server_evict(self._h, int(fid))
        if rc != OK:
            raise self._err(rc, "pmf_server_evict")
        self.nx.pop(int(fid), None)
        self.N.pop(int(fid), None)

    @property
    def bytes(self) -> int:
        return int(self._lib.pmf_server_bytes(self._h))

    def replay(self, t_arrival, ids, z, taus):
        """Replay a request log in real time; returns (latency seconds per request, stats dict)."""
        t = np.ascontiguousarray(t_arrival, dtype=np.float64)
        n = t.size
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        zz = np.zeros((n, MAX_NZ))
        z = np.asarray(z, dtype=np.float64).reshape(n, -1)
        zz[:, :z.shape[1]] = z
        taus = np.ascontiguousarray(taus, dtype=np.float64)
        lat = np.zeros(n)
        st = np.zeros(SERVE_NSTATS)
        rc = self._lib.pmf_server_replay(self._h, n, _dptr(t), _iptr(ids), _dptr(zz), _dptr(taus), _dptr(lat),
                                         _dptr(st))
        if rc != OK:
            raise self._err(rc, "pmf_server_replay")
        keys = ["wall_s", "batches", "launches", "max_batch", "mean_batch", "requests"]
        return lat, dict(zip(keys, st.tolist()))

    def moments(self, fid):
        n = self.nx[int(fid)]
        m = (C.c_double * n)()
        P = (C.c_double * (n * n))()
        rc = self._lib.pmf_server_moments(self._h, int(fid), m, P)
        if rc != OK:
            raise self._err(rc, "pmf_server_moments")
        return np.array(m[:]), np.array(P[:]).reshape(n, n)

    def pdf(self, fid):
        fid = int(fid)
        n = self.nx[fid]
        out = np.empty(int(np.prod(self.N[fid])))
        c = np.empty(n)
        M = np.empty(n * n)
        rc = self._lib.pmf_server_get_pdf(self._h, fid, _dptr(out), _dptr(c), _dptr(M))
        if rc != OK:
            raise self._err(rc, "pmf_server_get_pdf")
        return out.reshape(self.N[fid]), c, M.reshape(n, n)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.pmf_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fdm_transition(P_in, P_out, work, q, a, dt, l, delta0, stream=None) -> None:
    """pmf_fdm_transition on device float64 tensors P_in, P_out of shape (count, N)
    and work of at least count * N + 4 * N + 2 elements."""
    lib = load()
    count, N = int(P_in.shape[0]), int(P_in.shape[1])
    rc = lib.pmf_fdm_transition(C.c_void_p(int(P_in.data_ptr())), C.c_void_p(int(P_out.data_ptr())),
                                C.c_void_p(int(work.data_ptr())), N, count, float(q), float(a), float(dt), int(l),
                                float(delta0), _stream_handle(stream))
    if rc != OK:
        raise PmfError(rc, "pmf_fdm_transition failed")
