"""Thin Python binding of librbx (include/rbx.h): argument marshalling only.

Every step of the update runs in the library's CUDA kernels; this module only passes
device pointers of torch tensors (PyTorch provides device memory and streams) and
host scalars. It raises if the compiled library is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_build", "librbx.so")

RBX_FP32, RBX_BF16, RBX_BF16X3 = 0, 1, 2
STATUS = {0: "RBX_OK", 1: "RBX_EINVAL", 2: "RBX_ENOMEM", 3: "RBX_ECUDA", 4: "RBX_ESTATE", 5: "RBX_ENUMERIC",
          6: "RBX_ETIMEOUT"}
KERNELS = ["trace", "synth_fwd", "gemm_fwd", "synth_bp", "gemm_bp", "fields", "tables", "update"]

_lock = threading.Lock()
_lib = None


class RbxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("x0", C.c_double), ("y0", C.c_double),
                ("n_xducers", C.c_int), ("ring_radius", C.c_double), ("mask_radius", C.c_double),
                ("c0", C.c_double), ("ds", C.c_double), ("weight_mode", C.c_int), ("tau", C.c_double),
                ("precision", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("resid_norm2", C.c_double), ("rms_dc", C.c_double), ("max_abs_dc", C.c_double),
                ("dm_norm", C.c_double), ("n_uncovered", C.c_longlong), ("n_clamped", C.c_longlong),
                ("n_launches", C.c_longlong), ("ms_trace", C.c_float), ("ms_forward", C.c_float),
                ("ms_backproj", C.c_float), ("ms_total", C.c_float), ("ms_kernel", C.c_float * 8)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_kernel"}
        d["ms_kernel"] = dict(zip(KERNELS, list(self.ms_kernel)))
        return d


_P = C.c_void_p
_J = C.c_void_p
_SIGS = {
    "rbx_create": [C.POINTER(C.c_void_p), _P],
    "rbx_set_geometry": [_J, C.POINTER(Geometry), _P],
    "rbx_mask": [_J, C.POINTER(C.c_int), _P],
    "rbx_set_model": [_J, _P],
    "rbx_get_model": [_J, _P],
    "rbx_trace_rays": [_J, C.c_double],
    "rbx_set_tables": [_J, _P, _P, _P, _P, _P],
    "rbx_get_tables": [_J, _P, _P, _P, _P, _P, _P],
    "rbx_direct_green": [_J, C.c_double, _P],
    "rbx_forward": [_J, C.c_double, _P, _P],
    "rbx_predict": [_J, C.c_double, _P],
    "rbx_adjoint": [_J, C.c_double, _P, _P, C.c_int],
    "rbx_update_from_tables": [_J, C.c_double, C.c_double, _P, C.POINTER(Stats)],
    "rbx_update_frequency": [_J, C.c_double, C.c_double, _P, C.POINTER(Stats)],
    "rbx_update_frequency_host": [_J, C.c_double, C.c_double, _P, _P, C.POINTER(Stats)],
    "rbx_reconstruct": [_J, C.POINTER(C.c_double), C.c_int, _P, C.POINTER(Stats)],
    "rbx_synchronize": [_J],
    "rbx_destroy": [_J],
    "rbx_update_frequency_async": [_J, C.c_double, C.c_double, _P, C.c_int],
    "rbx_get_stats": [_J, C.c_int, C.POINTER(Stats)],
    "rbx_batch_run": [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.POINTER(C.c_double)), C.POINTER(C.c_int),
                      C.POINTER(C.c_void_p), C.c_int, C.POINTER(Stats), C.POINTER(C.c_float)],
    "rbx_server_create": [C.POINTER(C.c_void_p), C.c_size_t, C.c_int],
    "rbx_server_submit": [_P, C.POINTER(Geometry), _P, C.POINTER(C.c_double), C.c_int, _P,
                          C.POINTER(C.c_longlong)],
    "rbx_server_poll": [_P, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_double), _P, C.POINTER(Stats)],
    "rbx_server_wait": [_P, C.c_longlong, C.c_double],
    "rbx_server_cancel": [_P, C.c_longlong],
    "rbx_set_absorption": [_P, _P, C.c_double],
    "rbx_set_integration": [_P, C.c_int],
    "rbx_set_linking": [_P, C.c_int],
    "rbx_update_set": [_P, C.POINTER(C.c_double), C.c_int, C.c_double, _P, C.POINTER(Stats)],
    "rbx_get_tuning": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "rbx_get_tuning_times": [_P, C.POINTER(C.c_float), C.POINTER(C.c_int)],
    "rbx_set_slot_timing": [_J, C.c_int],
    "rbx_selftest_bounded_wait": [C.POINTER(C.c_int)],
    "rbx_pool_usage": [C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.c_int],
    "rbx_server_times": [_P, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "rbx_server_info": [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)],
    "rbx_server_destroy": [_P],
    "rbx_forward_noalloc": [_P, _P, _P, _P, C.c_int, C.c_int, C.c_double, C.c_double, _P, _P, C.c_char_p,
                            C.c_size_t],
}


def exported_symbols() -> list[str]:
    return list(_SIGS) + ["rbx_last_error", "rbx_server_error", "rbx_estimate_bytes", "rbx_autotune"]


def autotune(mode: int = -1) -> int:
    """Set (0 heuristic, 1 autotune) or query (-1) the forward split autotuning; returns the previous mode."""
    return int(load().rbx_autotune(int(mode)))


def selftest_bounded_wait() -> bool:
    """Run the bounded-wait diagnostic (rbx_selftest_bounded_wait): True when a wait on a barrier
    that nothing signals gave up after the library's bound, as it must."""
    t = C.c_int()
    st = load().rbx_selftest_bounded_wait(C.byref(t))
    if st != 0:
        raise RbxError(st, "rbx_selftest_bounded_wait failed")
    return bool(t.value)


def pool_usage(trim: bool = False) -> dict:
    """Bytes of the device's stream-ordered pool in live allocations and reserved (rbx_pool_usage)."""
    u, r = C.c_size_t(), C.c_size_t()
    st = load().rbx_pool_usage(C.byref(u), C.byref(r), int(trim))
    if st != 0:
        raise RbxError(st, "pool query failed")
    return dict(used=u.value, reserved=r.value)


def estimate_bytes(g, nf: int, precision: int = RBX_BF16) -> int:
    """Device bytes the server reserves for one request of this geometry (rbx_estimate_bytes)."""
    G = geometry_struct(g, precision)
    return int(load().rbx_estimate_bytes(C.byref(G), int(nf)))


def load(path: str | None = None):
    """Load librbx.so (built by paper_2211_00316_gb300.build); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB
            if not os.path.exists(p):
                raise RuntimeError(f"librbx.so not built ({p}); run __graft_entry__.build()")
            L = C.CDLL(p)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.rbx_last_error.argtypes = [_J]
            L.rbx_last_error.restype = C.c_char_p
            L.rbx_server_error.argtypes = [_P, C.c_longlong]
            L.rbx_server_error.restype = C.c_char_p
            L.rbx_autotune.argtypes = [C.c_int]
            L.rbx_autotune.restype = C.c_int
            L.rbx_estimate_bytes.argtypes = [C.POINTER(Geometry), C.c_int]
            L.rbx_estimate_bytes.restype = C.c_size_t
            _lib = L
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


class Job:
    """One reconstruction job: owns the library handle and its device workspaces."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        """Bind the job to `stream` (default: torch's current stream), so the library's
        kernels are ordered with torch's copies into and out of the tensors passed here."""
        self.L = load()
        self.h = C.c_void_p()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        sp = self.stream.cuda_stream or None
        self._check(self.L.rbx_create(C.byref(self.h), sp))
        self.geom = None
        self.N = self.X = self.nx = self.ny = 0

    def _check(self, st: int):
        if st != 0:
            msg = self.L.rbx_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise RbxError(st, msg)

    def close(self):
        if self.h:
            self.L.rbx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- set-up
    def set_geometry(self, g, precision: int = RBX_FP32, weight_mode: int | None = None, tau: float | None = None):
        """g: a phantoms.Geometry (or any object with the same attributes); its xducer_xy
        (N x 2, optional) places the transducers on the ring."""
        G = Geometry(g.nx, g.ny, g.dx, g.x0, g.y0, g.n_xducers, g.ring_radius, g.mask_radius, g.c0, g.ds,
                     g.weight_mode if weight_mode is None else weight_mode, g.tau if tau is None else tau, precision)
        xy = getattr(g, "xducer_xy", None)
        xy = None if xy is None else np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1))
        self._check(self.L.rbx_set_geometry(self.h, C.byref(G), None if xy is None else xy.ctypes.data))
        self.geom = g
        self.N, self.nx, self.ny = g.n_xducers, g.nx, g.ny
        X = C.c_int()
        self._check(self.L.rbx_mask(self.h, C.byref(X), None))
        self.X = X.value

    def mask_idx(self) -> torch.Tensor:
        idx = torch.empty(self.X, dtype=torch.int32, device="cuda")
        self._check(self.L.rbx_mask(self.h, None, _ptr(idx)))
        self.sync()
        return idx

    def set_model(self, c: torch.Tensor):
        self._check(self.L.rbx_set_model(self.h, _ptr(c)))

    def set_absorption(self, alpha0: torch.Tensor | None, y: float = 1.4):
        """Absorption map alpha0 [ny][nx] (Np (rad/s)^-y m^-1, float32 on the device) and
        power-law exponent y; None returns to a lossless medium (rbx_set_absorption)."""
        if alpha0 is None:
            self._check(self.L.rbx_set_absorption(self.h, None, float(y)))
            return
        a = alpha0.contiguous().to(torch.float32)
        self._check(self.L.rbx_set_absorption(self.h, _ptr(a), float(y)))

    def set_integration(self, raw: bool):
        """True: integrate on the non-smoothed map, no Born term (rbx_set_integration mode 1)."""
        self._check(self.L.rbx_set_integration(self.h, 1 if raw else 0))

    def set_linking(self, max_rays: int):
        """Secant linking of the direct term with at most max_rays new rays per pair (0: off)."""
        self._check(self.L.rbx_set_linking(self.h, int(max_rays)))

    def update_set(self, freqs, df: float, data: torch.Tensor) -> dict:
        """One update from a frequency set; data [nf][N][N] complex64 on the device."""
        fr = np.ascontiguousarray(freqs, dtype=np.float64)
        st = Stats()
        d = data.contiguous()
        self._check(self.L.rbx_update_set(self.h, fr.ctypes.data_as(C.POINTER(C.c_double)), len(fr), float(df),
                                          _ptr(d), C.byref(st)))
        return st.as_dict()

    def get_model(self) -> torch.Tensor:
        out = torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda")
        self._check(self.L.rbx_get_model(self.h, _ptr(out)))
        return out

    # ---------------------------------------------------------------- steps
    def trace_rays(self, f: float):
        self._check(self.L.rbx_trace_rays(self.h, f))

    def set_tables(self, T, a, gam, K, exits):
        self._check(self.L.rbx_set_tables(self.h, _ptr(T), _ptr(a), _ptr(gam), _ptr(K), _ptr(exits)))

    def get_tables(self):
        N, X = self.N, self.X
        T = torch.empty((N, X), dtype=torch.float32, device="cuda")
        a, gam, dg = torch.empty_like(T), torch.empty_like(T), torch.empty_like(T)
        K = torch.empty((N, X), dtype=torch.uint8, device="cuda")
        ex = torch.empty((N, N - 1, 4), dtype=torch.float32, device="cuda")
        self._check(self.L.rbx_get_tables(self.h, _ptr(T), _ptr(a), _ptr(gam), _ptr(K), _ptr(dg), _ptr(ex)))
        self.sync()
        return dict(T=T, a=a, gam=gam, K=K, dg=dg, exits=ex)

    def direct_green(self, f: float) -> torch.Tensor:
        out = torch.empty((self.N, self.N), dtype=torch.complex64, device="cuda")
        self._check(self.L.rbx_direct_green(self.h, f, _ptr(out)))
        return out

    def forward(self, f: float, dm: torch.Tensor) -> torch.Tensor:
        out = torch.empty((self.N, self.N), dtype=torch.complex64, device="cuda")
        self._check(self.L.rbx_forward(self.h, f, _ptr(dm), _ptr(out)))
        return out

    def predict(self, f: float, out: torch.Tensor | None = None) -> torch.Tensor:
        out = out if out is not None else torch.empty((self.N, self.N), dtype=torch.complex64, device="cuda")
        self._check(self.L.rbx_predict(self.h, f, _ptr(out)))
        return out

    def adjoint(self, f: float, R: torch.Tensor, preconditioned: bool) -> torch.Tensor:
        out = torch.empty(self.X, dtype=torch.complex64, device="cuda")
        self._check(self.L.rbx_adjoint(self.h, f, _ptr(R), _ptr(out), int(preconditioned)))
        return out

    def update_from_tables(self, f: float, df: float, data: torch.Tensor) -> dict:
        st = Stats()
        self._check(self.L.rbx_update_from_tables(self.h, f, df, _ptr(data), C.byref(st)))
        return st.as_dict()

    def update_frequency(self, f: float, df: float, data: torch.Tensor) -> dict:
        st = Stats()
        self._check(self.L.rbx_update_frequency(self.h, f, df, _ptr(data), C.byref(st)))
        return st.as_dict()

    def update_frequency_host(self, f: float, df: float, data_host, c_out_host=None) -> dict:
        st = Stats()
        self._check(self.L.rbx_update_frequency_host(self.h, f, df, _ptr(data_host), _ptr(c_out_host),
                                                     C.byref(st)))
        return st.as_dict()

    def reconstruct(self, freqs, data: torch.Tensor) -> list[dict]:
        fr = np.ascontiguousarray(freqs, dtype=np.float64)
        sts = (Stats * len(fr))()
        self._check(self.L.rbx_reconstruct(self.h, fr.ctypes.data_as(C.POINTER(C.c_double)), len(fr), _ptr(data),
                                           sts))
        return [s.as_dict() for s in sts]

    def update_frequency_async(self, f: float, df: float, data: torch.Tensor, slot: int = 0):
        self._check(self.L.rbx_update_frequency_async(self.h, f, df, _ptr(data), slot))

    def set_slot_timing(self, on: bool = True):
        """Per-slot device timings for update_frequency_async (rbx_set_slot_timing)."""
        self._check(self.L.rbx_set_slot_timing(self.h, int(on)))

    def get_stats(self, slot: int = 0) -> dict:
        st = Stats()
        self._check(self.L.rbx_get_stats(self.h, slot, C.byref(st)))
        return st.as_dict()

    def tuning(self) -> dict:
        sp, nc = C.c_int(), C.c_int()
        self._check(self.L.rbx_get_tuning(self.h, C.byref(sp), C.byref(nc)))
        ms, fu = (C.c_float * 4)(), C.c_int()
        self._check(self.L.rbx_get_tuning_times(self.h, ms, C.byref(fu)))
        return dict(fwd_splits=sp.value, candidates_timed=nc.value, fused_forward=bool(fu.value),
                    ms_synth_both=ms[0], ms_forward_gemm=ms[1], ms_synth_bp=ms[2], ms_forward_fused=ms[3])

    def sync(self):
        self._check(self.L.rbx_synchronize(self.h))


RBX_BATCH_GRAPH, RBX_BATCH_GROUPED = 1, 2


def batch_run(jobs: list, freqs: list, data: list, use_graph: bool = True, grouped: bool = False):
    """Batched form (rbx_batch_run): every job's sweep on its own stream, optionally one CUDA
    graph (use_graph) and one persistent trace launch per sweep step for all jobs (grouped).
    Returns (per-job last-update stats, device milliseconds of the whole batch)."""
    n = len(jobs)
    L = load()
    handles = (C.c_void_p * n)(*[j.h.value for j in jobs])
    fr = [np.ascontiguousarray(f, dtype=np.float64) for f in freqs]
    fptrs = (C.POINTER(C.c_double) * n)(*[f.ctypes.data_as(C.POINTER(C.c_double)) for f in fr])
    nf = (C.c_int * n)(*[len(f) for f in fr])
    dptrs = (C.c_void_p * n)(*[_ptr(d) for d in data])
    last = (Stats * n)()
    ms = C.c_float(0.0)
    flags = (RBX_BATCH_GRAPH if use_graph else 0) | (RBX_BATCH_GROUPED if grouped else 0)
    st = L.rbx_batch_run(handles, n, fptrs, nf, dptrs, flags, last, C.byref(ms))
    if st != 0:
        raise RbxError(st, L.rbx_last_error(jobs[0].h).decode())
    return [s.as_dict() for s in last], ms.value


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)


def geometry_struct(g, precision: int = RBX_FP32, weight_mode: int | None = None, tau: float | None = None):
    return Geometry(g.nx, g.ny, g.dx, g.x0, g.y0, g.n_xducers, g.ring_radius, g.mask_radius, g.c0, g.ds,
                    g.weight_mode if weight_mode is None else weight_mode, g.tau if tau is None else tau, precision)


class Server:
    """Served form (rbx_server_*): continuous batching of reconstruction requests."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 8):
        self.L = load()
        self.h = C.c_void_p()
        st = self.L.rbx_server_create(C.byref(self.h), int(hbm_budget_bytes), int(max_inflight))
        if st != 0:
            raise RbxError(st, "server creation failed")

    def submit(self, g, c_init, freqs, data, precision: int = RBX_BF16) -> int:
        """g: phantoms.Geometry; c_init (ny, nx) array; freqs (nf,); data (nf, N, N) complex."""
        G = geometry_struct(g, precision)
        c = np.ascontiguousarray(c_init, dtype=np.float32)
        fr = np.ascontiguousarray(freqs, dtype=np.float64)
        d = np.ascontiguousarray(data, dtype=np.complex64)
        t = C.c_longlong()
        st = self.L.rbx_server_submit(self.h, C.byref(G), c.ctypes.data, fr.ctypes.data_as(C.POINTER(C.c_double)),
                                      len(fr), d.ctypes.data, C.byref(t))
        if st != 0:
            raise RbxError(st, "submit failed")
        return t.value

    def poll(self, ticket: int, want_model: bool = False, shape=None):
        state, lat, last = C.c_int(), C.c_double(-1.0), Stats()
        out = np.empty(shape, np.float32) if want_model else None
        st = self.L.rbx_server_poll(self.h, ticket, C.byref(state), C.byref(lat),
                                    out.ctypes.data if out is not None else None, C.byref(last))
        return dict(state=state.value, status=st, latency_s=lat.value, model=out, last=last.as_dict(),
                    error=self.L.rbx_server_error(self.h, ticket).decode())

    def wait(self, ticket: int, timeout_s: float = 600.0) -> int:
        return self.L.rbx_server_wait(self.h, ticket, timeout_s)

    def cancel(self, ticket: int) -> int:
        return self.L.rbx_server_cancel(self.h, ticket)

    def times(self, ticket: int):
        """Seconds since server creation: submitted, started (-1 if not), ended (-1 if not)."""
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        st = self.L.rbx_server_times(self.h, ticket, C.byref(a), C.byref(b), C.byref(c))
        if st != 0:
            raise RbxError(st, "unknown ticket")
        return dict(submit=a.value, start=b.value, end=c.value)

    def info(self):
        q, r, b = C.c_int(), C.c_int(), C.c_size_t()
        self.L.rbx_server_info(self.h, C.byref(q), C.byref(r), C.byref(b))
        return dict(queued=q.value, running=r.value, bytes_in_use=b.value)

    def close(self):
        if self.h:
            self.L.rbx_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
