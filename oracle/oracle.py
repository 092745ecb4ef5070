"""ctypes front end of the FP64 CPU oracle (oracle/rbx_oracle.c).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import this module. It shares nothing with the CUDA library; both consume the
seeded inputs of paper_2211_00316_gb300.phantoms.

Every method below forwards to one C function of the oracle; the paper passage each
follows is cited in rbx_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rbx_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction so x86 and Arm agree)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(LIB)
            _declare(_lib)
    return _lib


class OGeom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("x0", C.c_double), ("y0", C.c_double),
                ("N", C.c_int), ("R", C.c_double), ("mask_r", C.c_double), ("c0", C.c_double),
                ("ds", C.c_double), ("weight_mode", C.c_int), ("tau", C.c_double), ("beta", C.POINTER(C.c_double))]


class OMedium(C.Structure):
    _fields_ = [("mode", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double), ("f", C.POINTER(C.c_double)), ("c1", C.c_double), ("gx", C.c_double),
                ("gy", C.c_double), ("al", C.POINTER(C.c_double)), ("nr", C.POINTER(C.c_double))]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_G = C.POINTER(OGeom)


def _declare(L):
    L.og_window.argtypes = [_G, C.c_double]; L.og_window.restype = C.c_int
    L.og_smooth.argtypes = [_G, _D, C.c_int, _D]; L.og_smooth.restype = None
    L.og_fields.argtypes = [_G, _D, _D]; L.og_fields.restype = None
    L.og_mask.argtypes = [_G, _I]; L.og_mask.restype = C.c_int
    L.og_trace_ray_flat.argtypes = [C.POINTER(OMedium), C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_int, _D]
    L.og_trace_ray_flat.restype = C.c_int
    L.og_tables.argtypes = [_G, _D, _I, C.c_int, _D, _D, _D, _I, _I, _D, C.POINTER(C.c_long)]
    L.og_tables.restype = C.c_long
    L.og_dgamma.argtypes = [_G, C.c_int, _D, _I, _D]; L.og_dgamma.restype = None
    L.og_direct_green.argtypes = [_G, C.c_double, _D, _D]; L.og_direct_green.restype = C.c_long
    L.og_forward.argtypes = [_G, C.c_double, C.c_int, _D, _D, _I, _D, _D]; L.og_forward.restype = None
    L.og_adjoint_plain.argtypes = [_G, C.c_double, C.c_int, _D, _D, _I, _D, _I, C.c_int, _D]
    L.og_adjoint_plain.restype = None
    L.og_backproject.argtypes = [_G, C.c_double, C.c_int, _D, _D, _D, _I, _D, _D, _I, C.c_int, _D]
    L.og_backproject.restype = None
    L.og_update.argtypes = [_G, C.c_double, C.c_double, C.c_int, _I, _D, _D, _D, _D]
    L.og_update.restype = C.c_int
    L.og_predict.argtypes = [_G, C.c_double, _D, _D, _D]; L.og_predict.restype = None
    L.og_update_frequency.argtypes = [_G, C.c_double, C.c_double, _D, _D, _D, _D]
    L.og_update_frequency.restype = C.c_int
    L.og_num_threads.argtypes = []; L.og_num_threads.restype = C.c_int
    L.og_smooth_abs.argtypes = [_G, _D, _D, C.c_double, C.c_double, C.c_int, _D, _D, _D]
    L.og_smooth_abs.restype = None
    L.og_tables_abs.argtypes = [_G, _D, _D, _I, C.c_int, _D, _D, _D, _I, _I, _D, C.POINTER(C.c_long)]
    L.og_tables_abs.restype = C.c_long
    L.og_forward_c.argtypes = [_G, C.c_double, C.c_int, _D, _D, _I, _D, _D]; L.og_forward_c.restype = None
    L.og_adjoint_plain_c.argtypes = [_G, C.c_double, C.c_int, _D, _D, _I, _D, _D, _I, C.c_int, _D]
    L.og_adjoint_plain_c.restype = None
    L.og_update_abs.argtypes = [_G, C.c_double, C.c_double, C.c_int, _I, _D, _D, _D, C.c_double, _D, _D]
    L.og_update_abs.restype = C.c_int
    L.og_predict_abs.argtypes = [_G, C.c_double, _D, _D, C.c_double, _D, _D]; L.og_predict_abs.restype = None
    L.og_update_frequency_abs.argtypes = [_G, C.c_double, C.c_double, _D, _D, C.c_double, _D, _D, _D]
    L.og_update_frequency_abs.restype = C.c_int
    L.og_tables_ext.argtypes = [_G, _D, _D, _D, _I, C.c_int, _D, _D, _D, _I, _I, _D, C.POINTER(C.c_long)]
    L.og_tables_ext.restype = C.c_long
    L.og_predict_ext.argtypes = [_G, C.c_double, _D, _D, C.c_double, C.c_int, _D, _D]
    L.og_predict_ext.restype = None
    L.og_update_set_ext.argtypes = [_G, _D, C.c_int, C.c_double, _D, _D, C.c_double, C.c_int, _D, _D, _D]
    L.og_update_set_ext.restype = C.c_int
    L.og_direct_green_linked.argtypes = [_G, C.POINTER(OMedium), C.c_double, _D, C.c_int, C.c_double, _D,
                                         C.POINTER(C.c_long), _D]
    L.og_direct_green_linked.restype = C.c_long


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _cplx_to_f64(z):
    z = np.ascontiguousarray(z, dtype=np.complex128)
    return z.view(np.float64)


class Tables:
    """Oracle tables of a set of fans: arrays [nfans][X]; exits [nfans][N-1][4]."""

    def __init__(self, fans, T, a, gam, K, cov, exits, uncovered, bad_rays):
        self.fans, self.T, self.a, self.gam, self.K, self.cov = fans, T, a, gam, K, cov
        self.exits, self.uncovered, self.bad_rays = exits, uncovered, bad_rays
        self.dg = None


class Oracle:
    """FP64 oracle bound to one geometry (a phantoms.Geometry)."""

    def __init__(self, geom, weight_mode: int | None = None):
        self.geom = geom
        wm = geom.weight_mode if weight_mode is None else weight_mode
        self.g = OGeom(geom.nx, geom.ny, geom.dx, geom.x0, geom.y0, geom.n_xducers, geom.ring_radius,
                       geom.mask_radius, geom.c0, geom.ds, wm, geom.tau)
        xy = getattr(geom, "xducer_xy", None)
        if xy is not None:
            # transducer positions on the ring (Sec. 2.1) as their angles, counterclockwise
            xy = np.asarray(xy, np.float64).reshape(geom.n_xducers, 2)
            self._beta = np.ascontiguousarray(np.arctan2(xy[:, 1], xy[:, 0]))
            self.g.beta = _d(self._beta)
        self.L = lib()
        self.N = geom.n_xducers
        self.X = self.L.og_mask(C.byref(self.g), None)
        self.idx = np.zeros(self.X, np.int32)
        self.L.og_mask(C.byref(self.g), _i(self.idx))

    @staticmethod
    def threads() -> int:
        return lib().og_num_threads()

    # a1
    def window(self, f: float) -> int:
        return self.L.og_window(C.byref(self.g), f)

    def smooth(self, c, w: int):
        c = _f64(c)
        out = np.zeros_like(c)
        self.L.og_smooth(C.byref(self.g), _d(c), w, _d(out))
        return out

    def fields(self, ns):
        ns = _f64(ns)
        out = np.zeros((6,) + ns.shape)
        self.L.og_fields(C.byref(self.g), _d(ns), _d(out))
        return out

    def fields_for(self, c, f: float):
        ns = self.smooth(c, self.window(f))
        return ns, self.fields(ns)

    def smooth_abs(self, c, alpha0, y: float, f: float, w: int | None = None):
        """Smoothed 1/c, ray slowness n_e and absorption coefficient alpha (Np/m)."""
        c, a0 = _f64(c), _f64(alpha0)
        ns, ne, al = np.zeros_like(c), np.zeros_like(c), np.zeros_like(c)
        self.L.og_smooth_abs(C.byref(self.g), _d(c), _d(a0), y, f, self.window(f) if w is None else w, _d(ns),
                             _d(ne), _d(al))
        return ns, ne, al

    def fields_for_abs(self, c, alpha0, y: float, f: float):
        """(ns, fields of n_e, alpha): the lossy counterpart of fields_for."""
        ns, ne, al = self.smooth_abs(c, alpha0, y, f)
        return ns, self.fields(ne), al

    # a2
    def trace_ray(self, xs, ys, gam0, f6=None, linear=None, maxs=None, R=None, ds=None, al=None, nr=None):
        """Samples of one ray: columns x, y, T, J, a, gamma, K, n, dH, px, py, s, B (al: alpha map,
        nr: slowness integrated along the ray)."""
        g = self.geom
        maxs = maxs or int(np.ceil(3 * g.ring_radius / (ds or g.ds))) + 8
        if linear is not None:
            c1, gx, gy = linear
            med = OMedium(1, g.nx, g.ny, g.dx, g.x0, g.y0, None, c1, gx, gy, None, None)
        else:
            f6 = _f64(f6)
            alp = None
            if al is not None:
                al = _f64(al)
                alp = _d(al)
            nrp = None
            if nr is not None:
                nr = _f64(nr)
                nrp = _d(nr)
            med = OMedium(0, g.nx, g.ny, g.dx, g.x0, g.y0, _d(f6), 0.0, 0.0, 0.0, alp, nrp)
        rows = np.zeros((maxs + 1, 13))
        M = self.L.og_trace_ray_flat(C.byref(med), R or g.ring_radius, ds or g.ds, xs, ys, gam0, maxs, _d(rows))
        self._keep = (f6, al, nr)
        if M < 0:
            raise RuntimeError("ray did not reach the ring")
        return rows[:M + 1]

    # a2 + a3 (+ a4 when all fans are traced)
    def tables(self, f6, fans=None, al=None, nr=None) -> Tables:
        """Tables of the listed fans (all when None); al: alpha map of a lossy medium; nr: the
        slowness integrated along the rays (default: the traced, smoothed one)."""
        f6 = _f64(f6)
        alp = nrp = None
        if al is not None:
            al = _f64(al)
            alp = _d(al)
        if nr is not None:
            nr = _f64(nr)
            nrp = _d(nr)
        N, X = self.N, self.X
        fl = np.arange(N, dtype=np.int32) if fans is None else _i32(fans)
        nf = len(fl)
        T = np.zeros((nf, X)); a = np.zeros((nf, X)); gam = np.zeros((nf, X))
        K = np.zeros((nf, X), np.int32); cov = np.zeros((nf, X), np.int32)
        exits = np.zeros((nf, N - 1, 4))
        bad = C.c_long(0)
        unc = self.L.og_tables_ext(C.byref(self.g), _d(f6), alp, nrp, _i(fl), nf, _d(T), _d(a), _d(gam), _i(K),
                                   _i(cov), _d(exits), C.byref(bad))
        t = Tables(fl, T, a, gam, K, cov, exits, int(unc), int(bad.value))
        if fans is None:
            t.dg = self.dgamma(gam, cov)
        return t

    def dgamma(self, gam, cov):
        gam, cov = _f64(gam), _i32(cov)
        out = np.zeros_like(gam)
        self.L.og_dgamma(C.byref(self.g), self.X, _d(gam), _i(cov), _d(out))
        return out

    # a5
    def direct_green(self, f: float, exits):
        exits = _f64(exits)
        out = np.zeros((self.N, self.N), np.complex128)
        cl = self.L.og_direct_green(C.byref(self.g), f, _d(exits), _d(out.view(np.float64)))
        return out, int(cl)

    def direct_green_linked(self, f: float, f6, exits, al=None, nr=None, maxit: int = 8, tol: float = 1e-6,
                            linear=None):
        """Direct Green's function on secant-linked rays (linear: analytic c1 + gx x + gy y medium)."""
        g = self.geom
        keep = []
        if linear is not None:
            c1, gx, gy = linear
            med = OMedium(1, g.nx, g.ny, g.dx, g.x0, g.y0, None, c1, gx, gy, None, None)
        else:
            f6 = _f64(f6)
            keep.append(f6)
            ptrs = []
            for arr in (al, nr):
                if arr is None:
                    ptrs.append(None)
                else:
                    arr = _f64(arr)
                    keep.append(arr)
                    ptrs.append(_d(arr))
            med = OMedium(0, g.nx, g.ny, g.dx, g.x0, g.y0, _d(f6), 0.0, 0.0, 0.0, ptrs[0], ptrs[1])
        exits = _f64(exits)
        out = np.zeros((self.N, self.N), np.complex128)
        Tl = np.zeros((self.N, self.N))
        unc = C.c_long(0)
        cl = self.L.og_direct_green_linked(C.byref(self.g), C.byref(med), f, _d(exits), maxit, tol,
                                           _d(out.view(np.float64)), C.byref(unc), _d(Tl))
        return out, int(cl), int(unc.value), Tl

    # a7
    def forward(self, f: float, T, a, K, v):
        """D[e, r] = sum_x G_r G_e v (v already includes omega^2 dA)."""
        T, a, K, v = _f64(T), _f64(a), _i32(K), _f64(v)
        D = np.zeros((self.N, self.N), np.complex128)
        self.L.og_forward(C.byref(self.g), f, self.X, _d(T), _d(a), _i(K), _d(v), _d(D.view(np.float64)))
        return D

    def forward_c(self, f: float, T, a, K, v):
        """D[e, r] = sum_x G_r G_e v with complex v (already Upsilon_m dA dm)."""
        T, a, K = _f64(T), _f64(a), _i32(K)
        vf = _cplx_to_f64(v)
        D = np.zeros((self.N, self.N), np.complex128)
        self.L.og_forward_c(C.byref(self.g), f, self.X, _d(T), _d(a), _i(K), _d(vf), _d(D.view(np.float64)))
        return D

    def adjoint_plain_c(self, f: float, T, a, K, ups, R, nodes=None):
        """dA conj(Upsilon_m) sum conj(G_r G_e) R at the listed nodes (ups: Upsilon_m there)."""
        T, a, K = _f64(T), _f64(a), _i32(K)
        Rf, uf = _cplx_to_f64(R), _cplx_to_f64(ups)
        nodes = np.arange(self.X, dtype=np.int32) if nodes is None else _i32(nodes)
        out = np.zeros(len(nodes), np.complex128)
        self.L.og_adjoint_plain_c(C.byref(self.g), f, self.X, _d(T), _d(a), _i(K), _d(uf), _d(Rf), _i(nodes),
                                  len(nodes), _d(out.view(np.float64)))
        return out

    def adjoint_plain(self, f: float, T, a, K, R, nodes=None):
        T, a, K = _f64(T), _f64(a), _i32(K)
        Rf = _cplx_to_f64(R)
        nodes = np.arange(self.X, dtype=np.int32) if nodes is None else _i32(nodes)
        out = np.zeros(len(nodes), np.complex128)
        self.L.og_adjoint_plain(C.byref(self.g), f, self.X, _d(T), _d(a), _i(K), _d(Rf), _i(nodes), len(nodes),
                                _d(out.view(np.float64)))
        return out

    # a8
    def backproject(self, f: float, T, a, gam, K, dg, R, nodes=None):
        T, a, gam, K, dg = _f64(T), _f64(a), _f64(gam), _i32(K), _f64(dg)
        Rf = _cplx_to_f64(R)
        nodes = np.arange(self.X, dtype=np.int32) if nodes is None else _i32(nodes)
        out = np.zeros(len(nodes), np.complex128)
        self.L.og_backproject(C.byref(self.g), f, self.X, _d(T), _d(a), _d(gam), _i(K), _d(dg), _d(Rf),
                              _i(nodes), len(nodes), _d(out.view(np.float64)))
        return out

    # a9
    def update(self, f: float, df: float, grad_re, c):
        grad_re, c = _f64(grad_re), _f64(c)
        out = np.zeros_like(c)
        st = np.zeros(3)
        bad = self.L.og_update(C.byref(self.g), f, df, self.X, _i(self.idx), _d(grad_re), _d(c), _d(out), _d(st))
        return out, st, bad

    def update_abs(self, f: float, df: float, grad, c, alpha0, y: float):
        gf, c, a0 = _cplx_to_f64(grad), _f64(c), _f64(alpha0)
        out = np.zeros_like(c)
        st = np.zeros(3)
        bad = self.L.og_update_abs(C.byref(self.g), f, df, self.X, _i(self.idx), _d(gf), _d(c), _d(a0), y, _d(out),
                                   _d(st))
        return out, st, bad

    # composites
    def predict_abs(self, f: float, c, alpha0, y: float):
        c, a0 = _f64(c), _f64(alpha0)
        out = np.zeros((self.N, self.N), np.complex128)
        st = np.zeros(3)
        self.L.og_predict_abs(C.byref(self.g), f, _d(c), _d(a0), y, _d(out.view(np.float64)), _d(st))
        return out, st

    def update_frequency_abs(self, f: float, df: float, c, alpha0, y: float, data):
        c, a0 = _f64(c), _f64(alpha0)
        dataf = _cplx_to_f64(data)
        out = np.zeros_like(c)
        st = np.zeros(7)
        bad = self.L.og_update_frequency_abs(C.byref(self.g), f, df, _d(c), _d(a0), y, _d(dataf), _d(out), _d(st))
        return out, st, bad

    def predict_ext(self, f: float, c, alpha0=None, y: float = 1.4, raw: bool = False, link: bool = False):
        """Predicted data; raw: integration on the non-smoothed map, no Born term (Sec. 6.3.2);
        link: direct Green's function on secant-linked rays."""
        c = _f64(c)
        a0 = None if alpha0 is None else _f64(alpha0)
        out = np.zeros((self.N, self.N), np.complex128)
        st = np.zeros(3)
        self.L.og_predict_ext(C.byref(self.g), f, _d(c), None if a0 is None else _d(a0), y,
                              int(raw) | (2 if link else 0), _d(out.view(np.float64)), _d(st))
        return out, st

    def update_set(self, freqs, df: float, c, data, alpha0=None, y: float = 1.4, raw: bool = False,
                   link: bool = False):
        """One update from a frequency set (data: [nf][N][N])."""
        fr = np.ascontiguousarray(freqs, dtype=np.float64)
        c = _f64(c)
        a0 = None if alpha0 is None else _f64(alpha0)
        dataf = _cplx_to_f64(data)
        out = np.zeros_like(c)
        st = np.zeros(7)
        bad = self.L.og_update_set_ext(C.byref(self.g), _d(fr), len(fr), df, _d(c), None if a0 is None else _d(a0),
                                       y, int(raw) | (2 if link else 0), _d(dataf), _d(out), _d(st))
        return out, st, bad

    def predict(self, f: float, c):
        c = _f64(c)
        out = np.zeros((self.N, self.N), np.complex128)
        st = np.zeros(3)
        self.L.og_predict(C.byref(self.g), f, _d(c), _d(out.view(np.float64)), _d(st))
        return out, st

    def update_frequency(self, f: float, df: float, c, data):
        c = _f64(c)
        dataf = _cplx_to_f64(data)
        out = np.zeros_like(c)
        st = np.zeros(7)
        bad = self.L.og_update_frequency(C.byref(self.g), f, df, _d(c), _d(dataf), _d(out), _d(st))
        return out, st, bad

    # helpers shared by tests
    @staticmethod
    def upsilon(f: float, c, alpha0, y: float):
        """Upsilon_m = omega c k~, k~ = omega/c + alpha0 omega^y (tan(pi y/2) + i) (elementwise)."""
        w = 2 * np.pi * f
        c, a0 = np.asarray(c, float), np.asarray(alpha0, float)
        return w * c * (w / c + a0 * w ** y * (np.tan(np.pi * y / 2) + 1j))

    def rough_v(self, f: float, c, ns):
        """v[x] = omega^2 dA (m - m_s) on the mask (Born term of the rough part)."""
        w = 2 * np.pi * f
        cm = np.asarray(c, float).ravel()[self.idx]
        nm = np.asarray(ns, float).ravel()[self.idx]
        return w * w * self.geom.dx ** 2 * (1.0 / cm ** 2 - nm ** 2)


def forward_rows(o: Oracle, f: float, T, a, K, v):
    """og_forward restricted to the fans whose tables are the rows of [n][X] arrays:
    returns the n x n block of D between those fans."""
    g = OGeom.from_buffer_copy(o.g)
    g.N = T.shape[0]
    T, a, K, v = _f64(T), _f64(a), _i32(K), _f64(v)
    D = np.zeros((g.N, g.N), np.complex128)
    o.L.og_forward(C.byref(g), f, T.shape[1], _d(T), _d(a), _i(K), _d(v), _d(D.view(np.float64)))
    return D


def backproject_nodes(o: Oracle, f: float, T, a, gam, K, dg, R):
    """og_backproject on tables given only at nn nodes ([N][nn] arrays): returns nn values."""
    T, a, gam, K, dg = _f64(T), _f64(a), _f64(gam), _i32(K), _f64(dg)
    nn = T.shape[1]
    nodes = np.arange(nn, dtype=np.int32)
    out = np.zeros(nn, np.complex128)
    o.L.og_backproject(C.byref(o.g), f, nn, _d(T), _d(a), _d(gam), _i(K), _d(dg), _d(_cplx_to_f64(R)),
                       _i(nodes), nn, _d(out.view(np.float64)))
    return out
