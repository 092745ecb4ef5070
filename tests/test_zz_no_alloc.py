"""rbx_forward_noalloc: the Born forward for callers that cannot allocate device memory.

It is called through the C ABI and must give the same D as rbx_forward on the same
tables, twice in a row (its fixed scratch array keeps the previous call's contents).
This file is collected last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


def test_noalloc_forward_matches_rbx_forward_twice():
    L = rbx.load()
    g = P.custom(50, 83, 1e-3, 36e-3, kind="water", ny=77)
    N = g.geom.n_xducers
    job = rbx.Job()
    job.set_geometry(g.geom)
    X = job.X
    rng = np.random.default_rng(5)
    T = torch.tensor(rng.uniform(1e-5, 6e-5, (N, X)), dtype=torch.float32, device="cuda")
    a = torch.tensor(rng.uniform(3.0, 30.0, (N, X)), dtype=torch.float32, device="cuda")
    a[3, 7] = 0.0                                                    # one uncovered entry
    gam = torch.tensor(rng.uniform(-3, 3, (N, X)), dtype=torch.float32, device="cuda")
    K = torch.zeros((N, X), dtype=torch.uint8, device="cuda")
    exits = torch.zeros((N, N - 1, 4), dtype=torch.float32, device="cuda")
    job.set_tables(T, a, gam, K, exits)
    f = 3.1e5
    dm = rng.standard_normal((g.geom.ny, g.geom.nx)) * 1e-9
    D_ref = job.forward(f, torch.tensor(dm, dtype=torch.float32, device="cuda")).cpu().numpy()
    idx = job.mask_idx().cpu().numpy()
    w = 2 * math.pi * f
    v = torch.tensor((w * w * g.geom.dx ** 2 * dm.astype(np.float32).astype(np.float64).ravel()[idx]),
                     dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream or None
    err = C.create_string_buffer(256)
    for call in range(2):
        D = torch.full((N, N), float("nan"), dtype=torch.complex64, device="cuda")
        st = L.rbx_forward_noalloc(T.data_ptr(), a.data_ptr(), K.data_ptr(), v.data_ptr(), N, X, f, g.geom.c0,
                                   D.data_ptr(), stream, err, len(err))
        assert st == 0, err.value.decode()
        Dn = D.cpu().numpy()
        rel = np.linalg.norm(Dn - D_ref) / np.linalg.norm(D_ref)
        assert rel <= 1e-5, (call, rel)
    job.close()


def test_noalloc_forward_rejects_oversized_problems():
    L = rbx.load()
    err = C.create_string_buffer(256)
    d = torch.zeros(16, device="cuda")
    st = L.rbx_forward_noalloc(d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 1025, 4, 3e5, 1500.0,
                               d.data_ptr(), None, err, len(err))
    assert st == 1 and b"1024" in err.value


def _noalloc(L, T, a, K, v, f, c0):
    """One call through the C ABI on device tensors; returns D as a host array."""
    N, X = T.shape
    D = torch.full((N, N), float("nan"), dtype=torch.complex64, device="cuda")
    err = C.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream or None
    st = L.rbx_forward_noalloc(T.data_ptr(), a.data_ptr(), K.data_ptr(), v.data_ptr(), N, X, f, c0, D.data_ptr(),
                               stream, err, len(err))
    assert st == 0, err.value.decode()
    return D.cpu().numpy()


def test_noalloc_forward_matches_oracle_through_caustics(oracle_mod):
    """Against the FP64 oracle's Born forward (Eqs. perturb1, derivative) on identical tables
    that carry caustic counts: a strong slow Gaussian lens sends the central rays of every fan
    through a caustic, so entries with K > 0 take the phase shift -pi K / 2 of Eq.
    phase-discretised. Relative L2 <= 1e-5 (FP32 tolerance), on two calls in a row."""
    L = rbx.load()
    g = P.Geometry(nx=96, ny=96, dx=1e-3, n_xducers=64, ring_radius=45e-3)
    Xg, Yg = g.coords()
    c = 1500.0 / (1 + 0.25 * np.exp(-(Xg ** 2 + Yg ** 2) / (8e-3) ** 2))
    f = 1e6
    o = oracle_mod.Oracle(g)
    ns, f6 = o.fields_for(c, f)
    tb = o.tables(f6)
    assert tb.uncovered == 0 and (tb.K > 0).sum() > 0
    T32, a32, K8 = tb.T.astype(np.float32), tb.a.astype(np.float32), tb.K.astype(np.uint8)
    rng = np.random.default_rng(11)
    w = 2 * math.pi * f
    v32 = (w * w * g.dx ** 2 * rng.standard_normal(o.X) * 1e-9).astype(np.float32)
    args = [T32.astype(np.float64), a32.astype(np.float64)]
    D_ref = oracle_mod.forward_rows(o, f, *args, K8.astype(np.int32), v32.astype(np.float64))
    D_noK = oracle_mod.forward_rows(o, f, *args, np.zeros_like(K8, np.int32), v32.astype(np.float64))
    assert np.linalg.norm(D_noK - D_ref) / np.linalg.norm(D_ref) > 1e-3     # the caustic phase matters here
    dv = lambda x: torch.tensor(x, device="cuda")
    for call in range(2):
        D = _noalloc(L, dv(T32), dv(a32), dv(K8), dv(v32), f, g.c0)
        rel = np.linalg.norm(D - D_ref) / np.linalg.norm(D_ref)
        assert rel <= 1e-5, (call, rel)


def test_noalloc_forward_at_the_largest_size(oracle_mod):
    """N = 1024, the largest ring the fixed scratch admits (its N x N partial sums then leave
    room for one split, so the contraction runs unsplit): against rbx_forward on the same
    tables over all pairs and against the oracle on sampled rows, with caustic counts 0-2."""
    L = rbx.load()
    g = P.custom(1024, 96, 1e-3, 45e-3, kind="water")
    N = g.geom.n_xducers
    job = rbx.Job()
    job.set_geometry(g.geom)
    X = job.X
    rng = np.random.default_rng(6)
    T = rng.uniform(1e-5, 6e-5, (N, X)).astype(np.float32)
    a = rng.uniform(3.0, 30.0, (N, X)).astype(np.float32)
    a[rng.integers(0, N, 50), rng.integers(0, X, 50)] = 0.0          # some uncovered entries
    K = rng.integers(0, 3, (N, X)).astype(np.uint8)
    dv = lambda x: torch.tensor(x, device="cuda")
    job.set_tables(dv(T), dv(a), dv(rng.uniform(-3, 3, (N, X)).astype(np.float32)), dv(K),
                   torch.zeros((N, N - 1, 4), dtype=torch.float32, device="cuda"))
    f = 4.2e5
    dm = rng.standard_normal((g.geom.ny, g.geom.nx)) * 1e-9
    D_job = job.forward(f, torch.tensor(dm, dtype=torch.float32, device="cuda")).cpu().numpy()
    idx = job.mask_idx().cpu().numpy()
    job.close()
    w = 2 * math.pi * f
    v32 = (w * w * g.geom.dx ** 2 * dm.astype(np.float32).astype(np.float64).ravel()[idx]).astype(np.float32)
    for call in range(2):
        D = _noalloc(L, dv(T), dv(a), dv(K), dv(v32), f, g.geom.c0)
        assert np.linalg.norm(D - D_job) / np.linalg.norm(D_job) <= 1e-5, call
    rows = np.array([0, 1, 333, 511, 512, 1023])
    o = oracle_mod.Oracle(g.geom)
    D_or = oracle_mod.forward_rows(o, f, T[rows].astype(np.float64), a[rows].astype(np.float64),
                                   K[rows].astype(np.int32), v32.astype(np.float64))
    blk = D[np.ix_(rows, rows)]
    assert np.linalg.norm(blk - D_or) / np.linalg.norm(D_or) <= 1e-5
