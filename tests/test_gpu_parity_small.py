"""CUDA path against the FP64 oracle on small cases (element by element).

Tolerances (stated for the method, read per stage):
  tables: T <= 1e-9 s absolute; a relative <= 1e-5; gamma <= 1e-5 rad; K exact; mask exact;
  forward / adjoint / direct Green's function on identical (oracle, FP32-rounded) tables:
  relative L2 <= 1e-5 (FP32 path);
  update: RMS of c_gpu - c_oracle over the mask <= 0.05 m/s (own tables), and much tighter
  on identical tables.
"""
import math

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def wrap(d):
    return np.angle(np.exp(1j * d))


class Case:
    def __init__(self, oracle_mod, w, f):
        self.w, self.g, self.f = w, w.geom, f
        self.o = oracle_mod.Oracle(self.g)
        self.c32 = w.c_init.astype(np.float32)
        self.c64 = self.c32.astype(np.float64)
        self.ns, self.f6 = self.o.fields_for(self.c64, f)
        self.tb = self.o.tables(self.f6)
        self.job = rbx.Job()
        self.job.set_geometry(self.g)
        self.job.set_model(dev(self.c32))

    def oracle_tables32(self):
        tb = self.tb
        return dict(T=tb.T.astype(np.float32), a=tb.a.astype(np.float32), gam=tb.gam.astype(np.float32),
                    K=tb.K.astype(np.uint8), exits=tb.exits.astype(np.float32))

    def inject(self):
        t = self.oracle_tables32()
        self.job.set_tables(dev(t["T"]), dev(t["a"]), dev(t["gam"]), dev(t["K"], torch.uint8), dev(t["exits"]))
        return {k: v.astype(np.float64) if k != "K" else v.astype(np.int32) for k, v in t.items()}


@pytest.fixture(scope="module")
def small(oracle_mod):
    return Case(oracle_mod, P.small_two_disc(), 2e5)


@pytest.fixture(scope="module")
def ragged(oracle_mod):
    # N not a multiple of any tile, non-square grid, ragged mask
    w = P.custom(50, 83, 1e-3, 36e-3, kind="discs", ny=77, freqs=(3e5,))
    return Case(oracle_mod, w, 3e5)


def check_tables(case):
    job, tb, o = case.job, case.tb, case.o
    job.trace_rays(case.f)
    gt = {k: v.cpu().numpy() for k, v in job.get_tables().items()}
    np.testing.assert_array_equal(job.mask_idx().cpu().numpy(), o.idx)
    cov_o = tb.cov.astype(bool)
    cov_g = gt["a"] > 0
    np.testing.assert_array_equal(cov_g, cov_o)
    assert cov_o.all()
    assert np.abs(gt["T"] - tb.T).max() <= 1e-9
    assert np.abs(gt["a"] / tb.a - 1).max() <= 1e-5
    assert np.abs(wrap(gt["gam"] - tb.gam)).max() <= 1e-5
    np.testing.assert_array_equal(gt["K"].astype(np.int32), tb.K)
    assert np.abs(gt["dg"] - tb.dg).max() <= 2e-5
    ex_g, ex_o = gt["exits"], tb.exits
    assert np.abs(wrap(ex_g[..., 0] - ex_o[..., 0])).max() <= 1e-5
    assert np.abs(ex_g[..., 1] - ex_o[..., 1]).max() <= 1e-9
    # exit amplitude: a ray meeting the ring at grazing angle pi j / N turns an FP32
    # position rounding dr (a few ulp of R) into an arc-length error dr / sin(pi j/N), so
    # a = s^-1/2 moves by dr / (2 s sin), s = 2 R sin(pi j/N)
    N = case.g.n_xducers
    j = np.arange(1, N)
    sn = np.sin(np.pi * j / N)
    dr = 8 * np.spacing(np.float32(case.g.ring_radius))
    tol = 1e-5 + dr / (4 * case.g.ring_radius * sn * sn)
    assert np.all(np.abs(ex_g[..., 2] / ex_o[..., 2] - 1) <= tol[None, :])
    np.testing.assert_array_equal(ex_g[..., 3], ex_o[..., 3])


def test_tables_parity_small(small):
    check_tables(small)


def test_tables_parity_ragged(ragged):
    check_tables(ragged)


def test_tables_deterministic(small):
    small.job.trace_rays(small.f)
    a = {k: v.cpu().numpy().copy() for k, v in small.job.get_tables().items()}
    small.job.trace_rays(small.f)
    b = {k: v.cpu().numpy() for k, v in small.job.get_tables().items()}
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_direct_green_identical_tables(which, request):
    case = request.getfixturevalue(which)
    t = case.inject()
    for f in (2e5, 4e5):
        g_gpu = case.job.direct_green(f).cpu().numpy()
        g_orc, _ = case.o.direct_green(f, t["exits"])
        assert rel_l2(g_gpu, g_orc) <= 1e-5
        assert np.all(np.diag(g_gpu) == 0)


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_direct_green_crossing_exits(which, request):
    """Exit angles perturbed so that neighbouring rays cross (as past a caustic), with runs of
    equal exit angles and, in some fans, a ray exiting just short of the transducer itself so
    that its pair straddles the angle wrap: the GPU's first bracketing pair per receiver and
    its interpolation match the oracle's linear scan over the pairs on the same exits."""
    case = request.getfixturevalue(which)
    t = case.oracle_tables32()
    N = case.g.n_xducers
    rng = np.random.default_rng(3)
    ex = t["exits"].copy()
    th = ex[..., 0].astype(np.float64) + rng.normal(0, 1.5 * 2 * math.pi / N, (N, N - 1))
    th[:, 5:8] = th[:, 5:6]
    for e in range(0, N, 4):
        th[e, rng.integers(2, N - 3)] = 2 * math.pi * e / N - 1e-4
    ex[..., 0] = np.angle(np.exp(1j * th)).astype(np.float32)
    case.job.set_tables(dev(t["T"]), dev(t["a"]), dev(t["gam"]), dev(t["K"], torch.uint8), dev(ex))
    for f in (2e5, 4e5):
        g_gpu = case.job.direct_green(f).cpu().numpy()
        g_orc, _ = case.o.direct_green(f, ex.astype(np.float64))
        assert rel_l2(g_gpu, g_orc) <= 1e-5
        assert np.abs(g_gpu - g_orc).max() <= 1e-4 * np.abs(g_orc).max()


@pytest.mark.parametrize("which", ["small", "ragged"])
def test_forward_identical_tables(which, request):
    case = request.getfixturevalue(which)
    t = case.inject()
    rng = np.random.default_rng(7)
    dm = (rng.standard_normal((case.g.ny, case.g.nx)) * 1e-9).astype(np.float32)
    f = case.f
    D_gpu = case.job.forward(f, dev(dm)).cpu().numpy()
    w = 2 * math.pi * f
    v = w * w * case.g.dx ** 2 * dm.astype(np.float64).ravel()[case.o.idx]
    D_orc = case.o.forward(f, t["T"], t["a"], t["K"], v)
    assert rel_l2(D_gpu, D_orc) <= 1e-5
    np.testing.assert_array_equal(D_gpu, D_gpu.T)


@pytest.mark.parametrize("which", ["small", "ragged"])
@pytest.mark.parametrize("weight_mode", [0, 1])
def test_adjoints_identical_tables(which, weight_mode, request, oracle_mod):
    case = request.getfixturevalue(which)
    job = rbx.Job()
    job.set_geometry(case.g, weight_mode=weight_mode)
    job.set_model(dev(case.c32))
    t = case.tb
    job.set_tables(dev(t.T.astype(np.float32)), dev(t.a.astype(np.float32)), dev(t.gam.astype(np.float32)),
                   dev(t.K.astype(np.uint8), torch.uint8), dev(t.exits.astype(np.float32)))
    T, a, gam = (x.astype(np.float32).astype(np.float64) for x in (t.T, t.a, t.gam))
    o = oracle_mod.Oracle(case.g, weight_mode=weight_mode)
    dg = o.dgamma(gam, t.cov)
    rng = np.random.default_rng(11)
    N = case.g.n_xducers
    R = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    f = case.f
    Rd = R.astype(np.complex128)
    plain_gpu = job.adjoint(f, dev(R, torch.complex64), False).cpu().numpy()
    plain_orc = o.adjoint_plain(f, T, a, t.K, Rd)
    assert rel_l2(plain_gpu, plain_orc) <= 1e-5
    pre_gpu = job.adjoint(f, dev(R, torch.complex64), True).cpu().numpy()
    pre_orc = o.backproject(f, T, a, gam, t.K, dg, Rd)
    assert rel_l2(pre_gpu, pre_orc) <= 1e-5
    job.close()


def oracle_update_on_tables(case, t, data, df):
    """Steps a5-a9 of the oracle on given (FP32-rounded) tables."""
    o, f = case.o, case.f
    gd, _ = o.direct_green(f, t["exits"])
    v = o.rough_v(f, case.c64, case.ns)
    D = o.forward(f, t["T"], t["a"], t["K"], v)
    R = gd + D - data
    np.fill_diagonal(R, 0)
    dg = o.dgamma(t["gam"], case.tb.cov)
    grad = o.backproject(f, t["T"], t["a"], t["gam"], t["K"], dg, R)
    c_out, st, bad = o.update(f, df, grad.real, case.c64)
    return c_out, float(np.sum(np.abs(R) ** 2))


def test_update_identical_tables_small(small):
    w, o, f, df = small.w, small.o, small.f, 1e5
    data, _ = o.predict(f, w.c_true)
    t = small.inject()
    c_ref, r2_ref = oracle_update_on_tables(small, t, data, df)
    small.job.set_model(dev(small.c32))
    st = small.job.update_from_tables(f, df, dev(data, torch.complex64))
    c_gpu = small.job.get_model().cpu().numpy().astype(np.float64)
    m = small.g.mask()
    dc_ref = c_ref[m] - small.c64[m]
    dc_gpu = c_gpu[m] - small.c64[m]
    assert abs(st["resid_norm2"] / r2_ref - 1) < 1e-4
    assert np.sqrt(np.mean((dc_gpu - dc_ref) ** 2)) <= 1e-3
    assert np.sqrt(np.mean(dc_ref ** 2)) > 0.05        # the update is not trivially small
    small.job.set_model(dev(small.c32))


def test_update_own_tables_small(small):
    """One full update (a1-a9) on each side from the same model: <= 0.05 m/s RMS."""
    w, o, f, df = small.w, small.o, small.f, 1e5
    data, _ = o.predict(f, w.c_true)
    c_ref, st_ref, bad = o.update_frequency(f, df, small.c64, data)
    assert bad == 0
    small.job.set_model(dev(small.c32))
    st = small.job.update_frequency(f, df, dev(data, torch.complex64))
    c_gpu = small.job.get_model().cpu().numpy().astype(np.float64)
    m = small.g.mask()
    assert np.sqrt(np.mean((c_gpu[m] - c_ref[m]) ** 2)) <= 0.05
    assert abs(st["rms_dc"] / st_ref[0] - 1) < 1e-2
    assert st["n_uncovered"] == 0 and st_ref[4] == 0
    assert np.all(c_gpu[~m] == np.float32(w.geom.c0))
    small.job.set_model(dev(small.c32))


def test_sweep_small(small):
    """Three-frequency sweep (Sec. 3.4) through rbx_reconstruct against sequential oracle updates."""
    w, o = small.w, small.o
    freqs = w.freqs
    data = np.stack([o.predict(f, w.c_true)[0] for f in freqs])
    data = P.add_noise(data, w.snr_db, seed=3)
    c = small.c64.copy()
    for f in freqs:
        c, st, bad = o.update_frequency(f, 1e5, c.astype(np.float32).astype(np.float64), data[list(freqs).index(f)])
    small.job.set_model(dev(small.c32))
    sts = small.job.reconstruct(freqs, dev(data, torch.complex64))
    c_gpu = small.job.get_model().cpu().numpy().astype(np.float64)
    m = small.g.mask()
    assert np.sqrt(np.mean((c_gpu[m] - c[m]) ** 2)) <= 0.05 * len(freqs)
    assert len(sts) == 3 and all(s["n_launches"] > 0 for s in sts)
    # the sweep moves the model towards the truth (relative error of Sec. 6.4 drops)
    re0 = np.linalg.norm((small.c64 - w.c_true)[m]) / np.linalg.norm((w.geom.c0 - w.c_true)[m])
    re1 = np.linalg.norm((c_gpu - w.c_true)[m]) / np.linalg.norm((w.geom.c0 - w.c_true)[m])
    assert re1 < re0
    small.job.set_model(dev(small.c32))


@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_uncovered_count_wide_mask(prec, oracle_mod):
    """Mask out to 0.97 R (ragged ring of 50): nodes next to each transducer between the
    tangent and its first ray stay uncovered. The count an update reports (the trace counts an
    entry when its first triangle writes it) equals the number of a = 0 entries the tables
    hold, and the covered sets of the CUDA path and the oracle agree but for entries within
    rounding of a ray-tube edge."""
    import dataclasses
    w = P.custom(50, 83, 1e-3, 36e-3, kind="discs", ny=77, freqs=(3e5,))
    g = dataclasses.replace(w.geom, mask_frac=0.97)
    o = oracle_mod.Oracle(g)
    c32 = w.c_init.astype(np.float32)
    ns, f6 = o.fields_for(c32.astype(np.float64), 3e5)
    tb = o.tables(f6)
    assert tb.uncovered > 100
    job = rbx.Job()
    job.set_geometry(g, precision=prec)
    job.set_model(dev(c32))
    data, _ = o.predict(3e5, w.c_true)
    st = job.update_frequency(3e5, 1e5, dev(data, torch.complex64))
    gt = job.get_tables()
    cov_g = gt["a"].cpu().numpy() > 0
    assert st["n_uncovered"] == int((~cov_g).sum())
    assert np.count_nonzero(cov_g != tb.cov.astype(bool)) <= 0.02 * tb.uncovered
    job.close()


def test_caustics_in_a_slow_lens(oracle_mod):
    """A strong slow Gaussian lens, c = 1500 / (1 + 0.25 exp(-r^2 / (8 mm)^2)), focuses the rays
    through it: the central rays of every fan pass a caustic before they reach the ring (the
    oracle's sign change of J is pinned against an independent ray integration in
    test_oracle_caustic.py). The caustic counts K of the CUDA path match the oracle's in the
    exit records and in the tables (first arrivals, so few table entries carry K = 1), and the
    travel times agree within the usual 1e-9 s."""
    g = P.Geometry(nx=96, ny=96, dx=1e-3, n_xducers=64, ring_radius=45e-3)
    X, Y = g.coords()
    c32 = (1500.0 / (1 + 0.25 * np.exp(-(X ** 2 + Y ** 2) / (8e-3) ** 2))).astype(np.float32)
    f = 1e6
    o = oracle_mod.Oracle(g)
    ns, f6 = o.fields_for(c32.astype(np.float64), f)
    tb = o.tables(f6)
    assert tb.bad_rays == 0 and (tb.exits[..., 3] > 0).sum() >= 64 and (tb.K > 0).sum() > 0
    job = rbx.Job()
    job.set_geometry(g)
    job.set_model(dev(c32))
    job.trace_rays(f)
    gt = {k: v.cpu().numpy() for k, v in job.get_tables().items()}
    np.testing.assert_array_equal(gt["exits"][..., 3], tb.exits[..., 3].astype(np.float32))
    cov = gt["a"] > 0
    np.testing.assert_array_equal(cov, tb.cov.astype(bool))
    np.testing.assert_array_equal(gt["K"].astype(np.int32)[cov], tb.K[cov])
    assert np.abs(gt["T"] - tb.T)[cov].max() <= 1e-9
    assert np.abs(gt["exits"][..., 1] - tb.exits[..., 1]).max() <= 1e-9
    job.close()


def test_fixed_point_gpu(small):
    """Data predicted by the GPU's own model give a zero residual and no update."""
    f = small.f
    small.job.set_model(dev(small.c32))
    small.job.trace_rays(f)
    data = small.job.predict(f)
    st = small.job.update_from_tables(f, 1e5, data)
    c_gpu = small.job.get_model().cpu().numpy()
    assert st["resid_norm2"] == 0.0
    np.testing.assert_array_equal(c_gpu[small.g.mask()], small.c32[small.g.mask()])
    small.job.set_model(dev(small.c32))


def test_errors_are_reported():
    g = P.Geometry(nx=40, ny=40, dx=1e-3, n_xducers=16, ring_radius=30e-3)   # ring outside the grid
    job = rbx.Job()
    with pytest.raises(rbx.RbxError) as e:
        job.set_geometry(g)
    assert e.value.status == 1
    g = P.Geometry(nx=64, ny=64, dx=1e-3, n_xducers=16, ring_radius=25e-3)
    job.set_geometry(g)
    with pytest.raises(rbx.RbxError) as e:
        job.forward(3e5, torch.zeros((64, 64), device="cuda"))
    assert e.value.status == 4                                                  # before trace_rays
    bad = torch.full((64, 64), 1500.0, device="cuda")
    bad[3, 5] = float("nan")
    with pytest.raises(rbx.RbxError) as e:
        job.set_model(bad)
    assert e.value.status == 5
    job.set_model(torch.full((64, 64), 1500.0, device="cuda"))
    data = torch.zeros((16, 16), dtype=torch.complex64, device="cuda")
    data[2, 3] = float("nan")
    with pytest.raises(rbx.RbxError) as e:
        job.update_frequency(3e5, 1e5, data)
    assert e.value.status == 5
    with pytest.raises(rbx.RbxError) as e:
        job.trace_rays(-1.0)
    assert e.value.status == 1
    job.close()
