"""Lossy, dispersive medium (Sec. 2.2, Szabo's power law) on the CUDA path against the FP64
oracle, with the tolerances of the lossless path: tables T <= 1e-9 s, a and gamma <= 1e-5;
forward / adjoint on identical tables relative L2 <= 1e-5 (FP32), 5e-3 (BF16), 2e-5 (split
BF16); one update <= 0.05 m/s RMS."""
import math

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu

Y = 1.4
TOL = {rbx.RBX_FP32: 1e-5, rbx.RBX_BF16: 5e-3, rbx.RBX_BF16X3: 2e-5}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def wrap(d):
    return np.angle(np.exp(1j * d))


def alpha0_map(g, db=0.8, floor_db=0.2):
    """alpha0 in Np (rad/s)^-y m^-1: a Gaussian bump of db dB/(cm MHz^y) on a floor inside the
    mask, water (0) outside."""
    X, Yc = g.coords()
    r2 = X ** 2 + Yc ** 2
    dbm = (floor_db + db * np.exp(-((X - 0.2 * g.ring_radius) ** 2 + Yc ** 2) / (2 * (0.25 * g.ring_radius) ** 2)))
    dbm = dbm * (r2 <= (0.7 * g.ring_radius) ** 2)
    np_m = dbm * 100.0 / (20.0 * math.log10(math.e))
    return (np_m / (2 * math.pi * 1e6) ** Y).astype(np.float32)


class LossyCase:
    def __init__(self, oracle_mod, w, f):
        self.w, self.g, self.f = w, w.geom, f
        self.o = oracle_mod.Oracle(self.g)
        self.c32 = w.c_init.astype(np.float32)
        self.c64 = self.c32.astype(np.float64)
        self.a32 = alpha0_map(self.g)
        self.a64 = self.a32.astype(np.float64)
        self.ns, self.f6, self.al = self.o.fields_for_abs(self.c64, self.a64, Y, f)
        self.tb = self.o.tables(self.f6, al=self.al)

    def job(self, prec=rbx.RBX_FP32):
        j = rbx.Job()
        j.set_geometry(self.g, precision=prec)
        j.set_model(dev(self.c32))
        j.set_absorption(dev(self.a32), Y)
        return j

    def inject(self, j):
        t = self.tb
        t32 = dict(T=t.T.astype(np.float32), a=t.a.astype(np.float32), gam=t.gam.astype(np.float32),
                   K=t.K.astype(np.uint8), exits=t.exits.astype(np.float32))
        j.set_tables(dev(t32["T"]), dev(t32["a"]), dev(t32["gam"]), dev(t32["K"], torch.uint8), dev(t32["exits"]))
        return {k: v.astype(np.float64) if k != "K" else v.astype(np.int32) for k, v in t32.items()}


@pytest.fixture(scope="module", params=["small", "ragged"])
def case(request, oracle_mod):
    if request.param == "small":
        return LossyCase(oracle_mod, P.small_two_disc(), 3e5)
    return LossyCase(oracle_mod, P.custom(50, 83, 1e-3, 36e-3, kind="discs", ny=77, freqs=(3e5,)), 3e5)


def test_lossy_tables(case):
    j = case.job()
    j.trace_rays(case.f)
    gt = {k: v.cpu().numpy() for k, v in j.get_tables().items()}
    tb = case.tb
    assert tb.uncovered == 0 and (gt["a"] > 0).all()
    assert np.abs(gt["T"] - tb.T).max() <= 1e-9
    assert np.abs(gt["a"] / tb.a - 1).max() <= 1e-5
    assert np.abs(wrap(gt["gam"] - tb.gam)).max() <= 1e-5
    np.testing.assert_array_equal(gt["K"].astype(np.int32), tb.K)
    # the absorption is visible in the tables: lossless amplitudes differ by far more
    o = case.o
    ns0, f60 = o.fields_for(case.c64, case.f)
    assert np.abs(o.tables(f60, fans=[0]).a[0] / tb.a[0] - 1).max() > 1e-2
    # exits with the lossless tolerances (the exit amplitude's FP32 floor at grazing angles
    # pi j / N: a position rounding dr moves a = s^-1/2 by dr / (4 R sin^2))
    ex_g, ex_o = gt["exits"], tb.exits
    assert np.abs(wrap(ex_g[..., 0] - ex_o[..., 0])).max() <= 1e-5
    assert np.abs(ex_g[..., 1] - ex_o[..., 1]).max() <= 1e-9
    N = case.g.n_xducers
    sn = np.sin(np.pi * np.arange(1, N) / N)
    tol = 1e-5 + 8 * np.spacing(np.float32(case.g.ring_radius)) / (4 * case.g.ring_radius * sn * sn)
    assert np.all(np.abs(ex_g[..., 2] / ex_o[..., 2] - 1) <= tol[None, :])
    np.testing.assert_array_equal(ex_g[..., 3], ex_o[..., 3])
    # direct Green's function from each side's own exits: within the exits' T and a bounds
    g_gpu = j.direct_green(case.f).cpu().numpy()
    g_orc, _ = o.direct_green(case.f, tb.exits)
    assert rel_l2(g_gpu, g_orc) <= 1e-5 + 2 * math.pi * case.f * 1e-9 + float(np.median(tol))
    j.close()


@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16, rbx.RBX_BF16X3])
def test_lossy_forward_identical_tables(case, prec):
    j = case.job(prec)
    t = case.inject(j)
    rng = np.random.default_rng(7)
    dm = (rng.standard_normal((case.g.ny, case.g.nx)) * 1e-9).astype(np.float32)
    D_gpu = j.forward(case.f, dev(dm)).cpu().numpy()
    idx = case.o.idx
    ups = case.o.upsilon(case.f, case.c64.ravel()[idx], case.a64.ravel()[idx], Y)
    v = ups * case.g.dx ** 2 * dm.astype(np.float64).ravel()[idx]
    D_orc = case.o.forward_c(case.f, t["T"], t["a"], t["K"], v)
    assert rel_l2(D_gpu, D_orc) <= TOL[prec]
    j.close()


def test_lossy_plain_adjoint_identical_tables(case):
    j = case.job()
    t = case.inject(j)
    rng = np.random.default_rng(11)
    N = case.g.n_xducers
    R = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    idx = case.o.idx
    ups = case.o.upsilon(case.f, case.c64.ravel()[idx], case.a64.ravel()[idx], Y)
    out_gpu = j.adjoint(case.f, dev(R, torch.complex64), False).cpu().numpy()
    out_orc = case.o.adjoint_plain_c(case.f, t["T"], t["a"], t["K"], ups, R.astype(np.complex128))
    assert rel_l2(out_gpu, out_orc) <= 1e-5
    j.close()


@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_lossy_update(case, prec):
    """One full update (a1-a9) on each side from the same lossy model: <= 0.05 m/s RMS."""
    w, o, f, df = case.w, case.o, case.f, 1e5
    data, _ = o.predict_abs(f, w.c_true, case.a64, Y)
    c_ref, st_ref, bad = o.update_frequency_abs(f, df, case.c64, case.a64, Y, data)
    assert bad == 0
    j = case.job(prec)
    st = j.update_frequency(f, df, dev(data, torch.complex64))
    c_gpu = j.get_model().cpu().numpy().astype(np.float64)
    m = case.g.mask()
    assert np.sqrt(np.mean((c_gpu[m] - c_ref[m]) ** 2)) <= 0.05
    assert np.sqrt(np.mean((c_ref[m] - case.c64[m]) ** 2)) > 0.05      # a real update
    assert st["n_uncovered"] == 0
    j.close()


def test_cleared_absorption_is_lossless(case):
    """rbx_set_absorption(NULL) returns the job to the lossless path, bit for bit."""
    f, df = case.f, 1e5
    data, _ = case.o.predict(f, case.w.c_true)
    j0 = rbx.Job()
    j0.set_geometry(case.g)
    j0.set_model(dev(case.c32))
    j0.update_frequency(f, df, dev(data, torch.complex64))
    j1 = case.job()
    j1.set_absorption(None)
    j1.update_frequency(f, df, dev(data, torch.complex64))
    np.testing.assert_array_equal(j1.get_model().cpu().numpy(), j0.get_model().cpu().numpy())
    j0.close()
    j1.close()


def test_absorption_argument_errors(case):
    j = rbx.Job()
    j.set_geometry(case.g)
    a = dev(case.a32)
    for y in (1.0, 0.0, 2.0, float("nan")):
        with pytest.raises(rbx.RbxError):
            j.set_absorption(a, y)
    bad = case.a32.copy()
    bad[3, 4] = -1.0
    with pytest.raises(rbx.RbxError):
        j.set_absorption(dev(bad), Y)
    j.close()
