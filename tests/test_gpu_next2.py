"""Frequency sets and integration on the non-smoothed map (Sec. 6.3.2) on the CUDA path
against the FP64 oracle: tables T <= 1e-9 s, a and gamma <= 1e-5 (as for the default mode);
one set update <= 0.05 m/s RMS in FP32 and BF16."""
import math

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def wrap(d):
    return np.angle(np.exp(1j * d))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module", params=["small", "ragged"])
def work(request):
    if request.param == "small":
        return P.small_two_disc()
    return P.custom(50, 83, 1e-3, 36e-3, kind="discs", ny=77, freqs=(3e5, 3.5e5))


def job_for(w, prec=rbx.RBX_FP32, raw=True):
    j = rbx.Job()
    j.set_geometry(w.geom, precision=prec)
    j.set_model(dev(w.c_init.astype(np.float32)))
    if raw:
        j.set_integration(True)
    return j


def test_raw_tables(work, oracle_mod):
    """Travel times and amplitudes integrated on the non-smoothed map, rays on the smoothed one."""
    o = oracle_mod.Oracle(work.geom)
    c64 = work.c_init.astype(np.float32).astype(np.float64)
    f = float(work.freqs[0])
    ns, f6 = o.fields_for(c64, f)
    tb = o.tables(f6, nr=1.0 / c64)
    j = job_for(work)
    j.trace_rays(f)
    gt = {k: v.cpu().numpy() for k, v in j.get_tables().items()}
    assert tb.uncovered == 0 and (gt["a"] > 0).all()
    assert np.abs(gt["T"] - tb.T).max() <= 1e-9
    assert np.abs(gt["a"] / tb.a - 1).max() <= 1e-5
    assert np.abs(wrap(gt["gam"] - tb.gam)).max() <= 1e-5
    np.testing.assert_array_equal(gt["K"].astype(np.int32), tb.K)
    assert np.abs(gt["exits"][..., 1] - tb.exits[..., 1]).max() <= 1e-9
    # the non-smoothed integration is visible: the smoothed tables differ by far more
    ts = o.tables(f6, fans=[0])
    assert np.abs(ts.T[0] - tb.T[0]).max() > 10 * 1e-9
    j.close()


def test_raw_predict_is_direct_green(work, oracle_mod):
    o = oracle_mod.Oracle(work.geom)
    f = float(work.freqs[0])
    j = job_for(work)
    j.set_model(dev(work.c_true.astype(np.float32)))
    j.trace_rays(f)
    g_gpu = j.predict(f).cpu().numpy()
    g_orc, _ = o.predict_ext(f, work.c_true.astype(np.float32).astype(np.float64), raw=True)
    assert rel_l2(g_gpu, g_orc) <= 1e-3          # own exits: within the exits' T bound (omega 1e-9 s)
    j.close()


@pytest.mark.parametrize("raw", [False, True])
@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_two_frequency_set_update(work, oracle_mod, raw, prec):
    """One update from two consecutive frequencies on each side, same model: <= 0.05 m/s RMS."""
    o = oracle_mod.Oracle(work.geom)
    freqs = [float(work.freqs[0]), float(work.freqs[0]) + 5e4]
    df = 5e4
    c_t = work.c_true.astype(np.float32).astype(np.float64)
    c64 = work.c_init.astype(np.float32).astype(np.float64)
    data = np.stack([o.predict_ext(f, c_t, raw=raw)[0] for f in freqs])
    c_ref, st_ref, bad = o.update_set(freqs, df, c64, data, raw=raw)
    assert bad == 0
    j = job_for(work, prec, raw)
    st = j.update_set(freqs, df, dev(data, torch.complex64))
    c_gpu = j.get_model().cpu().numpy().astype(np.float64)
    m = work.geom.mask()
    assert np.sqrt(np.mean((c_gpu[m] - c_ref[m]) ** 2)) <= 0.05
    assert np.sqrt(np.mean((c_ref[m] - c64[m]) ** 2)) > 0.02         # a real update
    assert abs(st["resid_norm2"] / st_ref[3] - 1) < 2e-2
    j.close()


def test_set_of_one_is_update_frequency(work):
    f, df = float(work.freqs[0]), 1e5
    data = dev(np.zeros((1, work.geom.n_xducers, work.geom.n_xducers)), torch.complex64)
    a, b = job_for(work, raw=False), job_for(work, raw=False)
    a.update_frequency(f, df, data[0])
    b.update_set([f], df, data)
    np.testing.assert_array_equal(a.get_model().cpu().numpy(), b.get_model().cpu().numpy())
    a.close()
    b.close()


def test_set_argument_errors(work):
    j = job_for(work)
    N = work.geom.n_xducers
    data = dev(np.zeros((2, N, N)), torch.complex64)
    with pytest.raises(rbx.RbxError):
        j.update_set([3e5, float("nan")], 1e5, data)
    assert j.L.rbx_set_integration(j.h, 2) == 1          # RBX_EINVAL
    j.close()


def test_linked_direct_green_water(oracle_mod):
    """In water the linked rays are the chords: g = App. B's g0 (and the fan already links)."""
    w = P.custom(64, 96, 1e-3, 45e-3, kind="water", freqs=(3e5,))
    j = rbx.Job()
    j.set_geometry(w.geom)
    j.set_model(dev(np.full((96, 96), 1500.0, np.float32)))
    j.set_linking(6)
    j.trace_rays(3e5)
    g = j.direct_green(3e5).cpu().numpy()
    N = 64
    k = 2 * math.pi * 3e5 / 1500.0
    b = 2 * math.pi * np.arange(N) / N
    xy = 45e-3 * np.stack([np.cos(b), np.sin(b)], 1)
    s = np.linalg.norm(xy[:, None, :] - xy[None, :, :], axis=-1)
    off = ~np.eye(N, dtype=bool)
    ref = (8 * math.pi * k * s[off]) ** -0.5 * np.exp(1j * (k * s[off] + math.pi / 4))
    assert rel_l2(g[off], ref) <= 1e-4          # own FP32 rays (T to ~1e-11 s, grazing a floor)
    j.close()


@pytest.mark.parametrize("raw", [False, True])
def test_linked_direct_green_parity(work, oracle_mod, raw):
    """Secant-linked direct Green's function against the oracle's, on each side's own rays."""
    o = oracle_mod.Oracle(work.geom)
    f = float(work.freqs[0])
    c_t = work.c_true.astype(np.float32).astype(np.float64)
    j = job_for(work, raw=raw)
    j.set_linking(8)
    j.set_model(dev(c_t.astype(np.float32)))
    j.trace_rays(f)
    g_gpu = j.direct_green(f).cpu().numpy()
    ns, f6 = o.fields_for(c_t, f)
    tb = o.tables(f6, nr=(1.0 / c_t) if raw else None)
    g_orc, cl, unc, Tl = o.direct_green_linked(f, f6, tb.exits, nr=(1.0 / c_t) if raw else None)
    assert unc == 0
    assert rel_l2(g_gpu, g_orc) <= 1e-4
    j.close()


def test_linked_set_update(work, oracle_mod):
    """One two-frequency update with linked rays and the non-smoothed integration (the paper's
    configuration) on each side: <= 0.05 m/s RMS."""
    o = oracle_mod.Oracle(work.geom)
    freqs = [float(work.freqs[0]), float(work.freqs[0]) + 5e4]
    c_t = work.c_true.astype(np.float32).astype(np.float64)
    c64 = work.c_init.astype(np.float32).astype(np.float64)
    data = np.stack([o.predict_ext(f, c_t, raw=True, link=True)[0] for f in freqs])
    c_ref, st_ref, bad = o.update_set(freqs, 5e4, c64, data, raw=True, link=True)
    assert bad == 0
    j = job_for(work, rbx.RBX_BF16, raw=True)
    j.set_linking(8)
    j.update_set(freqs, 5e4, dev(data, torch.complex64))
    c_gpu = j.get_model().cpu().numpy().astype(np.float64)
    m = work.geom.mask()
    assert np.sqrt(np.mean((c_gpu[m] - c_ref[m]) ** 2)) <= 0.05
    j.close()
