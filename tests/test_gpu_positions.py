"""Transducers placed by the caller on the ring (rbx_set_geometry's xducer_xy; Sec. 2.1 states
the problem for elements at given positions): the CUDA path against the FP64 oracle with the
same positions. Tolerances as in test_gpu_parity_small.py."""
import math

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx
from test_gpu_parity_small import Case, check_tables, dev, rel_l2

pytestmark = pytest.mark.gpu


def jittered_workload(N=48, seed=2):
    w = P.custom(N, 96, 1e-3, 45e-3, kind="discs", freqs=(3e5,))
    w.geom.xducer_xy = P.jittered_ring(N, 45e-3, 0.35, seed=seed)
    return w


@pytest.fixture(scope="module")
def jit(oracle_mod):
    return Case(oracle_mod, jittered_workload(), 3e5)


def test_positions_tables_parity(jit):
    check_tables(jit)


def test_positions_direct_green_identical_exits(jit):
    t = jit.inject()
    for f in (2e5, 4e5):
        g_gpu = jit.job.direct_green(f).cpu().numpy()
        g_orc, clamped = jit.o.direct_green(f, t["exits"])
        assert clamped > 0                   # receivers within 2 pi / N of their emitter
        assert rel_l2(g_gpu, g_orc) <= 1e-5
        assert np.all(np.diag(g_gpu) == 0)


@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_positions_full_update(prec, oracle_mod):
    w = jittered_workload(seed=5)
    f, df = 3e5, 1e5
    o = oracle_mod.Oracle(w.geom)
    data, _ = o.predict(f, w.c_true)
    c32 = w.c_init.astype(np.float32)
    c_ref, st_ref, bad = o.update_frequency(f, df, c32.astype(np.float64), data)
    assert bad == 0
    job = rbx.Job()
    job.set_geometry(w.geom, precision=prec)
    job.set_model(dev(c32))
    st = job.update_frequency(f, df, dev(data, torch.complex64))
    c = job.get_model().cpu().numpy().astype(np.float64)
    job.close()
    m = w.geom.mask()
    assert np.sqrt(np.mean((c_ref[m] - c32[m]) ** 2)) > 0.05          # a real update
    assert np.sqrt(np.mean((c[m] - c_ref[m]) ** 2)) <= 0.05
    assert st["n_clamped"] > 0


def test_positions_linked_direct_green(oracle_mod):
    w = jittered_workload(seed=7)
    f = 3e5
    c_t = w.c_true.astype(np.float32).astype(np.float64)
    o = oracle_mod.Oracle(w.geom)
    job = rbx.Job()
    job.set_geometry(w.geom)
    job.set_linking(8)
    job.set_model(dev(c_t.astype(np.float32)))
    job.trace_rays(f)
    g_gpu = job.direct_green(f).cpu().numpy()
    job.close()
    ns, f6 = o.fields_for(c_t, f)
    tb = o.tables(f6)
    g_orc, cl, unc, _ = o.direct_green_linked(f, f6, tb.exits)
    assert unc == 0
    assert rel_l2(g_gpu, g_orc) <= 1e-4


def test_uniform_positions_given_explicitly_match_the_default(oracle_mod):
    w = P.custom(40, 96, 1e-3, 45e-3, kind="discs", freqs=(3e5,))
    th = 2 * np.pi * np.arange(40) / 40
    out = []
    for xy in (None, np.stack([np.cos(th), np.sin(th)], 1) * 45e-3):
        w.geom.xducer_xy = xy
        job = rbx.Job()
        job.set_geometry(w.geom)
        job.set_model(dev(w.c_init.astype(np.float32)))
        job.trace_rays(3e5)
        t = {k: v.cpu().numpy() for k, v in job.get_tables().items()}
        out.append((t, job.direct_green(3e5).cpu().numpy()))
        job.close()
    (t0, g0), (t1, g1) = out
    assert np.abs(t0["T"] - t1["T"]).max() <= 1e-10
    assert rel_l2(g1, g0) <= 1e-5          # receivers e +/- 1 sit exactly on the ends of the fan


@pytest.mark.parametrize("bad", ["off_ring", "reversed", "duplicate"])
def test_positions_rejected(bad):
    N, R = 24, 45e-3
    th = 2 * np.pi * np.arange(N) / N
    xy = np.stack([np.cos(th), np.sin(th)], 1) * R
    if bad == "off_ring":
        xy[3] *= 1.01
    elif bad == "reversed":
        xy = xy[::-1].copy()
    else:
        xy[5] = xy[4]
    g = P.Geometry(nx=96, ny=96, dx=1e-3, n_xducers=N, ring_radius=R, xducer_xy=xy)
    job = rbx.Job()
    with pytest.raises(rbx.RbxError) as e:
        job.set_geometry(g)
    assert e.value.status == 1
    job.close()
