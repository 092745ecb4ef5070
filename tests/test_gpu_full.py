"""Full-size parity: the 1024-transducer, 512x512 workload that bench.py times (same library
calls, same launch configuration), compared with the oracle on sampled outputs it can
compute one by one; and one full update of the 256-transducer, 288x288 workload.
"""
import math

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def wrap(d):
    return np.angle(np.exp(1j * d))


@pytest.fixture(scope="module")
def big(oracle_mod):
    w = P.precision_ring1024()
    f = float(w.freqs[7])                      # 0.505 MHz
    o = oracle_mod.Oracle(w.geom)
    c32 = w.c_init.astype(np.float32)
    ns, f6 = o.fields_for(c32.astype(np.float64), f)
    return w, f, o, c32, ns, f6


def test_full_size_tables_sampled_fans(big):
    w, f, o, c32, ns, f6 = big
    N = w.geom.n_xducers
    fans = np.array([0, 1, 2, 255, 511, 512, 513, 767, 1022, 1023], np.int32)
    tb = o.tables(f6, fans=fans)
    assert tb.uncovered == 0 and tb.bad_rays == 0
    job = rbx.Job()
    job.set_geometry(w.geom, precision=rbx.RBX_BF16)
    job.set_model(dev(c32))
    job.trace_rays(f)
    gt = job.get_tables()
    T = gt["T"][fans.tolist()].cpu().numpy()
    a = gt["a"][fans.tolist()].cpu().numpy()
    gam = gt["gam"][fans.tolist()].cpu().numpy()
    K = gt["K"][fans.tolist()].cpu().numpy()
    assert np.all(a > 0)
    assert np.abs(T - tb.T).max() <= 1e-9
    assert np.abs(a / tb.a - 1).max() <= 1e-5
    assert np.abs(wrap(gam - tb.gam)).max() <= 1e-5
    np.testing.assert_array_equal(K.astype(np.int32), tb.K)
    # angular density of fans 1 and 512 from their neighbours' angles
    dg = gt["dg"][[1, 512]].cpu().numpy()
    for q, e in ((0, 1), (1, 512)):
        i = {int(v): k for k, v in enumerate(fans)}
        d = tb.gam[i[e + 1]] - tb.gam[i[e - 1]]
        ref = np.abs(wrap(d)) / 2
        assert np.abs(dg[q] - ref).max() <= 2e-5
    ex = gt["exits"][fans.tolist()].cpu().numpy()
    assert np.abs(ex[..., 1] - tb.exits[..., 1]).max() <= 1e-9
    job.close()


@pytest.fixture(scope="module")
def big_tables(big, oracle_mod):
    """Oracle tables of all 1024 fans, rounded to FP32 (built in chunks of 64 fans)."""
    w, f, o, c32, ns, f6 = big
    N, X = o.N, o.X
    T = np.zeros((N, X), np.float32); a = np.zeros_like(T); gam = np.zeros_like(T)
    K = np.zeros((N, X), np.uint8); cov = np.zeros((N, X), np.int32)
    exits = np.zeros((N, N - 1, 4), np.float32)
    for e0 in range(0, N, 64):
        fans = np.arange(e0, min(N, e0 + 64), dtype=np.int32)
        tb = o.tables(f6, fans=fans)
        sl = slice(e0, e0 + len(fans))
        T[sl], a[sl], gam[sl] = tb.T, tb.a, tb.gam
        K[sl], cov[sl], exits[sl] = tb.K, tb.cov, tb.exits
    return dict(T=T, a=a, gam=gam, K=K, cov=cov, exits=exits)


@pytest.fixture(scope="module")
def big_forward(big, big_tables, oracle_mod):
    """The oracle's Born forward of a random perturbation over all N x N pairs, on the
    FP32-rounded oracle tables (about a minute on 16 cores)."""
    w, f, o, c32, ns, f6 = big
    t = big_tables
    rng = np.random.default_rng(3)
    dm = (rng.standard_normal((w.geom.ny, w.geom.nx)) * 1e-9).astype(np.float32)
    om = 2 * math.pi * f
    v = om * om * w.geom.dx ** 2 * dm.astype(np.float64).ravel()[o.idx]
    D = oracle_mod.forward_rows(o, f, t["T"].astype(np.float64), t["a"].astype(np.float64), t["K"].astype(np.int32), v)
    return dm, D


@pytest.mark.parametrize("prec,tol", [(rbx.RBX_FP32, 1e-5), (rbx.RBX_BF16, 5e-3), (rbx.RBX_BF16X3, 2e-5)])
def test_full_size_contractions_identical_tables(big, big_tables, big_forward, prec, tol, oracle_mod):
    w, f, o, c32, ns, f6 = big
    t = big_tables
    N, X = o.N, o.X
    job = rbx.Job()
    job.set_geometry(w.geom, precision=prec)
    job.set_model(dev(c32))
    job.set_tables(dev(t["T"]), dev(t["a"]), dev(t["gam"]), dev(t["K"], torch.uint8), dev(t["exits"]))
    rng = np.random.default_rng(3)
    rng.standard_normal((w.geom.ny, w.geom.nx))          # the draw of the perturbation in big_forward
    dm, Dref = big_forward
    D = job.forward(f, dev(dm)).cpu().numpy()
    # every (e, r) pair, and every row on its own (no row may be off even if the total is fine)
    assert rel_l2(D, Dref) <= tol
    row_err = np.linalg.norm(D - Dref, axis=1) / np.linalg.norm(Dref, axis=1)
    assert row_err.max() <= 3 * tol, (int(row_err.argmax()), float(row_err.max()))
    np.testing.assert_array_equal(D, D.T)                 # D = D^T exactly (upper tiles mirrored)
    # preconditioned back-projection at sampled mask nodes
    R = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    out = job.adjoint(f, dev(R, torch.complex64), True).cpu().numpy()
    nodes = np.linspace(0, X - 1, 48).astype(np.int64)
    sub = {k: t[k][:, nodes] for k in ("T", "a", "gam", "K", "cov")}
    og = oracle_mod.Oracle(w.geom)
    og.X = len(nodes)
    dgn = og.dgamma(sub["gam"].astype(np.float64), sub["cov"])
    ref = oracle_mod.backproject_nodes(og, f, sub["T"].astype(np.float64), sub["a"].astype(np.float64),
                                       sub["gam"].astype(np.float64), sub["K"].astype(np.int32), dgn,
                                       R.astype(np.complex128))
    assert rel_l2(out[nodes], ref) <= tol
    job.close()


@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_ring256_full_update(prec, oracle_mod):
    """One full update (a1-a9) of the 256-transducer workload on both sides: <= 0.05 m/s RMS."""
    w = P.fp32_ring256()
    f, df = float(w.freqs[3]), w.dfreq
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
    m = w.geom.mask()
    assert np.sqrt(np.mean((c[m] - c_ref[m]) ** 2)) <= 0.05
    assert np.sqrt(np.mean((c_ref[m] - c32[m]) ** 2)) > 0.05          # a real update happened
    assert st["n_uncovered"] == 0
    job.close()


@pytest.mark.parametrize("seed", [7, 5, 21, 8])
def test_batched_slices_spot_check(seed, oracle_mod):
    """Slices of the uneven batch (sizes drawn from N in {256,512,768,1024}, grids 192-512 at
    0.45-1.0 mm): one update at the lowest and at the highest frequency of the sweep from the
    initial model, FP32 and BF16 contractions against the oracle, <= 0.05 m/s RMS."""
    w = P.batched_slice(seed)
    o = oracle_mod.Oracle(w.geom)
    m = w.geom.mask()
    c32 = w.c_init.astype(np.float32)
    for q in (0, len(w.freqs) - 1):
        f, df = float(w.freqs[q]), w.dfreq
        data, _ = o.predict(f, w.c_true)
        c_ref, _, bad = o.update_frequency(f, df, c32.astype(np.float64), data)
        assert bad == 0
        for prec in (rbx.RBX_FP32, rbx.RBX_BF16):
            job = rbx.Job()
            job.set_geometry(w.geom, precision=prec)
            job.set_model(dev(c32))
            st = job.update_frequency(f, df, dev(data, torch.complex64))
            c = job.get_model().cpu().numpy().astype(np.float64)
            job.close()
            assert st["n_uncovered"] == 0
            assert np.sqrt(np.mean((c[m] - c_ref[m]) ** 2)) <= 0.05, (seed, f, prec)
