"""BF16 and split-BF16 tensor-core paths (tcgen05) against the FP64 oracle.

Tolerance (stated for the method): forward / back-projection relative L2 <= 5e-3 for BF16 on identical
(oracle, FP32-rounded) tables; split BF16 (hi + lo, three products) keeps about 16 bits,
tested at 2e-5; one update <= 0.05 m/s RMS from the oracle's."""
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


class Case:
    def __init__(self, oracle_mod, w, f, weight_mode=0):
        self.w, self.g, self.f = w, w.geom, f
        self.o = oracle_mod.Oracle(self.g, weight_mode=weight_mode)
        self.c32 = w.c_init.astype(np.float32)
        self.c64 = self.c32.astype(np.float64)
        self.ns, self.f6 = self.o.fields_for(self.c64, f)
        self.tb = self.o.tables(self.f6)
        self.jobs = {}
        for prec in (rbx.RBX_FP32, rbx.RBX_BF16, rbx.RBX_BF16X3):
            j = rbx.Job()
            j.set_geometry(self.g, precision=prec, weight_mode=weight_mode)
            j.set_model(dev(self.c32))
            self.jobs[prec] = j
        t = self.tb
        self.t32 = dict(T=t.T.astype(np.float32), a=t.a.astype(np.float32), gam=t.gam.astype(np.float32),
                        K=t.K.astype(np.uint8), exits=t.exits.astype(np.float32))

    def inject(self, job):
        t = self.t32
        job.set_tables(dev(t["T"]), dev(t["a"]), dev(t["gam"]), dev(t["K"], torch.uint8), dev(t["exits"]))


@pytest.fixture(scope="module", params=["small", "ragged"])
def case(request, oracle_mod):
    if request.param == "small":
        return Case(oracle_mod, P.small_two_disc(), 3e5)
    return Case(oracle_mod, P.custom(50, 83, 1e-3, 36e-3, kind="discs", ny=77, freqs=(3e5,)), 3e5)


TOL = {rbx.RBX_BF16: 5e-3, rbx.RBX_BF16X3: 2e-5}


@pytest.mark.parametrize("prec", [rbx.RBX_BF16, rbx.RBX_BF16X3])
def test_bf16_forward_identical_tables(case, prec):
    job = case.jobs[prec]
    case.inject(job)
    rng = np.random.default_rng(7)
    dm = (rng.standard_normal((case.g.ny, case.g.nx)) * 1e-9).astype(np.float32)
    D = job.forward(case.f, dev(dm)).cpu().numpy()
    w = 2 * math.pi * case.f
    v = w * w * case.g.dx ** 2 * dm.astype(np.float64).ravel()[case.o.idx]
    t = case.t32
    D_orc = case.o.forward(case.f, t["T"].astype(np.float64), t["a"].astype(np.float64), t["K"].astype(np.int32), v)
    assert rel_l2(D, D_orc) <= TOL[prec]
    np.testing.assert_array_equal(D, D.T)


@pytest.mark.parametrize("prec", [rbx.RBX_BF16, rbx.RBX_BF16X3])
@pytest.mark.parametrize("weight_mode", [0, 1])
def test_bf16_backprojection_identical_tables(case, weight_mode, prec, oracle_mod):
    job = rbx.Job()
    job.set_geometry(case.g, precision=prec, weight_mode=weight_mode)
    job.set_model(dev(case.c32))
    case.inject(job)
    o = oracle_mod.Oracle(case.g, weight_mode=weight_mode)
    t = case.t32
    T, a, gam = (t[k].astype(np.float64) for k in ("T", "a", "gam"))
    dg = o.dgamma(gam, case.tb.cov)
    rng = np.random.default_rng(11)
    N = case.g.n_xducers
    R = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    out = job.adjoint(case.f, dev(R, torch.complex64), True).cpu().numpy()
    ref = o.backproject(case.f, T, a, gam, t["K"].astype(np.int32), dg, R.astype(np.complex128))
    assert rel_l2(out, ref) <= TOL[prec]
    job.close()


@pytest.mark.parametrize("prec", [rbx.RBX_BF16, rbx.RBX_BF16X3])
def test_bf16_update_matches_oracle(case, prec):
    w, o, f, df = case.w, case.o, case.f, 1e5
    data, _ = o.predict(f, w.c_true)
    c_ref, st_ref, bad = o.update_frequency(f, df, case.c64, data)
    job = case.jobs[prec]
    job.set_model(dev(case.c32))
    st = job.update_frequency(f, df, dev(data, torch.complex64))
    c_gpu = job.get_model().cpu().numpy().astype(np.float64)
    m = case.g.mask()
    assert np.sqrt(np.mean((c_gpu[m] - c_ref[m]) ** 2)) <= 0.05
    assert st["n_uncovered"] == 0


def test_bf16_and_fp32_paths_agree(case):
    """Same tables, same data: the BF16 and FP32 updates differ by far less than 0.05 m/s."""
    w, o, f = case.w, case.o, case.f
    data, _ = o.predict(f, w.c_true)
    out = {}
    for prec, job in case.jobs.items():
        case.inject(job)
        job.set_model(dev(case.c32))
        job.update_from_tables(f, 1e5, dev(data, torch.complex64))
        out[prec] = job.get_model().cpu().numpy().astype(np.float64)
    m = case.g.mask()
    dc = out[rbx.RBX_FP32][m] - case.c64[m]
    scale = max(1.0, np.sqrt(np.mean(dc ** 2)))
    d = out[rbx.RBX_BF16][m] - out[rbx.RBX_FP32][m]
    assert np.sqrt(np.mean(d ** 2)) <= 0.01 * scale
    d3 = out[rbx.RBX_BF16X3][m] - out[rbx.RBX_FP32][m]
    assert np.sqrt(np.mean(d3 ** 2)) <= 1e-3 * scale


def test_forward_split_autotuning():
    """The first job of a shape times the candidate K splits and keeps one; later jobs of the
    shape reuse it; the fixed heuristic gives the same forward within the BF16 rounding."""
    w = P.custom(72, 96, 0.9e-3, 38e-3, kind="discs", freqs=(3e5,))
    c = dev(w.c_init.astype(np.float32))
    prev = rbx.autotune(1)
    try:
        outs, tunings = [], []
        for mode in (1, 1, 0):
            rbx.autotune(mode)
            j = rbx.Job()
            j.set_geometry(w.geom, precision=rbx.RBX_BF16)
            j.set_model(c)
            j.trace_rays(3e5)
            dm = torch.full((w.geom.ny, w.geom.nx), 1e-9, device="cuda")
            outs.append(j.forward(3e5, dm).cpu().numpy())
            tunings.append(j.tuning())
            j.close()
        assert tunings[0]["candidates_timed"] >= 2 and tunings[1]["candidates_timed"] == 0
        assert tunings[0]["fwd_splits"] == tunings[1]["fwd_splits"] >= 1
        np.testing.assert_array_equal(outs[0], outs[1])
        assert rel_l2(outs[2], outs[0]) <= 1e-5
    finally:
        rbx.autotune(prev)


def holes_of(N, X, seed=5):
    """Seeded uncovered entries: 3 % at random plus a quarter of the nodes of transducers on
    both sides of every 32-transducer tile border and of the ring's wrap (0 and N - 1)."""
    rng = np.random.default_rng(seed)
    hole = rng.random((N, X)) < 0.03
    rows = {0, N - 1} | {e for b in range(32, N, 32) for e in (b - 1, b)}
    for e in rows:
        hole[e, rng.choice(X, X // 4, replace=False)] = True
    return hole


@pytest.mark.parametrize("prec", [rbx.RBX_BF16, rbx.RBX_BF16X3])
def test_backprojection_tables_with_holes(case, prec, oracle_mod):
    """Uncovered entries (a = 0) zero the angular density of both neighbouring transducers
    (step a4). The tensor-core operand synthesis forms that density itself inside
    32-transducer tiles with one halo row on each side, wrapping around the ring, so holes sit
    on tile borders and at the wrap. The back-projection matches the oracle's with the same
    holes, the FP32 path's angular density array (rbx_get_tables) is the oracle's, and an
    update reports exactly the injected number of uncovered entries."""
    t = case.t32
    assert case.tb.cov.all()
    N, X = t["a"].shape
    hole = holes_of(N, X)
    a = np.where(hole, np.float32(0), t["a"])
    o = oracle_mod.Oracle(case.g)
    T, a64, gam = t["T"].astype(np.float64), a.astype(np.float64), t["gam"].astype(np.float64)
    dg = o.dgamma(gam, (~hole).astype(np.int32))
    assert (dg == 0).sum() > hole.sum()                     # holes also zero their neighbours
    rng = np.random.default_rng(11)
    R = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    ref = o.backproject(case.f, T, a64, gam, t["K"].astype(np.int32), dg, R.astype(np.complex128))
    data, _ = o.predict(case.f, case.w.c_true)
    for p in (prec, rbx.RBX_FP32):
        job = rbx.Job()
        job.set_geometry(case.g, precision=p)
        job.set_model(dev(case.c32))
        job.set_tables(dev(t["T"]), dev(a), dev(t["gam"]), dev(t["K"], torch.uint8), dev(t["exits"]))
        out = job.adjoint(case.f, dev(R, torch.complex64), True).cpu().numpy()
        assert rel_l2(out, ref) <= (TOL[p] if p != rbx.RBX_FP32 else 1e-5)
        dg_gpu = job.get_tables()["dg"].cpu().numpy()
        assert np.abs(dg_gpu - dg).max() <= 2e-5
        np.testing.assert_array_equal(dg_gpu == 0, dg == 0)
        st = job.update_from_tables(case.f, 1e5, dev(data, torch.complex64))
        assert st["n_uncovered"] == int(hole.sum())
        job.close()


@pytest.mark.parametrize("prec", [rbx.RBX_BF16, rbx.RBX_BF16X3])
def test_update_synthesis_matches_forward_bits(case, prec):
    """Data the job predicts on its own model leave a residual of exactly zero in an update:
    the update's single synthesis pass (both contractions' operands) writes forward planes
    bit-identical to those of the forward's own pass."""
    job = case.jobs[prec]
    job.set_model(dev(case.c32))
    job.trace_rays(case.f)
    data = job.predict(case.f)
    st = job.update_from_tables(case.f, 1e5, data)
    assert st["resid_norm2"] == 0.0
    job.set_model(dev(case.c32))


@pytest.mark.parametrize("N,nx", [(72, 96), (300, 160)])
def test_fused_synthesis_forward_is_bit_identical(N, nx, oracle_mod):
    """The fused-synthesis forward (operand tiles formed from the tables inside the
    contraction, the tuner's candidate) against the separate synthesis pass plus TMA-fed
    planes, at the same heuristic split: the same BF16 operands, so the same D bit for bit,
    and the same update, on rings that fill their 128-row tiles raggedly (72, 300). A job of a
    new shape under the default tuning times both forms and keeps the faster."""
    w = P.custom(N, nx, 0.9e-3, (nx - 1) * 0.9e-3 / 2 - 3e-3, kind="discs", freqs=(3e5,))
    c32 = w.c_init.astype(np.float32)
    f = 3e5
    prev = rbx.autotune(1)
    try:
        outs, ups, tun = [], [], []
        data, _ = oracle_mod.Oracle(w.geom).predict(f, w.c_true)
        for mode in (0, 2):
            rbx.autotune(mode)
            j = rbx.Job()
            j.set_geometry(w.geom, precision=rbx.RBX_BF16)
            j.set_model(dev(c32))
            j.trace_rays(f)
            rng = np.random.default_rng(4)
            dm = dev((rng.standard_normal((w.geom.ny, w.geom.nx)) * 1e-9).astype(np.float32))
            outs.append(j.forward(f, dm).cpu().numpy())
            tun.append(j.tuning())
            j.update_frequency(f, 1e5, dev(data, torch.complex64))
            ups.append(j.get_model().cpu().numpy())
            j.close()
        assert not tun[0]["fused_forward"] and tun[1]["fused_forward"]
        np.testing.assert_array_equal(outs[1], outs[0])
        np.testing.assert_array_equal(ups[1], ups[0])
        rbx.autotune(1)
        j = rbx.Job()
        j.set_geometry(P.custom(N + 1, nx, 0.9e-3, (nx - 1) * 0.9e-3 / 2 - 3e-3).geom, precision=rbx.RBX_BF16)
        t = j.tuning()
        j.close()
        assert t["ms_synth_both"] > 0 and t["ms_forward_gemm"] > 0 and t["ms_synth_bp"] > 0 and t["ms_forward_fused"] > 0
        assert t["fused_forward"] == (t["ms_synth_bp"] + t["ms_forward_fused"] < t["ms_synth_both"] + t["ms_forward_gemm"])
    finally:
        rbx.autotune(prev)
