"""Served form: requests of different sizes admitted under an HBM budget and run concurrently
(continuous batching). Each result must be the same alone and in the mix; failures stay with
their own request."""
import time

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


def requests():
    return [P.small_two_disc(),
            P.custom(50, 83, 1e-3, 36e-3, kind="discs", ny=77, freqs=(2e5, 3e5, 4e5)),
            P.custom(96, 120, 0.8e-3, 40e-3, kind="breast", seed=3, freqs=(2e5, 3e5, 4e5)),
            P.custom(128, 112, 0.9e-3, 44e-3, kind="breast", seed=4, freqs=(2e5, 3e5, 4e5))]


def make_data(w, precision=rbx.RBX_BF16):
    j = rbx.Job()
    j.set_geometry(w.geom, precision=precision)
    j.set_model(torch.tensor(w.c_true, dtype=torch.float32, device="cuda"))
    d = []
    for f in w.freqs:
        j.trace_rays(float(f))
        d.append(j.predict(float(f)).cpu().numpy())
    j.close()
    return P.add_noise(np.stack(d), 40.0, seed=11)


def alone(w, data, precision=rbx.RBX_BF16):
    j = rbx.Job()
    j.set_geometry(w.geom, precision=precision)
    j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
    j.reconstruct(w.freqs, torch.tensor(data, dtype=torch.complex64, device="cuda"))
    c = j.get_model().cpu().numpy()
    j.close()
    return c


@pytest.fixture(scope="module")
def cases():
    ws = requests()
    datas = [make_data(w) for w in ws]
    refs = [alone(w, d) for w, d in zip(ws, datas)]
    return ws, datas, refs


def test_results_same_alone_and_in_mix(cases):
    ws, datas, refs = cases
    srv = rbx.Server(hbm_budget_bytes=150 << 30, max_inflight=8)
    tickets = [srv.submit(w.geom, w.c_init, w.freqs, d) for w, d in zip(ws, datas)]
    for t in tickets:
        assert srv.wait(t, 300.0) == 0
    for w, t, ref in zip(ws, tickets, refs):
        r = srv.poll(t, want_model=True, shape=(w.geom.ny, w.geom.nx))
        assert r["state"] == rbx.REQ_DONE and r["status"] == 0
        assert r["latency_s"] > 0
        np.testing.assert_array_equal(r["model"], ref)
        assert r["last"]["rms_dc"] > 0
    srv.close()


def test_admission_under_a_small_budget(cases):
    ws, datas, refs = cases
    # room for the first two requests together but not for the third beside either of them:
    # the third waits until one of the first two has ended, and all three still finish
    est = [rbx.estimate_bytes(w.geom, len(w.freqs)) for w in ws[:3]]
    assert est[0] + est[1] < est[2] + min(est[0], est[1])
    budget = est[0] + est[1]
    srv = rbx.Server(hbm_budget_bytes=budget, max_inflight=8)
    tickets = [srv.submit(w.geom, w.c_init, w.freqs, d) for w, d in zip(ws[:3], datas[:3])]
    big = P.precision_ring1024()
    nn = big.geom.n_xducers
    t_big = srv.submit(big.geom, big.c_init, big.freqs[:1], np.zeros((1, nn, nn), np.complex64))
    for _ in range(2000):
        assert srv.info()["bytes_in_use"] <= budget
        if all(srv.poll(t)["state"] >= rbx.REQ_DONE for t in tickets + [t_big]):
            break
        time.sleep(0.005)
    for w, t, ref in zip(ws, tickets, refs):
        assert srv.wait(t, 300.0) == 0
        np.testing.assert_array_equal(srv.poll(t, True, (w.geom.ny, w.geom.nx))["model"], ref)
    assert srv.wait(t_big, 60.0) == 2                       # RBX_ENOMEM: above the whole budget
    assert srv.poll(t_big)["state"] == rbx.REQ_FAILED
    tm = [srv.times(t) for t in tickets]
    assert tm[2]["start"] >= min(tm[0]["end"], tm[1]["end"])
    assert all(0 <= x["submit"] <= x["start"] <= x["end"] for x in tm)
    assert srv.times(t_big)["start"] == -1.0
    srv.close()


def test_failure_stays_with_its_request(cases):
    ws, datas, refs = cases
    srv = rbx.Server(hbm_budget_bytes=150 << 30, max_inflight=8)
    bad = datas[1].copy()
    bad[1, 3, 7] = np.nan
    t_bad = srv.submit(ws[1].geom, ws[1].c_init, ws[1].freqs, bad)
    t_ok = [srv.submit(w.geom, w.c_init, w.freqs, d) for w, d in ((ws[0], datas[0]), (ws[2], datas[2]))]
    assert srv.wait(t_bad, 300.0) == 5                      # RBX_ENUMERIC
    assert "non-finite" in srv.poll(t_bad)["error"]
    for t, w, ref in zip(t_ok, (ws[0], ws[2]), (refs[0], refs[2])):
        assert srv.wait(t, 300.0) == 0
        np.testing.assert_array_equal(srv.poll(t, True, (w.geom.ny, w.geom.nx))["model"], ref)
    srv.close()


def test_cancel_a_queued_request(cases):
    ws, datas, refs = cases
    srv = rbx.Server(hbm_budget_bytes=150 << 30, max_inflight=1)
    t1 = srv.submit(ws[3].geom, ws[3].c_init, ws[3].freqs, datas[3])
    t2 = srv.submit(ws[0].geom, ws[0].c_init, ws[0].freqs, datas[0])
    st = srv.cancel(t2)
    assert st in (0, 4)                                     # cancelled, or already running
    assert srv.wait(t1, 300.0) == 0
    if st == 0:
        assert srv.poll(t2)["state"] == rbx.REQ_CANCELLED
    srv.close()
