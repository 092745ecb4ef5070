"""Batched form: independent slices of different sizes, each a low-to-high sweep, run as one
CUDA graph (and as plain multi-stream work) must give exactly the models that running the
slices one after the other gives (every kernel is deterministic; only scheduling differs)."""
import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


def slices():
    return [P.small_two_disc(),
            P.custom(50, 83, 1e-3, 36e-3, kind="discs", ny=77, freqs=(2e5, 3e5, 4e5)),
            P.custom(96, 120, 0.8e-3, 40e-3, kind="breast", seed=3, freqs=(2e5, 3e5, 4e5))]


def prepare(ws, precision):
    jobs, data = [], []
    for w in ws:
        j = rbx.Job()
        j.set_geometry(w.geom, precision=precision)
        j.set_model(torch.tensor(w.c_true, dtype=torch.float32, device="cuda"))
        d = []
        for f in w.freqs:
            j.trace_rays(float(f))
            d.append(j.predict(float(f)).clone())
        j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
        jobs.append(j)
        data.append(torch.stack(d).contiguous())
    return jobs, data


@pytest.mark.parametrize("precision", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_batch_equals_sequential(precision):
    ws = slices()
    jobs, data = prepare(ws, precision)
    seq = []
    for w, j, d in zip(ws, jobs, data):
        j.reconstruct(w.freqs, d)
        seq.append(j.get_model().cpu().numpy())
    for use_graph in (True, False):
        for w, j in zip(ws, jobs):
            j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
        last, ms = rbx.batch_run(jobs, [w.freqs for w in ws], data, use_graph=use_graph)
        assert ms > 0
        for k, j in enumerate(jobs):
            np.testing.assert_array_equal(j.get_model().cpu().numpy(), seq[k])
            assert last[k]["rms_dc"] > 0 and last[k]["n_uncovered"] == 0
    for j in jobs:
        j.close()


def test_async_stats_match_sync():
    w = P.small_two_disc()
    jobs, data = prepare([w], rbx.RBX_BF16)
    j, d = jobs[0], data[0]
    st_sync = j.update_frequency(float(w.freqs[0]), 1e5, d[0])
    c_sync = j.get_model().cpu().numpy()
    j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
    j.update_frequency_async(float(w.freqs[0]), 1e5, d[0], slot=5)
    st = j.get_stats(5)
    np.testing.assert_array_equal(j.get_model().cpu().numpy(), c_sync)
    for k in ("resid_norm2", "rms_dc", "max_abs_dc", "dm_norm", "n_uncovered"):
        assert st[k] == st_sync[k]
    with pytest.raises(rbx.RbxError):
        j.get_stats(64)
    j.close()


def test_async_updates_with_slot_timing():
    """Updates queued back to back with per-slot timing: each slot returns its update's
    scalars (equal to the synchronous updates') and its own device timings and launch count."""
    w = P.small_two_disc()
    jobs, data = prepare([w], rbx.RBX_BF16)
    j, d = jobs[0], data[0]
    freqs = [float(f) for f in w.freqs]
    sync = []
    for f, dd in zip(freqs, d):
        sync.append(j.update_frequency(f, 1e5, dd))
    c_sync = j.get_model().cpu().numpy()
    j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
    j.set_slot_timing(True)
    for s, (f, dd) in enumerate(zip(freqs, d)):
        j.update_frequency_async(f, 1e5, dd, slot=s)
    asy = [j.get_stats(s) for s in range(len(freqs))]
    np.testing.assert_array_equal(j.get_model().cpu().numpy(), c_sync)
    for a, b in zip(asy, sync):
        for k in ("resid_norm2", "rms_dc", "max_abs_dc", "dm_norm", "n_uncovered"):
            assert a[k] == b[k]
        assert a["n_launches"] == b["n_launches"] > 0
        assert a["ms_total"] > 0 and a["ms_kernel"]["trace"] > 0 and a["ms_kernel"]["gemm_bp"] > 0
        assert a["ms_total"] >= a["ms_kernel"]["trace"]
    j.set_slot_timing(False)
    j.close()


def test_batch_reports_a_failure_inside_the_sweep():
    """A non-finite datum at the second frequency fails that update (the model is kept) and the
    later updates succeed; the batch must still report the failure."""
    ws = slices()[:2]
    jobs, data = prepare(ws, rbx.RBX_BF16)
    data[1][1, 3, 7] = complex(float("nan"), 0.0)
    with pytest.raises(rbx.RbxError) as e:
        rbx.batch_run(jobs, [w.freqs for w in ws], data, use_graph=True)
    assert e.value.status == 5 and "update 2 of 3" in str(e.value)
    for j in jobs:
        j.close()

