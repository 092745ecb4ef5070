"""Batched form: independent slices of different sizes, each a low-to-high sweep, run as one
CUDA graph (and as plain multi-stream work), with per-job traces or one persistent grouped
trace per sweep step, must give the models that running the slices one after the other
gives: exactly with per-job traces (every kernel is deterministic; only scheduling differs),
to rounding with the grouped trace (another compilation of the trace's arithmetic)."""
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
    grouped_models = []
    for use_graph, grouped in ((True, False), (False, False), (True, True), (False, True)):
        for w, j in zip(ws, jobs):
            j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
        last, ms = rbx.batch_run(jobs, [w.freqs for w in ws], data, use_graph=use_graph, grouped=grouped)
        assert ms > 0
        for k, j in enumerate(jobs):
            c = j.get_model().cpu().numpy()
            if grouped:
                # the grouped trace is another compilation of the same arithmetic: its tables
                # agree with the per-job trace's to rounding, and so do the models after 3 updates
                assert np.abs(c.astype(np.float64) - seq[k]).max() <= 0.01
                grouped_models.append(c)
            else:
                np.testing.assert_array_equal(c, seq[k])
            assert last[k]["rms_dc"] > 0 and last[k]["n_uncovered"] == 0
    for a, b in zip(grouped_models[:len(jobs)], grouped_models[len(jobs):]):
        np.testing.assert_array_equal(a, b)   # grouped: graph and direct queueing give the same bits
    for j in jobs:
        j.close()


def test_grouped_uneven_sweeps():
    """Sweeps of different lengths: the grouped trace of step q holds only the jobs still
    sweeping; the models equal those of the jobs run one after the other."""
    ws = slices()
    keep = (3, 1, 2)
    jobs, data = prepare(ws, rbx.RBX_BF16)
    fr = [w.freqs[:k] for w, k in zip(ws, keep)]
    dd = [d[:k].contiguous() for d, k in zip(data, keep)]
    seq = []
    for w, j, f, d in zip(ws, jobs, fr, dd):
        j.reconstruct(f, d)
        seq.append(j.get_model().cpu().numpy())
    for w, j in zip(ws, jobs):
        j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
    last, ms = rbx.batch_run(jobs, fr, dd, use_graph=True, grouped=True)
    for k, j in enumerate(jobs):
        assert np.abs(j.get_model().cpu().numpy().astype(np.float64) - seq[k]).max() <= 0.01
        assert last[k]["n_uncovered"] == 0
    for j in jobs:
        j.close()


def test_grouped_more_jobs_than_one_launch():
    """66 jobs: the grouped trace of a sweep step takes two launches (at most 64 jobs in one
    launch's job list); every job gets the update the job run alone gets, to rounding."""
    w = P.small_two_disc()
    jobs, data = prepare([w], rbx.RBX_BF16)
    jobs[0].reconstruct(w.freqs[:2], data[0][:2].contiguous())
    ref = jobs[0].get_model().cpu().numpy().astype(np.float64)
    jobs[0].close()
    many = []
    for _ in range(66):
        j = rbx.Job()
        j.set_geometry(w.geom, precision=rbx.RBX_BF16)
        j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
        many.append(j)
    d = data[0][:2].contiguous()
    last, ms = rbx.batch_run(many, [w.freqs[:2]] * 66, [d] * 66, use_graph=True, grouped=True)
    first = many[0].get_model().cpu().numpy()
    for k, j in enumerate(many):
        c = j.get_model().cpu().numpy()
        np.testing.assert_array_equal(c, first)       # same job, same bits, in either launch
        assert last[k]["n_uncovered"] == 0
    assert np.abs(first.astype(np.float64) - ref).max() <= 0.01
    for j in many:
        j.close()


def test_grouped_ignored_for_mixed_media():
    """A batch whose jobs differ in their absorption setting has no single trace kernel for
    all of them: the grouped flag is then ignored and the models equal those of the jobs run
    one after the other, bit for bit."""
    ws = slices()
    jobs, data = prepare(ws, rbx.RBX_BF16)
    w1 = ws[1]
    a0 = torch.tensor(P.absorption_map(w1.c_true).astype(np.float32), device="cuda")
    jobs[1].set_absorption(a0, 1.4)
    seq = []
    for w, j, d in zip(ws, jobs, data):
        j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
        j.reconstruct(w.freqs, d)
        seq.append(j.get_model().cpu().numpy())
    for w, j in zip(ws, jobs):
        j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
    rbx.batch_run(jobs, [w.freqs for w in ws], data, use_graph=True, grouped=True)
    for k, j in enumerate(jobs):
        np.testing.assert_array_equal(j.get_model().cpu().numpy(), seq[k])
    for j in jobs:
        j.close()


def test_grouped_tables_match_per_job():
    """The tables of one grouped trace equal the per-job trace's within the oracle parity
    tolerances (T 1e-9 s, a 1e-5 relative, gamma 1e-5 rad, exits), K and coverage exactly."""
    ws = slices()
    jobs, data = prepare(ws, rbx.RBX_BF16)
    for w, j in zip(ws, jobs):
        j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
    rbx.batch_run(jobs, [w.freqs[:1] for w in ws], [d[:1].contiguous() for d in data], use_graph=False, grouped=True)
    tg = [{k: v.cpu().numpy() for k, v in j.get_tables().items()} for j in jobs]
    for w, j in zip(ws, jobs):
        j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
        j.trace_rays(float(w.freqs[0]))
    for k, j in enumerate(jobs):
        t = {n: v.cpu().numpy() for n, v in j.get_tables().items()}
        g = tg[k]
        cov = t["a"] > 0
        np.testing.assert_array_equal(g["a"] > 0, cov)
        np.testing.assert_array_equal(g["K"], t["K"])
        assert np.abs(g["T"][cov].astype(np.float64) - t["T"][cov]).max() <= 1e-9
        assert np.abs(g["a"][cov] / t["a"][cov] - 1).max() <= 1e-5
        assert np.abs(np.angle(np.exp(1j * (g["gam"][cov].astype(np.float64) - t["gam"][cov])))).max() <= 1e-5
        assert np.abs(g["exits"][..., 1].astype(np.float64) - t["exits"][..., 1]).max() <= 1e-9
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

