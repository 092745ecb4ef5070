"""The host-buffer entry point (rbx_update_frequency_host: the data copied from pinned host
memory beside the trace on a copy stream, the model copied back) gives the same bits as the
device-buffer entry (rbx_update_frequency) over consecutive updates, which reuse the job's
data buffer while the previous update may still be queued."""
import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_host_entry_equals_device_entry(precision):
    w = P.fp32_ring256()
    g = w.geom
    job = rbx.Job()
    job.set_geometry(g, precision=precision)
    job.set_model(torch.tensor(w.c_true, dtype=torch.float32, device="cuda"))
    freqs = [float(f) for f in w.freqs[:3]]
    data = []
    for f in freqs:
        job.trace_rays(f)
        data.append(job.predict(f).clone())
    c0 = torch.tensor(w.c_init, dtype=torch.float32, device="cuda")
    job.set_model(c0)
    ref, ref_st = [], []
    for f, d in zip(freqs, data):
        ref_st.append(job.update_frequency(f, w.dfreq, d))
        ref.append(job.get_model().cpu().numpy())
    job.set_model(c0)
    c_host = torch.empty((g.ny, g.nx), dtype=torch.float32).pin_memory()
    for k, (f, d) in enumerate(zip(freqs, data)):
        st = job.update_frequency_host(f, w.dfreq, d.cpu().pin_memory(), c_host)
        np.testing.assert_array_equal(c_host.numpy(), ref[k])
        np.testing.assert_array_equal(job.get_model().cpu().numpy(), ref[k])
        for key in ("resid_norm2", "rms_dc", "max_abs_dc", "n_uncovered"):
            assert st[key] == ref_st[k][key], key
    job.close()
