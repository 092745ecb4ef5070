"""Checkpoint and resume of a sweep from host memory.

A job's whole state between two frequencies of a sweep is its model: the tables, fields and
operands are recomputed from it at every update, and every reduction runs in a fixed order.
So a sweep stopped after its first frequency, its model copied to the host and the job
destroyed, then resumed in a new job from that copy, ends with the same bits as the sweep run
without a stop (both precisions).
"""
import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_resume_from_a_host_checkpoint_is_bit_identical(prec, oracle_mod):
    w = P.small_two_disc()
    g, freqs, df = w.geom, [float(f) for f in w.freqs], w.dfreq
    o = oracle_mod.Oracle(g)
    data = [torch.tensor(o.predict(f, w.c_true)[0], dtype=torch.complex64, device="cuda") for f in freqs]
    c0 = torch.tensor(w.c_init, dtype=torch.float32, device="cuda")

    def new_job(model):
        job = rbx.Job()
        job.set_geometry(g, precision=prec)
        job.set_model(model)
        return job

    whole = new_job(c0)
    for f, d in zip(freqs, data):
        whole.update_frequency(f, df, d)
    c_whole = whole.get_model().cpu().numpy()
    whole.close()

    first = new_job(c0)
    first.update_frequency(freqs[0], df, data[0])
    checkpoint = first.get_model().cpu().numpy().copy()        # host copy
    first.close()
    resumed = new_job(torch.tensor(checkpoint, device="cuda"))
    for f, d in zip(freqs[1:], data[1:]):
        resumed.update_frequency(f, df, d)
    c_resumed = resumed.get_model().cpu().numpy()
    resumed.close()

    assert not np.array_equal(checkpoint, c_whole)             # the later updates moved the model
    np.testing.assert_array_equal(c_resumed, c_whole)
