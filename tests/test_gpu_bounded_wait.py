"""Failure detection without a GPU fault: the bounded waits of the tensor-core kernels.

Every spin-wait in the library's tensor-core kernels gives up after about one second,
records a timeout and returns, so a lost signal ends in an error status instead of a hang.
rbx_selftest_bounded_wait runs one kernel whose thread waits, with that bound, on a barrier
that nothing ever signals. The test checks that the wait gave up and that the CUDA context
is still usable afterwards: a small BF16 update runs and matches the oracle.
"""
import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


def test_wait_on_a_barrier_nothing_signals_gives_up(oracle_mod):
    assert rbx.selftest_bounded_wait() is True
    torch.cuda.synchronize()
    w = P.small_two_disc()
    g, f = w.geom, 3e5
    o = oracle_mod.Oracle(g)
    data, _ = o.predict(f, w.c_true)
    c64 = w.c_init.astype(np.float32).astype(np.float64)
    c_ref, _, _ = o.update_frequency(f, 1e5, c64, data)
    job = rbx.Job()
    job.set_geometry(g, precision=rbx.RBX_BF16)
    job.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))
    job.update_frequency(f, 1e5, torch.tensor(data, dtype=torch.complex64, device="cuda"))
    c_gpu = job.get_model().cpu().numpy().astype(np.float64)
    m = g.mask()
    assert np.sqrt(np.mean((c_gpu[m] - c_ref[m]) ** 2)) <= 0.05
    job.close()
