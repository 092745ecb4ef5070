"""rbx_forward_noalloc: the Born forward for callers that cannot allocate device memory.

It is called through the C ABI and must give the same D as rbx_forward on the same
tables, twice in a row (its fixed scratch array keeps the previous call's contents).
This file is collected last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = pytest.mark.gpu


def test_noalloc_forward_matches_rbx_forward_twice():
    L = rbx.load()
    g = P.custom(50, 83, 1e-3, 36e-3, kind="water", ny=77)
    N = g.geom.n_xducers
    job = rbx.Job()
    job.set_geometry(g.geom)
    X = job.X
    rng = np.random.default_rng(5)
    T = torch.tensor(rng.uniform(1e-5, 6e-5, (N, X)), dtype=torch.float32, device="cuda")
    a = torch.tensor(rng.uniform(3.0, 30.0, (N, X)), dtype=torch.float32, device="cuda")
    a[3, 7] = 0.0                                                    # one uncovered entry
    gam = torch.tensor(rng.uniform(-3, 3, (N, X)), dtype=torch.float32, device="cuda")
    K = torch.zeros((N, X), dtype=torch.uint8, device="cuda")
    exits = torch.zeros((N, N - 1, 4), dtype=torch.float32, device="cuda")
    job.set_tables(T, a, gam, K, exits)
    f = 3.1e5
    dm = rng.standard_normal((g.geom.ny, g.geom.nx)) * 1e-9
    D_ref = job.forward(f, torch.tensor(dm, dtype=torch.float32, device="cuda")).cpu().numpy()
    idx = job.mask_idx().cpu().numpy()
    w = 2 * math.pi * f
    v = torch.tensor((w * w * g.geom.dx ** 2 * dm.astype(np.float32).astype(np.float64).ravel()[idx]),
                     dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream or None
    err = C.create_string_buffer(256)
    for call in range(2):
        D = torch.full((N, N), float("nan"), dtype=torch.complex64, device="cuda")
        st = L.rbx_forward_noalloc(T.data_ptr(), a.data_ptr(), K.data_ptr(), v.data_ptr(), N, X, f, g.geom.c0,
                                   D.data_ptr(), stream, err, len(err))
        assert st == 0, err.value.decode()
        Dn = D.cpu().numpy()
        rel = np.linalg.norm(Dn - D_ref) / np.linalg.norm(D_ref)
        assert rel <= 1e-5, (call, rel)
    job.close()


def test_noalloc_forward_rejects_oversized_problems():
    L = rbx.load()
    err = C.create_string_buffer(256)
    d = torch.zeros(16, device="cuda")
    st = L.rbx_forward_noalloc(d.data_ptr(), d.data_ptr(), d.data_ptr(), d.data_ptr(), 1025, 4, 3e5, 1500.0,
                               d.data_ptr(), None, err, len(err))
    assert st == 1 and b"1024" in err.value
