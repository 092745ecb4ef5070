"""Full-size end-to-end parity: one whole Hessian-free update (steps a1-a9 on the library's own
tables, with the forward split the autotuner picks and the launch configuration bench.py
times) compared with the FP64 oracle's update (Eqs. sound_speed_update /
sound_speed_update2, step of Sec. 3.4) at every mask node, at the lowest and highest
frequency of the sweep, FP32 and BF16 contractions: RMS of the difference <= 0.05 m/s.

Workloads: the 1024-transducer, 512 x 512 workload of the bench (152,088 mask nodes) and the
largest-ring slice of the uneven batch with a grid of at least 384 (slice 28: 768
transducers, 448 x 448 at 0.66 mm).

The oracle's updates (minutes each) are stored under tests/golden/ by
tests/golden/make_full_updates.py, which calls only oracle/. This test regenerates the data
those updates were computed from with the oracle (ray-Born prediction on the true model,
seeded 40 dB noise), checks them against the stored checksums, and also compares the
library's own predicted data on the true model with the oracle's over every (e, r) pair.
"""
import math
import os

import numpy as np
import pytest
import torch

from paper_2211_00316_gb300 import phantoms as P
from paper_2211_00316_gb300 import rbx

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NOISE_SEED = 300
CASES = {
    "ring1024": (P.precision_ring1024, "ring1024_grid512_update.npz", (0, 19)),
    "slice28": (lambda: P.batched_slice(28), "slice28_ring768_grid448_update.npz", (0, 9)),
}
_cache = {}


def dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def load(name, oracle_mod):
    """Workload, and per frequency index: (f, noise-free data, noisy data, oracle dc on the mask)."""
    if name in _cache:
        return _cache[name]
    make, fname, fidx = CASES[name]
    G = np.load(os.path.join(GOLDEN, fname))
    assert tuple(int(v) for v in G["freq_index"]) == fidx
    w = make()
    o = oracle_mod.Oracle(w.geom)
    per = {}
    for q in fidx:
        f = float(w.freqs[q])
        clean, _ = o.predict(f, w.c_true)
        # the regenerated data are the ones the stored update was computed from
        assert abs(np.linalg.norm(clean) / float(G[f"clean_norm_{q}"]) - 1.0) <= 1e-9
        probe = np.array([clean[e, r] for e, r in G["probe"]])
        assert np.abs(probe - G[f"clean_probe_{q}"]).max() <= 1e-9 * np.abs(clean).max()
        data = P.add_noise(clean, w.snr_db, seed=NOISE_SEED + q)
        per[q] = (f, clean, data, G[f"dc_{q}"].astype(np.float64))
    _cache[name] = (w, per)
    return _cache[name]


PARAMS = [(n, q) for n, (_, _, fi) in CASES.items() for q in fi]


@pytest.mark.parametrize("name,q", PARAMS)
@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_full_update_all_mask_nodes(name, q, prec, oracle_mod):
    w, per = load(name, oracle_mod)
    f, _, data, dc_ref = per[q]
    c32 = w.c_init.astype(np.float32)
    m = w.geom.mask().ravel()
    job = rbx.Job()
    job.set_geometry(w.geom, precision=prec)
    assert job.X == dc_ref.size
    job.set_model(dev(c32))
    st = job.update_frequency(f, w.dfreq, dev(data, torch.complex64))
    c = job.get_model().cpu().numpy().astype(np.float64).ravel()
    job.close()
    dc = c[m] - c32.astype(np.float64).ravel()[m]
    rms_err = float(np.sqrt(np.mean((dc - dc_ref) ** 2)))
    assert st["n_uncovered"] == 0
    assert np.sqrt(np.mean(dc_ref ** 2)) > 0.1            # a real update (0.27 m/s RMS at 0.1 MHz)
    assert rms_err <= 0.05, (name, prec, f, rms_err)


@pytest.mark.parametrize("name,q", PARAMS)
@pytest.mark.parametrize("prec", [rbx.RBX_FP32, rbx.RBX_BF16])
def test_predicted_data_all_pairs(name, q, prec, oracle_mod):
    """The library's prediction g_dir + F[m - m_s] on the true model, from its own tables,
    against the oracle's over all N(N-1) off-diagonal pairs. Bound per pair, relative to |g|:
    the table tolerance T <= 1e-9 s is a phase error of at most 2 pi f 1e-9 rad; the amplitude
    tolerance 1e-5 grows with the focusing of the ray, because a = sc / |J|^(1/2) turns an
    absolute error in the ray Jacobian J into a relative one of |dJ| / (2 |J|), which scales as
    rho^2 = (a / a_water)^2, a_water = s^(-1/2) at the chord s = |x_r - x_e| (rho from the
    oracle's |g| = C a); the exit amplitude of a ray meeting the ring m places from its
    transducer carries dr / (4 R sin^2(pi m / N)), dr = 8 ulp(R) of FP32 position rounding at
    grazing incidence (the bound the table parity tests derive); plus the contraction tolerance
    on identical tables (1e-5 FP32, 5e-3 BF16). The relative L2 error must stay within the
    |g|-weighted RMS of that bound."""
    w, per = load(name, oracle_mod)
    f, clean, _, _ = per[q]
    job = rbx.Job()
    job.set_geometry(w.geom, precision=prec)
    job.set_model(dev(w.c_true.astype(np.float32)))
    job.trace_rays(f)
    g = job.predict(f).cpu().numpy().astype(np.complex128)
    job.close()
    N = w.geom.n_xducers
    off = ~np.eye(N, dtype=bool)
    assert np.all(g[~off] == 0)
    rel = float(np.linalg.norm(g[off] - clean[off]) / np.linalg.norm(clean[off]))
    R = w.geom.ring_radius
    m = (np.arange(N)[None, :] - np.arange(N)[:, None]) % N
    sn2 = np.sin(np.pi * np.where(off, m, 1) / N) ** 2
    dr = 8 * float(np.spacing(np.float32(R)))
    beta = 2 * math.pi * np.arange(N) / N
    xy = R * np.stack([np.cos(beta), np.sin(beta)], 1)
    chord = np.linalg.norm(xy[:, None, :] - xy[None, :, :], axis=-1)
    C = (8 * math.pi * (2 * math.pi * f) / w.geom.c0) ** -0.5
    rho2 = np.where(off, (np.abs(clean) / C) ** 2 * chord, 1.0)
    b = (2 * math.pi * f * 1e-9 + 1e-5 * np.maximum(1.0, rho2) + dr / (4 * R * sn2)
         + (1e-5 if prec == rbx.RBX_FP32 else 5e-3))
    a2 = np.abs(clean[off]) ** 2
    tol = float(np.sqrt(np.sum(a2 * b[off] ** 2) / np.sum(a2)))
    assert rel <= tol, (name, prec, f, rel, tol)
