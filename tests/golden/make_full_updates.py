"""Writes the oracle's one-step Hessian-free updates of two large workloads, used by
tests/test_gpu_full_update.py:

  ring1024_grid512_update.npz   the 1024-transducer, 512 x 512 workload (ring radius 110 mm,
                                grid 0.45 mm, breast-like phantom of seed 0), at the sweep's
                                lowest and highest frequency (0.1 and 1.2 MHz);
  slice28_ring768_grid448_update.npz   slice 28 of the uneven batch (768 transducers,
                                448 x 448 grid at 0.66 mm), at 0.1 and 1 MHz.

Each update starts from the workload's initial model (the truth blurred by a 5 mm Gaussian,
rounded to float32). Inputs come from the seeded generators of
paper_2211_00316_gb300.phantoms; every number written comes from oracle/ (the update of
Eqs. sound_speed_update / sound_speed_update2 with the step of Sec. 3.4; data = the oracle's
ray-Born prediction on the true model plus 40 dB noise of seed 300 + frequency index). The
test regenerates the data with the oracle and checks them against the checksums stored here
before it uses the update.

    python tests/golden/make_full_updates.py [ring1024|slice28]   # ~20 / ~10 min on 8 cores
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O                       # noqa: E402
from paper_2211_00316_gb300 import phantoms as P     # noqa: E402

NOISE_SEED = 300
PROBE = ((0, 1), (1, 0), (17, 530), (511, 700), (700, 300), (200, 11))   # (e, r) entries kept


def case(name):
    """(workload, frequency indices, output file) of a named case."""
    if name == "ring1024":
        return P.precision_ring1024(), (0, 19), os.path.join(HERE, "ring1024_grid512_update.npz")
    if name == "slice28":
        return P.batched_slice(28), (0, 9), os.path.join(HERE, "slice28_ring768_grid448_update.npz")
    raise SystemExit(f"unknown case {name}")


def make(name):
    w, fidx, out = case(name)
    o = O.Oracle(w.geom)
    c32 = w.c_init.astype(np.float32)
    m = w.geom.mask().ravel()
    rec = {"workload": w.name, "freq_index": np.array(fidx), "freqs": w.freqs[list(fidx)], "dfreq": w.dfreq,
           "tau": w.geom.tau, "threads": O.Oracle.threads(), "probe": np.array(PROBE)}
    for q in fidx:
        f = float(w.freqs[q])
        clean, _ = o.predict(f, w.c_true)
        data = P.add_noise(clean, w.snr_db, seed=NOISE_SEED + q)
        c_ref, st, bad = o.update_frequency(f, w.dfreq, c32.astype(np.float64), data)
        assert bad == 0
        rec[f"dc_{q}"] = (c_ref.ravel()[m] - c32.astype(np.float64).ravel()[m]).astype(np.float32)
        rec[f"stats_{q}"] = np.asarray(st)
        rec[f"clean_norm_{q}"] = np.linalg.norm(clean)
        rec[f"clean_probe_{q}"] = np.array([clean[e, r] for e, r in PROBE])
        print(f"{w.name} f = {f:.0f} Hz: rms dc {np.sqrt(np.mean(rec[f'dc_{q}'].astype(np.float64) ** 2)):.4f} m/s",
              flush=True)
    np.savez_compressed(out, **rec)
    print(out)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or ["ring1024", "slice28"]):
        make(nm)
