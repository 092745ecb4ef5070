#!/usr/bin/env python
"""Benchmark: Hessian-free ray-Born frequency updates per second on GB300.

One step = one full update at one frequency (smoothing, ray tracing and tables, direct
Green's function, Born forward and residual, preconditioned back-projection, update) of
the 1024-transducer / 512x512 workload, through the library's C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--precision P]
  python bench.py --impl reference ...     # the FP64 CPU oracle on the machine's host cores

Under torchrun each rank runs an independent replica job (its own phantom seed) on its
own GPU: there is no data-path collective (weak scaling). Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-Born freq-updates/s at 1024 xducers, 512² grid; p50/p99 request latency"
UNIT = "freq-updates/s"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128


def workload(name: str, seed: int):
    from paper_2211_00316_gb300 import phantoms as P
    if name == "precision_ring1024":
        w = P.breast(1024, 512, 0.45e-3, 110e-3, np.linspace(1e5, 1.2e6, 20), seed=seed, name="ring1024_grid512_breast")
    elif name == "fp32_ring256":
        w = P.breast(256, 288, 0.8e-3, 110e-3, np.linspace(1e5, 1e6, 10), seed=seed, name="ring256_grid288_breast")
    elif name == "ring1024_grid288":
        w = P.breast(1024, 288, 0.8e-3, 110e-3, np.linspace(1e5, 1e6, 10), seed=seed, name="ring1024_grid288_breast")
    elif name == "small":
        w = P.small_two_disc()
    else:
        raise SystemExit(f"unknown workload {name}")
    return w


def describe(w) -> str:
    g = w.geom
    return (f"{w.name}: N={g.n_xducers} ring R={g.ring_radius*1e3:.0f} mm, {g.nx}x{g.ny} grid at "
            f"{g.dx*1e3:.2f} mm, {len(w.freqs)} freqs {w.freqs[0]/1e6:.2f}-{w.freqs[-1]/1e6:.2f} MHz, "
            f"{w.snr_db:.0f} dB, one update per step")


def peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
    except OSError:
        pass
    return {"hbm_gbs": p.get("hbm_gbs", 6800.0), "bf16_tflops": p.get("bf16_tflops", 1900.0),
            "bf16_tflops_sustained": p.get("bf16_tflops_sustained", 1700.0),
            "source": "measured" if p else "fallback"}


# source files that define each timed kernel (a recorded ncu traffic figure is valid only for
# the sources it was taken on)
KERNEL_SRC = {
    "trace": ["k_rays.cu"],
    "gemm_fwd": ["k_gemm_tc.cu", "tc_sm100.cuh", "k_gemm_simt.cu"],
    "gemm_bp": ["k_gemm_tc.cu", "tc_sm100.cuh", "k_gemm_simt.cu"],
    "synth_fwd": ["k_gemm_tc.cu", "k_gemm_simt.cu"],
    "synth_bp": ["k_gemm_tc.cu", "k_gemm_simt.cu"],
    "synth": ["k_gemm_tc.cu"],
}


def kernel_src_hash(kernel: str) -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2211_00316_gb300", "csrc")
    for f in KERNEL_SRC.get(kernel, sorted(os.listdir(d))):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


# DRAM bytes per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum), keyed by
# (workload, kernel); valid only for the kernel sources they were taken on.
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
    #     -k regex:k_trace_raster -s 3 -c 1 --csv   (k_synth_tc: -k regex:k_synth_tc -s 6 -c 1)
    #     python bench.py --steps 2 --warmup 1 --no-cpu-baseline --no-e2e --no-forms   (1 pass)
    ("precision_ring1024", "trace"): {"bytes": 2.521059840e9 + 2.463850752e9, "src": "40dc5317b6bf"},
    ("precision_ring1024", "synth"): {"bytes": 2.496856832e9 + 3.071679744e9, "src": "861bfb904eef"},
}


def algorithmic(kernel: str, N: int, X: int, precision: str):
    """Algorithmic work per launch of each timed kernel: (amount, unit, bound)."""
    NX = N * X
    if kernel == "gemm_bp":
        return 8.0 * 2 * X * N * N, "flop", "alu" if precision == "fp32" else "tensor"
    if kernel == "gemm_fwd":
        return 8.0 * N * (N + 1) / 2 * X, "flop", "alu" if precision == "fp32" else "tensor"
    if kernel == "trace":
        return 16.0 * NX + 16.0 * N * (N - 1), "byte", "hbm"
    planes = 2.0 if precision == "bf16x3" else 1.0   # split BF16 writes a lo plane per hi plane
    if kernel == "synth_fwd":
        return (16.0 + (8.0 * planes if precision != "fp32" else 8.0)) * NX, "byte", "hbm"
    if kernel == "synth":
        # fused: tables in once; forward (4 planes) and back-projection (6 planes) BF16 out
        return (16.0 + 20.0 * planes) * NX, "byte", "hbm"
    if kernel == "synth_bp":
        # tables in; FP32: angular density in, U and kappa out; BF16: 6 planes out (x2 when split)
        out = {"fp32": 4.0 + 16.0, "bf16": 12.0, "bf16x3": 24.0}[precision]
        return (16.0 + out) * NX, "byte", "hbm"
    if kernel == "tables":
        # direct Green's function (exits in, N x N complex out); FP32 also forms the angular
        # density array (tables in, one float out per entry)
        green = 16.0 * N * (N - 1) + 8.0 * N * N
        return green + ((16.0 + 4.0) * NX if precision == "fp32" else 0.0), "byte", "hbm"
    return None, None, None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "50",
                                       "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        # the timed region starts once the sampler is running (its first sample is written)
        t0 = time.perf_counter()
        while self.p is not None and time.perf_counter() - t0 < 3.0 and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample(w, f: float, o, tables_at) -> dict:
    """A bounded sample of one update of the FP64 oracle, as it stands, scaled to a whole
    update: ray fans of 4 x threads transducers (tables), the Born forward over all mask nodes
    for the (2 x threads)^2 (e, r) entries of 2 x threads fans, and the unfactorised
    back-projection at 32 x threads mask nodes on the workload's own tables (tables_at: the
    oracle tables of all fans at those nodes); the O(N^2) direct Green's function and the
    update are negligible beside them."""
    from oracle import oracle as O
    N, X = o.N, o.X
    rng = np.random.default_rng(0)
    nth = O.Oracle.threads()
    t0 = time.perf_counter()
    ns, f6 = o.fields_for(w.c_init, f)
    t_fields = time.perf_counter() - t0
    nfans = min(N, 4 * nth)
    fans = np.linspace(0, N - 1, nfans).astype(np.int32)
    t0 = time.perf_counter()
    tb = o.tables(f6, fans=fans)
    t_rays = (time.perf_counter() - t0) / nfans * N
    nr = min(nfans, 2 * nth)
    v = rng.standard_normal(X) * 1e-3
    t0 = time.perf_counter()
    O.forward_rows(o, f, tb.T[:nr], tb.a[:nr], tb.K[:nr], v)
    t_fwd = (time.perf_counter() - t0) / (nr * nr) * N * N
    T, a, gam, K, dg = tables_at
    nn = T.shape[1]
    R = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    t0 = time.perf_counter()
    O.backproject_nodes(o, f, T, a, gam, K, dg, R)
    t_bp = (time.perf_counter() - t0) / nn * X
    total = t_fields + t_rays + t_fwd + t_bp
    return {"seconds_per_update": total, "cores": nth,
            "sample": (f"one update extrapolated from: ray fans of {nfans}/{N} transducers, Born forward of "
                       f"{nr}x{nr}/{N}x{N} (e,r) entries over all {X} mask nodes, back-projection at {nn}/{X} "
                       f"nodes on the workload's tables (s per full update: rays {t_rays:.1f}, forward {t_fwd:.1f}, "
                       f"back-projection {t_bp:.1f})")}


def oracle_tables_at(w, f: float, o, nodes):
    """The oracle's tables of all fans at the given mask nodes (for the sampled back-projection)."""
    ns, f6 = o.fields_for(w.c_init, f)
    tb = o.tables(f6)
    og = type(o)(w.geom)
    og.X = len(nodes)
    sub = [x[:, nodes] for x in (tb.T, tb.a, tb.gam, tb.K, tb.cov)]
    dg = og.dgamma(sub[2].astype(np.float64), sub[4])
    return sub[0], sub[1], sub[2], sub[3], dg


def cpu_full_update(w, f: float, data) -> dict:
    """One whole update (a1-a9) of the FP64 oracle, as it stands, timed on all host threads."""
    from oracle import oracle as O
    o = O.Oracle(w.geom)
    t0 = time.perf_counter()
    _, _, bad = o.update_frequency(f, w.dfreq, np.asarray(w.c_init, np.float64), np.asarray(data, np.complex128))
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": O.Oracle.threads(), "kind": "oracle",
            "sample": (f"one whole update of the workload at {f/1e6:.2f} MHz (tables of all {o.N} fans, Born forward "
                       f"of all pairs, unfactorised back-projection at all {o.X} mask nodes, update): {dt:.1f} s"),
            "seconds_per_update": dt}


def time_noalloc(job, rbx, torch, g, f: float, stream, reps: int = 5) -> dict:
    """Device time (CUDA events on the job's stream) of rbx_forward and of
    rbx_forward_noalloc on the job's own tables for one perturbation: 3 warm-up calls each,
    then the mean of reps."""
    import ctypes as C
    L = rbx.load()
    job.trace_rays(f)
    t = job.get_tables()
    T, a, K = t["T"], t["a"], t["K"]
    del t
    N, X = job.N, job.X
    rng = np.random.default_rng(9)
    dm = torch.tensor(rng.standard_normal((g.ny, g.nx)) * 1e-9, dtype=torch.float32, device="cuda")
    idx = job.mask_idx().long()
    w = 2 * math.pi * f
    v = (dm.reshape(-1)[idx].double() * (w * w * g.dx ** 2)).float().contiguous()
    D = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    err = C.create_string_buffer(256)

    def na():
        st = L.rbx_forward_noalloc(T.data_ptr(), a.data_ptr(), K.data_ptr(), v.data_ptr(), N, X, f, g.c0,
                                   D.data_ptr(), C.c_void_p(stream.cuda_stream), err, len(err))
        assert st == 0, err.value.decode()

    out = {}
    for name, fn in (("rbx_forward", lambda: job.forward(f, dm)), ("rbx_forward_noalloc", na)):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms"] = e0.elapsed_time(e1) / reps
    out["scratch_split_cap"] = (1 << 20) // (N * N)    # 8 MiB of float2 partial sums / (N x N per split)
    out["note"] = ("rbx_forward at the job's precision (synthesis pass + contraction); rbx_forward_noalloc FP32 SIMT "
                   "with the Green's functions formed in the tile loads, unsplit at N = 1024")
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    w = workload(args.workload, 0)
    o = O.Oracle(w.geom)
    t_start = time.perf_counter()
    # the sampled back-projection runs on the workload's own tables (those of the lowest
    # frequency's window; its cost does not depend on the values)
    nodes = np.linspace(0, o.X - 1, 32 * O.Oracle.threads()).astype(np.int64)
    tab = oracle_tables_at(w, float(w.freqs[0]), o, nodes)
    vals = []
    for k in range(args.warmup + args.steps):
        f = float(w.freqs[k % len(w.freqs)])
        cb = cpu_sample(w, f, o, tab)
        if k >= args.warmup:
            vals.append(cb["seconds_per_update"])
    value = len(vals) / sum(vals)
    # one whole update beside the sampled steps, on the oracle's own data (prediction on the
    # true model + 40 dB noise)
    full = None
    if not args.no_cpu_baseline:
        from paper_2211_00316_gb300 import phantoms as P
        f0 = float(w.freqs[0])
        clean, _ = o.predict(f0, w.c_true)
        full = cpu_full_update(w, f0, P.add_noise(clean, w.snr_db, seed=100))
    wall = time.perf_counter() - t_start
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": describe(w), "parallelism": "host threads"},
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"], "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "full_update": full, "wall_s": wall}
    print(json.dumps(line), flush=True)
    return 0


def slice_pool(n_slices: int, rbx, P, torch) -> list:
    """The uneven slices of the batched workload (seeds 0..n-1) with their data: the library's
    FP32 ray-Born prediction on each true model plus 40 dB noise, as host arrays."""
    pool = []
    for s in range(n_slices):
        w = P.batched_slice(s)
        j = rbx.Job()
        j.set_geometry(w.geom, precision=rbx.RBX_FP32)
        j.set_model(torch.tensor(w.c_true, dtype=torch.float32, device="cuda"))
        d = []
        for f in w.freqs:
            j.trace_rays(float(f))
            d.append(j.predict(float(f)).cpu().numpy())
        j.close()
        pool.append((w, P.add_noise(np.stack(d), w.snr_db, seed=200 + s).astype(np.complex64)))
    return pool


def batched_form(args, rbx, P, torch, pool=None, steps=None, warmup=None, variants=None) -> dict:
    """32 independent slices of uneven size, each a full 10-frequency sweep (320 updates per
    step): one CUDA graph of all sweeps (BF16), the same work as plain multi-stream launches,
    and the plain per-job forms (each job's sweep after the other's, synchronising per update)
    in BF16 and FP32. variants: the forms to time (default: all five)."""
    pool = pool or slice_pool(args.slices, rbx, P, torch)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    variants = variants or ("graph_bf16", "grouped_bf16", "streams_bf16", "sequential_bf16", "graph_fp32",
                            "sequential_fp32")
    freqs = [w.freqs for w, _ in pool]
    updates = sum(len(f) for f in freqs)
    out = {"updates_per_step": updates}
    models = {}

    def make(prec):
        jobs, data = [], []
        for w, d in pool:
            j = rbx.Job()
            j.set_geometry(w.geom, precision=prec)
            jobs.append(j)
            data.append(torch.tensor(d, device="cuda"))
        est = sum(rbx.estimate_bytes(w.geom, len(w.freqs), prec) for w, _ in pool)
        return jobs, data, est

    def reset(jobs):
        for (w, _), j in zip(pool, jobs):
            j.set_model(torch.tensor(w.c_init, dtype=torch.float32, device="cuda"))

    def timed(name, jobs, run):
        if name not in variants:
            return
        for _ in range(warmup):
            reset(jobs)
            run()
        dev, wall = [], []
        for _ in range(steps):
            reset(jobs)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ms = run()
            torch.cuda.synchronize()
            wall.append(time.perf_counter() - t0)
            dev.append(ms / 1e3 if ms is not None else wall[-1])
        models[name] = [j.get_model().cpu().numpy() for j in jobs]
        out[name] = {"value": updates / float(np.mean(dev)), "unit": UNIT, "s_per_step_device": float(np.mean(dev)),
                     "s_per_step_wall": float(np.mean(wall))}

    kernel_ms = {}

    def sequential(jobs, data, tag):
        def run():
            acc = {}
            for w, j, d in zip(pool, jobs, data):
                for st in j.reconstruct(w[0].freqs, d):
                    for k, v in st["ms_kernel"].items():
                        acc[k] = acc.get(k, 0.0) + v
            kernel_ms[tag] = acc   # per-kernel device time of the step's updates, each run alone
        return run

    for prec, tag in ((rbx.RBX_BF16, "bf16"), (rbx.RBX_FP32, "fp32")):
        used0 = rbx.pool_usage(trim=True)["used"]
        jobs, data, est = make(prec)
        data_bytes = sum(d.numel() * d.element_size() for d in data)
        used1 = rbx.pool_usage()["used"]
        reset(jobs)
        batch_run = lambda g: (lambda: rbx.batch_run(jobs, freqs, data, use_graph=g)[1])
        timed(f"graph_{tag}", jobs, batch_run(True))
        timed(f"grouped_{tag}", jobs, lambda: rbx.batch_run(jobs, freqs, data, use_graph=True, grouped=True)[1])
        timed(f"streams_{tag}", jobs, batch_run(False))
        timed(f"sequential_{tag}", jobs, sequential(jobs, data, tag))
        out[f"device_bytes_{tag}"] = {"jobs_measured": int(used1 - used0 + data_bytes), "estimate": int(est)}
        for j in jobs:
            j.close()
        del data
        torch.cuda.empty_cache()
    # agreement of the BF16 graph form with the plain FP32 form after the whole sweep
    diffs = [float(np.sqrt(np.mean((a - b) ** 2))) for a, b in zip(models["graph_bf16"], models["sequential_fp32"])]
    same = all(np.array_equal(a, b) for a, b in zip(models["graph_bf16"], models["sequential_bf16"]))
    out["graph_bf16_over_sequential_fp32"] = out["graph_bf16"]["value"] / out["sequential_fp32"]["value"]
    if "grouped_bf16" in out:
        out["grouped_bf16_over_sequential_fp32"] = out["grouped_bf16"]["value"] / out["sequential_fp32"]["value"]
    # where the device time of the slices' updates goes (each update run alone, BF16): shares
    if "bf16" in kernel_ms:
        tot = sum(kernel_ms["bf16"].values())
        out["kernel_share_bf16"] = {k: v / tot for k, v in sorted(kernel_ms["bf16"].items(), key=lambda x: -x[1])}
    out["rms_dc_bf16_vs_fp32_m_s"] = {"max": max(diffs), "median": float(np.median(diffs))}
    # error against the true model on the mask after the sweep, per slice: initial, BF16, FP32
    errs = []
    for k, (w, _) in enumerate(pool):
        mk = w.geom.mask()
        e = [float(np.sqrt(np.mean((x[mk] - w.c_true[mk]) ** 2)))
             for x in (w.c_init, models["graph_bf16"][k], models["sequential_fp32"][k])]
        errs.append([w.name] + [round(v, 4) for v in e] + [round(diffs[k], 4)])
    out["rms_vs_true_m_s"] = {"columns": ["slice", "initial", "bf16_graph", "fp32_plain", "bf16_vs_fp32"], "rows": errs}
    out["graph_equals_sequential_bf16"] = bool(same)
    if "grouped_bf16" in models:
        # the grouped trace agrees with the per-job trace to rounding; a 10-update sweep carries
        # that into the models as it carries the BF16 / FP32 difference (RMS over each mask)
        dg = [float(np.sqrt(np.mean((a[w.geom.mask()].astype(np.float64) - b[w.geom.mask()]) ** 2)))
              for (w, _), a, b in zip(pool, models["grouped_bf16"], models["sequential_bf16"])]
        out["rms_dc_grouped_vs_sequential_bf16_m_s"] = {"max": max(dg), "median": float(np.median(dg))}
    out["slices"] = [f"{w.name} dx={w.geom.dx*1e3:.2f}mm" for w, _ in pool]
    return out


def served_form(rbx, P, torch, pool, n_req: int, rate: float, budget: float, max_inflight: int, closed: int,
                serial_fp32: bool) -> dict:
    """Poisson arrivals (seeded) of reconstruction requests drawn from the slice pool, each a full
    sweep, submitted to the library's server. Latency of both arms = scheduled arrival to
    completion: for the served form, the server's submit-to-completion time plus the lag of the
    submit call behind its scheduled arrival (host clock). Also a closed-loop burst (all
    requests at once: maximum throughput) and, optionally, the same arrival stream served by the
    plain per-job FP32 form one request after the other."""
    rng = np.random.default_rng(5)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    res = {"requests": n_req, "rate_req_s": rate, "hbm_budget_gb": budget / 1e9, "max_inflight": max_inflight}

    def pct(lat):
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(np.mean(lat)), "max_s": float(np.max(lat))}

    srv = rbx.Server(int(budget), max_inflight)
    warm = [srv.submit(w.geom, w.c_init, w.freqs, d) for w, d in pool[:4]]
    for t in warm:
        assert srv.wait(t, 600.0) == 0
    t0 = time.perf_counter()
    tickets, lag = [], []
    for k in range(n_req):
        dt = t0 + arrivals[k] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        w, d = pool[k % len(pool)]
        lag.append(time.perf_counter() - (t0 + arrivals[k]))   # submit call behind its scheduled arrival
        tickets.append(srv.submit(w.geom, w.c_init, w.freqs, d))
    for t in tickets:
        assert srv.wait(t, 600.0) == 0, srv.poll(t)["error"]
    tm = [srv.times(t) for t in tickets]
    ups = sum(len(pool[k % len(pool)][0].freqs) for k in range(n_req))
    span = max(x["end"] for x in tm) - min(x["submit"] for x in tm)
    res["open_loop"] = dict(pct([x["end"] - x["submit"] + l for x, l in zip(tm, lag)]),
                            from_submit=pct([x["end"] - x["submit"] for x in tm]),
                            submit_lag_max_s=float(max(lag)),
                            queue_wait_p99_s=float(np.percentile([x["start"] - x["submit"] for x in tm], 99)),
                            updates_per_s=ups / span)
    if closed > 0:
        tk = [srv.submit(*(lambda w, d: (w.geom, w.c_init, w.freqs, d))(*pool[k % len(pool)])) for k in range(closed)]
        for t in tk:
            assert srv.wait(t, 600.0) == 0
        tm = [srv.times(t) for t in tk]
        ups = sum(len(pool[k % len(pool)][0].freqs) for k in range(closed))
        span = max(x["end"] for x in tm) - min(x["submit"] for x in tm)
        res["closed_loop"] = dict(pct([x["end"] - x["submit"] for x in tm]), requests=closed, updates_per_s=ups / span)
    srv.close()
    if serial_fp32:
        lat, busy = [], 0.0
        t0 = time.perf_counter()
        for k in range(n_req):
            dt = t0 + arrivals[k] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            w, d = pool[k % len(pool)]
            ts = time.perf_counter()
            j = rbx.Job()
            j.set_geometry(w.geom, precision=rbx.RBX_FP32)
            j.set_model(torch.tensor(w.c_init, dtype=torch.float32).cuda())
            j.reconstruct(w.freqs, torch.tensor(d).cuda())
            j.get_model().cpu()
            j.close()
            te = time.perf_counter()
            busy += te - ts
            lat.append(te - (t0 + arrivals[k]))
        ups = sum(len(pool[k % len(pool)][0].freqs) for k in range(n_req))
        res["serial_plain_fp32"] = dict(pct(lat), updates_per_s_busy=ups / busy)
    return res


def run_forms(args) -> int:
    import torch
    torch.cuda.set_device(0)
    from paper_2211_00316_gb300 import build as B
    B.build()
    from paper_2211_00316_gb300 import phantoms as P
    from paper_2211_00316_gb300 import rbx
    clocks = Clocks(0)
    if args.workload == "batched_slices32":
        r = batched_form(args, rbx, P, torch)
        clk = clocks.stop()
        line = {"metric": "ray-Born freq-updates/s, 32 uneven slices, full 10-frequency sweeps",
                "value": r["graph_bf16"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["graph_bf16"]["s_per_step_device"] * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic (library FP32 ray-Born prediction on seeded breast-like slices + 40 dB noise)",
                "config": {"workload": f"{args.slices} slices: N in {{256,512,768,1024}}, grids 192-512 at "
                                       "0.45-1.0 mm, seeds 0-31, 100 kHz-1 MHz",
                           "form": "one CUDA graph of all sweeps, per-job traces, BF16 (grouped trace in forms)",
                           "l2": "inputs larger than L2"},
                "clocks": clk, "forms": r}
    else:
        pool = slice_pool(args.slices, rbx, P, torch)
        r = served_form(rbx, P, torch, pool, args.requests, args.rate, args.budget_gb * 1e9, args.max_inflight,
                        args.closed, not args.no_serial)
        clk = clocks.stop()
        line = {"metric": "p50/p99 request latency, Poisson arrivals", "value": r["open_loop"]["p50_s"], "unit": "s",
                "n_gpus": 1, "higher_is_better": False, "dtype": "bf16",
                "data": "synthetic (library FP32 ray-Born prediction on seeded breast-like slices + 40 dB noise)",
                "config": {"workload": f"{args.requests} requests at {args.rate} req/s drawn from {args.slices} "
                                       "uneven slices, 10-frequency sweeps", "hbm_budget_gb": args.budget_gb},
                "clocks": clk, "serve": r}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="rbx", choices=["rbx", "reference"])
    ap.add_argument("--workload", default="precision_ring1024",
                    choices=["precision_ring1024", "fp32_ring256", "ring1024_grid288", "small", "batched_slices32",
                             "served_poisson"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--slices", type=int, default=32, help="batched/served forms: slices in the pool")
    ap.add_argument("--requests", type=int, default=500, help="served form: Poisson requests")
    ap.add_argument("--rate", type=float, default=4.0, help="served form: arrivals per second")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served form: HBM admission budget")
    ap.add_argument("--max-inflight", type=int, default=16)
    ap.add_argument("--closed", type=int, default=64, help="served form: closed-loop burst size (0 = none)")
    ap.add_argument("--no-serial", action="store_true", help="served form: skip the serial plain FP32 replay")
    ap.add_argument("--absorption", action="store_true",
                    help="lossy medium: breast absorption map 0-1 dB/(MHz^1.4 cm), y = 1.4 (rbx_set_absorption)")
    ap.add_argument("--integration", default="smoothed", choices=["smoothed", "raw"],
                    help="raw: integrate on the non-smoothed map, no Born term (rbx_set_integration 1)")
    ap.add_argument("--link", type=int, default=0,
                    help="secant ray linking of the direct term, new rays per pair (rbx_set_linking; 0: off)")
    ap.add_argument("--set-size", type=int, default=1,
                    help="frequencies per update (rbx_update_set); value then counts frequencies per second")
    ap.add_argument("--log-jsonl", default=None,
                    help="append one JSON line per timed update (frequency, residual, model change, stage times)")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the batched and served forms reported beside throughput")
    ap.add_argument("--forms-steps", type=int, default=3, help="batched form beside the default workload: timed steps")
    ap.add_argument("--forms-warmup", type=int, default=3, help="batched form beside the default workload: warm-up")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batched_slices32", "served_poisson"):
        return run_forms(args)

    import torch
    import torch.distributed as dist
    from paper_2211_00316_gb300 import replicas as REP
    info = REP.RankInfo.from_env()
    world, rank, local = info.world, info.rank, info.local
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2211_00316_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2211_00316_gb300 import phantoms as P
    from paper_2211_00316_gb300 import rbx

    prec = {"fp32": rbx.RBX_FP32, "bf16": rbx.RBX_BF16, "bf16x3": rbx.RBX_BF16X3}[args.precision]
    w = workload(args.workload, REP.replica_seed(rank))
    g = w.geom
    stream = torch.cuda.Stream()
    total_steps = args.warmup + args.steps
    with torch.cuda.stream(stream):
        job = rbx.Job(stream)
        job.set_geometry(g, precision=prec)
        N, X = job.N, job.X
        tuning = job.tuning() if args.precision != "fp32" else None
        if args.absorption:
            job.set_absorption(torch.tensor(P.absorption_map(w.c_true), dtype=torch.float32, device="cuda"), 1.4)
        if args.integration == "raw":
            job.set_integration(True)
        if args.link > 0:
            job.set_linking(args.link)
        K = max(1, args.set_size)
        # synthetic data: the library's own ray-Born prediction on the true model + 40 dB noise
        job.set_model(torch.tensor(w.c_true, dtype=torch.float32, device="cuda"))
        fidx = [(k * K) % (len(w.freqs) - K + 1) for k in range(total_steps)]
        fset = [[fidx[k] + q for q in range(K)] for k in range(total_steps)]
        uniq = sorted(set(q for fs in fset for q in fs))
        data = {}
        for q in uniq:
            f = float(w.freqs[q])
            job.trace_rays(f)
            data[q] = job.predict(f).cpu().numpy()
        noisy = P.add_noise(np.stack([data[q] for q in uniq]), w.snr_db, seed=100 + rank)
        data_dev = {q: torch.tensor(noisy[i], dtype=torch.complex64, device="cuda") for i, q in enumerate(uniq)}
        data_host = {q: torch.tensor(noisy[i], dtype=torch.complex64).pin_memory() for i, q in enumerate(uniq)}
        c_init = torch.tensor(w.c_init, dtype=torch.float32, device="cuda")
        job.set_model(c_init)
        df = w.dfreq
        set_data = {k: torch.stack([data_dev[q] for q in fset[k]]).contiguous() for k in range(total_steps)} if K > 1 else {}

        def one_update(k):
            if K > 1:
                return job.update_set([float(w.freqs[q]) for q in fset[k]], df, set_data[k])
            return job.update_frequency(float(w.freqs[fidx[k]]), df, data_dev[fidx[k]])

        for k in range(args.warmup):
            one_update(k)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        # single-frequency updates are queued back to back (rbx_update_frequency_async, one
        # stats slot each, with per-slot device timings), so host time between updates is not
        # in the timed region; frequency sets go through the synchronous rbx_update_set
        if K == 1:
            job.set_slot_timing(True)
        clocks = Clocks(local)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        stats = []
        for k in range(args.warmup, total_steps):
            if K == 1:
                job.update_frequency_async(float(w.freqs[fidx[k]]), df, data_dev[fidx[k]], (k - args.warmup) % 64)
            else:
                stats.append(one_update(k))
        ev1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        if K == 1:   # the last (up to 64) timed updates' scalars and device timings
            stats = [job.get_stats((k - args.warmup) % 64) for k in range(max(args.warmup, total_steps - 64), total_steps)]
            job.set_slot_timing(False)
        if args.log_jsonl and rank == 0:
            with open(args.log_jsonl, "a") as fh:
                for k, st in zip(range(total_steps - len(stats), total_steps), stats):
                    fq = [float(w.freqs[q]) for q in fset[k]] if K > 1 else float(w.freqs[fidx[k]])
                    fh.write(json.dumps({"step": k, "freq_hz": fq, **st}) + "\n")
        # image quality after the timed updates: RE of Sec. 6.4 on the mask, in percent
        m = g.mask()
        ct = np.asarray(w.c_true, dtype=np.float64)[m]
        den = np.linalg.norm(g.c0 - ct)
        re = {"initial": float(np.linalg.norm(np.asarray(w.c_init, np.float64)[m] - ct) / den * 100),
              "after_timed_updates": float(np.linalg.norm(job.get_model().cpu().numpy().astype(np.float64)[m] - ct)
                                           / den * 100)}
        ms = REP.max_over_ranks(ms, "cuda")
        if world > 1:
            dist.barrier()
        value = REP.aggregate_throughput(world * args.steps * K, ms / 1e3)

        # end to end through the host-buffer entry point: H2D of the step's data and D2H of the model
        e2e = None
        if not args.no_e2e and K == 1:
            job.set_model(c_init)
            c_host = torch.empty((g.ny, g.nx), dtype=torch.float32).pin_memory()
            for k in range(min(2, args.warmup)):
                job.update_frequency_host(float(w.freqs[fidx[k]]), df, data_host[fidx[k]], c_host)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            for k in range(args.warmup, total_steps):
                job.update_frequency_host(float(w.freqs[fidx[k]]), df, data_host[fidx[k]], c_host)
            torch.cuda.synchronize()
            el = REP.max_over_ranks(time.perf_counter() - t0, "cuda")
            e2e = {"value": REP.aggregate_throughput(world * args.steps, el), "unit": UNIT,
                   "h2d_bytes_per_step": N * N * 8,
                   "d2h_bytes_per_step": g.nx * g.ny * 4}
        # the allocation-free Born forward (rbx_forward_noalloc: Green's functions formed inside an
        # FP32 SIMT contraction, fixed scratch) beside rbx_forward on the same tables
        noalloc = None
        if not args.no_forms and world == 1 and N <= 1024:
            noalloc = time_noalloc(job, rbx, torch, g, float(w.freqs[fidx[0]]), stream)
        job.close()

    # the batched and served forms on the uneven slices (one GPU): the batched graph against the
    # plain per-job FP32 form, and the Poisson request stream with its serial FP32 replay
    serve, batched = None, None
    if not args.no_forms and world == 1:
        torch.cuda.empty_cache()
        pool = slice_pool(args.slices, rbx, P, torch)
        batched = batched_form(args, rbx, P, torch, pool=pool, steps=args.forms_steps, warmup=args.forms_warmup,
                               variants=("grouped_bf16", "graph_bf16", "sequential_bf16", "sequential_fp32"))
        torch.cuda.empty_cache()
        if args.requests > 0:
            serve = served_form(rbx, P, torch, pool, args.requests, args.rate, args.budget_gb * 1e9,
                                args.max_inflight, args.closed, not args.no_serial)
        del pool

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # per-kernel device time averaged over the timed steps; roofline of every kernel with an
    # algorithmic work figure, and of the dominant one
    kms = {k: float(np.mean([s["ms_kernel"][k] for s in stats])) for k in stats[0]["ms_kernel"]}
    if args.precision != "fp32" and args.integration != "raw":
        # one pass over the tables writes both contractions' operands (timed as the forward's)
        kms["synth"] = kms.pop("synth_fwd") + kms.pop("synth_bp")
    dom = max(kms, key=kms.get)
    pk = peaks()

    def roofline(kernel):
        amount, unit, bound = algorithmic(kernel, N, X, args.precision)
        if amount is None or kms.get(kernel, 0.0) <= 0.0:
            return None
        dur = kms[kernel] / 1e3
        if bound == "hbm":
            achieved, peak, u = amount / dur / 1e9, pk["hbm_gbs"], "GB/s"
        elif bound == "tensor":
            # the contractions run as ~2 ms bursts between SIMT kernels, below the power cap a
            # seconds-long GEMM loop reaches: the burst peak is theirs (the sustained one beside it)
            achieved, peak, u = amount / dur / 1e12, pk["bf16_tflops"], "TFLOP/s"
        else:
            achieved = amount / dur / 1e12
            peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
            u = "TFLOP/s"
        tr = NCU_TRAFFIC.get((args.workload, kernel))
        traffic = tr["bytes"] if tr and tr.get("src") == kernel_src_hash(kernel) else None
        r = {"kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak, "unit": u,
             "frac": achieved / peak, "traffic": traffic, "algorithmic_per_launch": amount, "ms": kms[kernel],
             "peak_source": ((pk["source"] + (" burst bf16" if bound == "tensor" else " copy bandwidth"))
                             if bound != "alu" else "FP32 SIMT: 152 SMs x 128 lanes x 2 flop x 2070 MHz")}
        if bound == "tensor":
            r["frac_of_sustained"] = achieved / pk["bf16_tflops_sustained"]
        return r

    roof = roofline(dom)
    roofs = [r for r in (roofline(k) for k in sorted(kms, key=kms.get, reverse=True)) if r is not None]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "bf16x3": "bf16x3"}[args.precision],
            "data": "synthetic (library ray-Born prediction on a seeded breast-like phantom + 40 dB noise)",
            "config": {"workload": describe(w), "mask_nodes": X, "precision": args.precision,
                       "absorption": ("breast map 0-1 dB/(MHz^1.4 cm), y=1.4" if args.absorption else "none"),
                       "integration": args.integration, "frequencies_per_update": K, "linking": args.link,
                       "l2": "inputs larger than L2 (tables N*X*16 B = %.2f GB)" % (16.0 * N * X / 1e9),
                       "parallelism": f"replicas x{world}",
                       "forward_k_split": tuning},
            "gpu_launches": int(round(np.mean([s["n_launches"] for s in stats]) * args.steps)),
            "clocks": clk, "e2e": e2e, "roofline": roof, "rooflines": roofs,
            "kernel_ms": kms, "stage_ms": {k: float(np.mean([s[k] for s in stats]))
                                           for k in ("ms_trace", "ms_forward", "ms_backproj", "ms_total")},
            "n_uncovered": int(stats[-1]["n_uncovered"]), "rms_dc_last": stats[-1]["rms_dc"],
            "relative_error_percent": re}
    if noalloc is not None:
        line["noalloc_forward"] = noalloc
    if batched is not None:
        line["forms"] = {
            "workload": f"{args.slices} uneven slices (N in {{256,512,768,1024}}, grids 192-512 at 0.45-1.0 mm, "
                        f"seeds 0-{args.slices - 1}), full 10-frequency sweeps, {batched['updates_per_step']} updates "
                        f"per step, {args.forms_warmup} warm-up + {args.forms_steps} timed steps",
            "grouped_bf16": batched["grouped_bf16"], "graph_bf16": batched["graph_bf16"],
            "sequential_bf16": batched["sequential_bf16"], "sequential_fp32": batched["sequential_fp32"],
            "graph_bf16_over_sequential_fp32": batched["graph_bf16_over_sequential_fp32"],
            "grouped_bf16_over_sequential_fp32": batched["grouped_bf16_over_sequential_fp32"],
            "kernel_share_bf16": batched.get("kernel_share_bf16"),
            "graph_equals_sequential_bf16": batched["graph_equals_sequential_bf16"],
            "rms_dc_grouped_vs_sequential_bf16_m_s": batched["rms_dc_grouped_vs_sequential_bf16_m_s"],
            "rms_dc_bf16_vs_fp32_m_s": batched["rms_dc_bf16_vs_fp32_m_s"],
            "detail": batched}
    if serve is not None:
        ol = serve["open_loop"]
        line["latency"] = {"p50_s": ol["p50_s"], "p99_s": ol["p99_s"], "from": "scheduled arrival",
                           "requests": serve["requests"], "rate_req_s": serve["rate_req_s"],
                           "updates_per_s": ol["updates_per_s"],
                           "workload": f"Poisson arrivals of 10-frequency sweeps drawn from {args.slices} uneven "
                                       "slices (N 256-1024, grids 192-512), BF16, served form"}
        if "serial_plain_fp32" in serve:
            sp = serve["serial_plain_fp32"]
            line["latency"]["serial_plain_fp32"] = {"p50_s": sp["p50_s"], "p99_s": sp["p99_s"],
                                                    "updates_per_s_busy": sp["updates_per_s_busy"]}
        if "closed_loop" in serve:
            line["latency"]["closed_loop_updates_per_s"] = serve["closed_loop"]["updates_per_s"]
        line["serve"] = serve
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_full_update(w, float(w.freqs[0]), noisy[uniq.index(0)])
        cb.pop("seconds_per_update", None)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
