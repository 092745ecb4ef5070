"""Host logic of bench.py's roofline accounting (CPU only): the algorithmic work per launch
of each timed kernel, and the source keys of the recorded DRAM traffic."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_work_per_kernel():
    b = bench()
    N, X = 1024, 152088
    NX = N * X
    assert b.algorithmic("gemm_bp", N, X, "bf16") == (8.0 * 2 * X * N * N, "flop", "tensor")
    assert b.algorithmic("gemm_bp", N, X, "fp32")[2] == "alu"
    assert b.algorithmic("gemm_fwd", N, X, "bf16") == (8.0 * N * (N + 1) / 2 * X, "flop", "tensor")
    assert b.algorithmic("trace", N, X, "bf16") == (16.0 * NX + 16.0 * N * (N - 1), "byte", "hbm")
    # one pass over the tables writes 4 forward and 6 back-projection BF16 planes (twice when split)
    assert b.algorithmic("synth", N, X, "bf16") == ((16.0 + 20.0) * NX, "byte", "hbm")
    assert b.algorithmic("synth", N, X, "bf16x3") == ((16.0 + 40.0) * NX, "byte", "hbm")
    assert b.algorithmic("synth_bp", N, X, "fp32") == ((16.0 + 20.0) * NX, "byte", "hbm")
    assert b.algorithmic("tables", N, X, "bf16")[0] == 16.0 * N * (N - 1) + 8.0 * N * N
    assert b.algorithmic("unknown", N, X, "bf16") == (None, None, None)


def test_recorded_traffic_is_keyed_to_kernel_sources():
    b = bench()
    for (workload, kernel), rec in b.NCU_TRAFFIC.items():
        assert kernel in b.KERNEL_SRC
        assert rec["bytes"] > 0 and len(rec["src"]) == 12
        assert b.kernel_src_hash(kernel) == b.kernel_src_hash(kernel)      # deterministic
