"""Host logic of bench.py (no GPU): clock-sample summaries and throttle reasons,
the traffic record's source-hash gate, replica throughput."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary(bench):
    lines = [
        "0, 2070, 2070, 700.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1399.9, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 10, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = bench.ClockSampler.summarize(lines)
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = bench.ClockSampler.summarize([
        "0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize(["garbage"]) is None
    assert bench.ClockSampler.summarize([]) is None


def test_traffic_only_for_the_profiled_kernel_source_and_shape(bench, monkeypatch):
    rec = bench.NCU_TRAFFIC[("sel16", "f64", "k_sigma")]
    monkeypatch.setattr(bench, "_source_hash", lambda name: rec["sha1"])
    shapes = rec["shapes"]

    def counts(threads, nv, stage):
        return {"tuned_threads": [threads, 0], "tuned_nv": [nv, 0], "tuned_stage": [stage, 0]}

    # the captured shape: three vectors in one launch
    assert bench._traffic("sel16", "f64", "k_sigma", counts(512, 3, 2), 3) == pytest.approx(shapes[(512, 3, 2)])
    # three vectors in groups of two need the shapes of a 2-vector and a 1-vector launch
    two = dict(shapes)
    two[(512, 2, 2)], two[(512, 1, 2)] = 4.0e9, 1.0e9
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("sel16", "f64", "k_sigma"), dict(rec, shapes=two))
    assert bench._traffic("sel16", "f64", "k_sigma", counts(512, 2, 2), 3) == pytest.approx(2.5e9)
    monkeypatch.setitem(bench.NCU_TRAFFIC, ("sel16", "f64", "k_sigma"), rec)
    assert bench._traffic("sel16", "f64", "k_sigma", counts(256, 3, 2), 3) is None  # shape not captured
    assert bench._traffic("sel16", "f64", "k_sigma", counts(512, 0, 2), 3) is None  # not tuned
    assert bench._traffic("fci16", "f64", "k_sigma", counts(512, 1, 0), 1) is None  # workload not captured
    assert bench._traffic("sel16", "f64", "k_sigma_parts", counts(512, 1, 3), 1) is None  # kernel not captured
    monkeypatch.setattr(bench, "_source_hash", lambda name: "0" * 40)
    assert bench._traffic("sel16", "f64", "k_sigma", counts(512, 3, 2), 3) is None  # source changed since
    assert bench._traffic("sel16", "bf16tc", "k_sigma", counts(512, 3, 2), 3) is None


def test_kernel_table_shares_and_fractions(bench):
    """Per-kernel rows from a synthetic trace of two split-path steps: shares sum
    to one, the row kernel's work counts the diagonal, single and alpha-beta
    classes, and the transposes are measured against HBM."""
    c = {"la": 100, "lb": 200, "ndet": 20000, "nnz": 0, "n1a": 300, "n2a": 900, "n1b": 500, "n2b": 1100,
         "norb": 10}
    step = [("k_transpose", 1.0), ("k_dbl_spmm_beta", 4.0), ("k_sigma_parts", 10.0), ("k_combine", 1.0),
            ("k_dbl_spmm_alpha", 4.0)]
    rows = bench._kernel_table(step * 2, 2, c, 1, "f64")
    assert [r["kernel"] for r in rows][0] == "k_sigma_parts"
    assert sum(r["share"] for r in rows) == pytest.approx(1.0)
    k1 = rows[0]
    assert k1["launches_per_step"] == 1 and k1["ms_per_launch"] == 10.0
    assert k1["work_per_launch"] == 2.0 * (20000 + 300 * 200 + 500 * 100 + 300 * 500)
    assert k1["achieved"] == pytest.approx(k1["work_per_launch"] / 1e-2 / 1e12)
    assert k1["frac"] == pytest.approx(k1["achieved"] / bench.FP64_NOMINAL_TFLOPS)
    tr = [r for r in rows if r["kernel"] == "k_transpose"][0]
    assert tr["bound"] == "hbm" and tr["work_per_launch"] == 2 * 20000 * 8
    beta = [r for r in rows if r["kernel"] == "k_dbl_spmm_beta"][0]
    assert beta["work_per_launch"] == 2.0 * 1100 * 100

def test_replica_throughput_and_single_rank_max(bench):
    assert bench.replica_throughput(2, 9e6, 0.5) == pytest.approx(3.6e7)
    assert bench.max_over_ranks(1.25) == 1.25


def test_clock_sampler_start_stop_with_a_stand_in_tool(bench, tmp_path, monkeypatch):
    """The sampler's process handling end to end: a stand-in `nvidia-smi` on PATH
    prints three samples and waits; stop() terminates it and summarises."""
    tool = tmp_path / "nvidia-smi"
    tool.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 600, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2040, 2070, 900, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2070, 2070, 950, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    tool.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    import time
    s = bench.ClockSampler(0)
    s.start()
    deadline = time.time() + 10
    while len(s.lines) < 3 and time.time() < deadline:
        time.sleep(0.05)
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert s.proc.poll() is not None  # the tool was terminated


def test_kernel_table_tensor_and_unmodelled_kernels(bench):
    """The tensor-core alpha-beta kernel is measured against the tensor peak (the
    TF32 type at half the BF16 peak), the column-tiled beta product of the
    tensor-core types counts the beta singles too, and a kernel without an
    algorithmic model (the cuBLAS products of rest mode 5) reports no fraction."""
    c = {"la": 64, "lb": 64, "ndet": 4096, "nnz": 0, "n1a": 640, "n2a": 1000, "n1b": 640, "n2b": 1000,
         "norb": 8}
    trace = [("k_sigma_ab_tc", 2.0), ("k_dbl_spmm_beta", 1.0), ("gemm_same_spin", 0.5)]
    rows = {r["kernel"]: r for r in bench._kernel_table(trace, 1, c, 1, "tf32tc")}
    tc = rows["k_sigma_ab_tc"]
    assert tc["bound"] == "tensor" and tc["work_per_launch"] == 2.0 * 28 * 640 * 64
    bf = bench._measured_peaks().get("bf16_tflops", 1900.0)
    assert tc["peak"] == pytest.approx(0.5 * bf)
    assert rows["k_dbl_spmm_beta"]["work_per_launch"] == 2.0 * (1000 + 640) * 64
    g = rows["gemm_same_spin"]
    assert g["work_per_launch"] is None and g["achieved"] is None and g["frac"] is None

