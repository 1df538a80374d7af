"""Benchmark: sigma = H.c throughput (GDet/s) on one GB300, plus Davidson time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]
                    [--workload sel24|sel16|fci8|fci16] [--dtype f64|f32|tf32tc|bf16tc]

A step is one sigma evaluation of ``nvec`` vectors over the whole space (all of
its Slater-Condon classes). The default workload is the largest single-GPU one:
norb=24, 12+12 electrons, 40,000 x 40,000 selected strings (1.6B determinants),
FP64, 1 vector -- 12.8 GB of input and 12.8 GB of output per step, both far
larger than the 129 MB L2, so no flush is needed between steps.

value  = nvec * ndet / (device time per step) / 1e9, timed with CUDA events on
         the launching stream after W warm-up steps, max over ranks.
e2e    = the same metric through tbsci_sigma_host with pinned host buffers:
         host->device copy of c and device->host copy of sigma inside the timed
         region.
roofline = the kernel with the largest share of the step (the fused sigma
         kernel, or the split path's row kernel) against the FP64 ALU (2 flops
         per non-zero H_IJ of the classes it computes, per vector), the FP32
         ALU, the tensor cores or HBM; its launch time comes from the library's
         kernel trace (CUDA events around each launch on its stream).
         roofline.step gives the whole step the same way, and `kernels` every
         kernel of the step.
cpu_baseline = the CPU oracle timed on a bounded row sample of the same
         workload on this host's cores (rank 0, N = 1 only).
sel16_sigma = the same measurement on norb=16, 3,000 x 3,000 selected strings
         (9.0M determinants), FP64, 3 vectors.
davidson = Davidson time to 1e-9 / 1e-5 on the 9.0M-determinant space, FP64,
         mixed precision with FP32 sigma, and mixed precision with the split-TF32
         tensor-core sigma.
serving = the 512-request stream replayed live at twice the FP64 sequential
         service rate through a one-slot FP64 server and through the
         mixed-precision batching server: p50 / p99 latency, throughput and the
         energy difference of every result (--no-serving skips it).
--impl reference runs the oracle alone as the reference arm.

Under torchrun (N > 1) every rank runs an independent replica (the path does
not shard); value sums the ranks' work over the max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from tbsci_inputs import WORKLOADS, random_vectors, selected_strings  # noqa: E402

METRIC = "σ GDet/s and Davidson time to 1e-8 Eh; serving p50/p99 vs plain FP64 on GB300"
UNIT = "GDet/s"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 dense FP64 (recipe nominal)
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 128 FP32 lanes/SM/clk, FMA = 2 flops


# DRAM bytes (read + write) per launch, by workload, dtype and kernel, at a launch
# shape, from one ncu capture of the kernel source file with this sha1 (the
# captures are summarised in the kernels' profiles); a workload, shape or source
# not captured reports null. Shapes: k_sigma (threads, vectors per CTA,
# shared-memory mode); k_sigma_parts (threads, stage).
NCU_TRAFFIC = {
    ("sel16", "f64", "k_sigma"): {
        "source": "sigma.cu", "sha1": "2e38dd72db29d3137f5f54aee410b1a51db79613",
        "shapes": {(512, 3, 2): 21.10e9}},
    ("sel24", "f64", "k_sigma_parts"): {
        "source": "sigma_split.cu", "sha1": "bbca57e694e9aafe0b9476961be6286e724c7b3a",
        "shapes": {(1024, 3): 380.95e9}},
}


def _source_hash(name):
    import hashlib
    with open(os.path.join(ROOT, "paper_2503_10335_gb300", "csrc", name), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def _traffic(workload, dtype, kernel, counts, nvec=1):
    """Average DRAM bytes per launch of `kernel` in one step at the tuned shape,
    or None. k_sigma runs nvec vectors in launch groups of the tuned vectors per
    CTA (the last group smaller); the other kernels take one vector a launch."""
    rec = NCU_TRAFFIC.get((workload, dtype, kernel))
    if not rec or rec["sha1"] != _source_hash(rec["source"]):
        return None
    t = 0 if dtype == "f64" else 1
    threads, nv, stage = counts["tuned_threads"][t], counts["tuned_nv"][t], counts["tuned_stage"][t]
    if kernel != "k_sigma":
        return rec["shapes"].get((threads, stage))
    if nv < 1:
        return None
    groups = [min(nv, nvec - v) for v in range(0, nvec, nv)]
    try:
        return sum(rec["shapes"][(threads, g, stage)] for g in groups) / len(groups)
    except KeyError:
        return None


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _kernel_work(name, c, nvec, dtype):
    """Algorithmic work of one step for the launches of kernel `name`:
    (amount, kind, rule); kind is "fp" (flops on the ALU), "tensor" (flops on
    the tensor cores) or "bytes" (HBM)."""
    la, lb, nd = c["la"], c["lb"], c["ndet"]
    elem = 8 if dtype == "f64" else 4
    tc = dtype in ("tf32tc", "bf16tc")
    if name in ("k_sigma", "k_sigma_batch"):
        return 2.0 * c["nnz"] * nvec, "fp", "2 flops per non-zero H_IJ per vector"
    if name == "k_sigma_parts":
        return (2.0 * (nd + c["n1a"] * lb + c["n1b"] * la + c["n1a"] * c["n1b"]) * nvec, "fp",
                "2 flops per non-zero of the diagonal, single and alpha-beta classes per vector")
    if name == "k_dbl_spmm_alpha":
        return 2.0 * c["n2a"] * lb * nvec, "fp", "2 flops per non-zero of the alpha doubles per vector"
    if name == "k_dbl_spmm_beta":
        n = c["n2b"] + (c["n1b"] if tc else 0)
        return 2.0 * n * la * nvec, "fp", "2 flops per non-zero of the beta %s per vector" % (
            "singles and doubles" if tc else "doubles")
    if name in ("k_sigma_rest", "k_sigma_rest_pair"):
        return (2.0 * ((c["n1b"] + c["n2b"]) * la + c["n2a"] * lb) * nvec, "fp",
                "2 flops per non-zero of the beta singles and doubles and the alpha doubles per vector")
    if name == "k_sigma_ab_tc":
        noff = c["norb"] * (c["norb"] - 1) // 2
        return (2.0 * noff * c["n1a"] * lb * nvec, "tensor",
                "2 flops per (alpha single, off-diagonal pair kl, beta column) of the dense contraction per vector")
    if name == "k_transpose":
        return None, "bytes", "read + write of one vector"
    if name == "k_combine":
        return None, "bytes", "two vectors read, one written"
    return None, "fp", "not modelled"


def _kernel_table(trace, steps, c, nvec, dtype):
    """Per-kernel launches, device time and roofline fraction of the timed steps
    (from the library's kernel trace)."""
    peaks = _measured_peaks()
    elem = 8 if dtype == "f64" else 4
    by = {}
    for name, ms in trace:
        by.setdefault(name, []).append(ms)
    total = sum(sum(v) for v in by.values()) or 1.0
    out = []
    for name, v in by.items():
        launches = len(v) / steps
        mean = statistics.mean(v)
        work_step, kind, rule = _kernel_work(name, c, nvec, dtype)
        if kind == "bytes":
            per = (2 if name == "k_transpose" else 3) * c["ndet"] * elem
            peak, unit = peaks.get("hbm_gbs", 6800.0), "GB/s"
            src = "HBM copy of measured" if "hbm_gbs" in peaks else "HBM of fallback (6.8 TB/s)"
            achieved = per / (mean * 1e-3) / 1e9
            bound = "hbm"
        elif kind == "tensor":
            per = work_step / launches
            bf = peaks.get("bf16_tflops", 1900.0)
            peak = bf * (0.5 if dtype == "tf32tc" else 1.0)
            unit, bound = "TFLOP/s", "tensor"
            src = ("BF16 burst of measured" if "bf16_tflops" in peaks else "BF16 of fallback") + (
                " x 0.5 (nominal TF32 : BF16)" if dtype == "tf32tc" else "")
            achieved = per / (mean * 1e-3) / 1e12
        else:
            per = work_step / launches if work_step is not None else None
            peak = FP64_NOMINAL_TFLOPS if dtype == "f64" else FP32_NOMINAL_TFLOPS
            unit, bound = "TFLOP/s", "alu"
            src = "%s ALU derived from unit counts and clocks (152 SMs x %s per clock x 2070 MHz)" % (
                ("FP64", "2 DFMA") if dtype == "f64" else ("FP32", "128 FFMA"))
            achieved = per / (mean * 1e-3) / 1e12 if per is not None else None
        out.append({"kernel": name, "launches_per_step": launches, "ms_per_launch": mean,
                    "ms_per_step": sum(v) / steps, "share": sum(v) / total, "bound": bound,
                    "work_per_launch": per, "rule": rule, "achieved": achieved, "peak": peak, "unit": unit,
                    "frac": achieved / peak if achieved is not None else None, "peak_source": src})
    out.sort(key=lambda r: -r["ms_per_step"])
    return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, max clock and the throttle reasons seen in nvidia-smi CSV
        lines (FIELDS order, no header or units); None without a usable sample."""
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def max_over_ranks(value: float, dist_mod=None, device="cpu") -> float:
    """The slowest rank's time (replicas run independently; the job ends with the last)."""
    if dist_mod is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world_size: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput of independent replicas: every rank's units over the max time."""
    return world_size * units_per_rank / max_seconds


def _oracle_space(wl, count_alpha=None):
    import oracle
    asel = wl.alpha_selection()
    if count_alpha is not None:
        asel = selected_strings(wl.norb, wl.nalpha, count_alpha, wl.seed_sel)
    return oracle.make_space(wl.norb, wl.nalpha, wl.nbeta, asel, wl.beta_selection())


def _host_vector(nvec, ndet, seed):
    """A seeded host vector [nvec, ndet] for timing the oracle (uniform in
    [-0.5, 0.5): drawing 1.6B normal deviates would take longer than the timing)."""
    c = np.random.default_rng(seed).random((nvec, ndet))
    c -= 0.5
    return c


def cpu_baseline(wl, nvec, budget_s=15.0, C=None, count_alpha=None):
    """Oracle sigma over a bounded, seeded row sample of the workload; C is the
    host copy [nvec, ndet] of the vector the GPU leg used (drawn here if None)."""
    import oracle
    h, eri, ecore = wl.hamiltonian()
    sp = _oracle_space(wl, count_alpha)
    if C is None:
        C = _host_vector(nvec, sp.ndet, wl.seed_vec)
    rng = np.random.default_rng(wl.seed_vec + 17)
    # calibrate on a small sample, then size the measured sample to the budget
    probe = rng.choice(sp.ndet, 500, replace=False)
    t0 = time.perf_counter()
    oracle.sigma(sp, h, eri, ecore, C, rows=probe)
    rate = 500 / max(time.perf_counter() - t0, 1e-6)
    nrows = int(min(sp.ndet, max(1000, rate * budget_s)))
    rows = rng.choice(sp.ndet, nrows, replace=False)
    t0 = time.perf_counter()
    oracle.sigma(sp, h, eri, ecore, C, rows=rows)
    dt = time.perf_counter() - t0
    return {"value": nrows * nvec / dt / 1e9, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": "%d seeded determinant rows of %d (%d vectors), %.1f s" % (nrows, sp.ndet, nvec, dt),
            "seconds": dt, "rows": nrows}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload]
    nvec = wl.nvec
    h, eri, ecore = wl.hamiltonian()
    sp = _oracle_space(wl, args.count_alpha)
    C = _host_vector(nvec, sp.ndet, wl.seed_vec)
    rng = np.random.default_rng(wl.seed_vec + 29)
    rows_per_step = args.ref_rows
    if rows_per_step <= 0:  # about 2 s of oracle work per step
        probe = rng.choice(sp.ndet, 500, replace=False)
        t0 = time.perf_counter()
        oracle.sigma(sp, h, eri, ecore, C, rows=probe)
        rows_per_step = int(max(1000, 2.0 * 500 / max(time.perf_counter() - t0, 1e-6)))
    rows_per_step = min(sp.ndet, rows_per_step)
    for _ in range(args.warmup):
        oracle.sigma(sp, h, eri, ecore, C, rows=rng.choice(sp.ndet, rows_per_step, replace=False))
    times = []
    for _ in range(args.steps):
        rows = rng.choice(sp.ndet, rows_per_step, replace=False)
        t0 = time.perf_counter()
        oracle.sigma(sp, h, eri, ecore, C, rows=rows)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = rows_per_step * nvec * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(_config(wl, nvec, "f64", la=sp.la, lb=sp.lb), parallelism="replicas" if ws > 1 else "single"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": "%d seeded determinant rows per step of %d, %d vectors" %
                                   (rows_per_step, sp.ndet, nvec)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(wl, nvec, dtype, la=None, lb=None):
    if la is None:
        la = math.comb(wl.norb, wl.nalpha) if wl.count_alpha is None else min(wl.count_alpha,
                                                                               math.comb(wl.norb, wl.nalpha))
    if lb is None:
        lb = math.comb(wl.norb, wl.nbeta) if wl.count_beta is None else min(wl.count_beta,
                                                                             math.comb(wl.norb, wl.nbeta))
    name = wl.notes if (la, lb) == _config_default_sizes(wl) else \
        "norb=%d, %d+%d electrons, %d x %d selected strings (%.1fM determinants; a smaller case of %s)" % (
            wl.norb, wl.nalpha, wl.nbeta, la, lb, la * lb / 1e6, wl.name)
    return {"workload": name, "name": wl.name, "norb": wl.norb, "nalpha": wl.nalpha, "nbeta": wl.nbeta,
            "l_alpha": la, "l_beta": lb, "ndet": la * lb, "nvec": nvec, "sigma_dtype": dtype,
            "l2_policy": "inputs larger than L2 (no flush)" if la * lb * nvec * (8 if dtype == "f64" else 4) > 129e6
            else "inputs smaller than L2 (not flushed; not a headline configuration)"}


def _config_default_sizes(wl):
    la = math.comb(wl.norb, wl.nalpha) if wl.count_alpha is None else min(wl.count_alpha,
                                                                           math.comb(wl.norb, wl.nalpha))
    lb = math.comb(wl.norb, wl.nbeta) if wl.count_beta is None else min(wl.count_beta,
                                                                         math.comb(wl.norb, wl.nbeta))
    return la, lb


def _serving_requests(nreq, seed, max_count):
    """The serving stream's requests (host data), in arrival order."""
    from tbsci_inputs import selected_strings, serving_stream, synth_hamiltonian
    reqs = []
    for r in serving_stream(nreq=nreq, seed=seed, rate_hz=1.0, hi=max_count):
        h, eri, ecore = synth_hamiltonian(r["norb"], r["seed_ints"])
        sel = selected_strings(r["norb"], r["nelec"], r["count"], r["seed_sel"])
        reqs.append(dict(norb=r["norb"], nalpha=r["nelec"], nbeta=r["nelec"], h=h, eri=eri, ecore=ecore,
                         alpha=sel, beta=sel, nroots=r["nroots"], gap=r["t_arrival"]))
    return reqs


def _replay(tb, reqs, arrivals, mixed, **server_kw):
    """Submits every request at its arrival time (seconds from the start) to a new
    server and waits for all results. Returns (results, makespan seconds)."""
    srv = tb.Server(0, **server_kw)
    t0 = time.perf_counter()
    tickets = []
    try:
        for r, a in zip(reqs, arrivals):
            delay = a - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            kw = {k: r[k] for k in ("norb", "nalpha", "nbeta", "h", "eri", "ecore", "alpha", "beta", "nroots")}
            tickets.append(srv.submit(mixed=mixed, **kw))
        res = []
        for t in tickets:
            st, d = srv.poll(t, timeout_ms=-1)
            res.append(d)
        makespan = time.perf_counter() - t0
    finally:
        srv.close()
    return res, makespan


def _latency_summary(res, makespan):
    lat = [d["t_done"] - d["t_submit"] for d in res]
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat)), "throughput_per_s": len(res) / makespan, "makespan_s": makespan,
            "statuses": sorted(set(int(d["status"]) for d in res))}


def run_serving(args, print_line=True):
    """Serving stream (Poisson arrivals, norb 8..16, 50..max strings per spin, 1-3
    roots): plain FP64 one-at-a-time (a one-slot server, unbatched, FP64 sigma)
    against the mixed-precision continuous-batching server, both fed the same
    arrival timestamps live, at arrival rates that are multiples of the FP64
    sequential service rate (calibrated on the first requests of the stream)."""
    import torch
    import paper_2503_10335_gb300 as tb
    reqs = _serving_requests(args.nreq, 5005, args.max_count)
    ncal = min(len(reqs), args.calibrate)
    ctx = tb.Context(0)
    # calibration: FP64 one-at-a-time service times (set-up + solve through the C ABI)
    service = []
    for r in reqs[:ncal]:
        t0 = time.perf_counter()
        sp = tb.Space(ctx, r["norb"], r["nalpha"], r["nbeta"], r["h"], r["eri"], r["ecore"], alpha=r["alpha"],
                      beta=r["beta"])
        sp.davidson(r["nroots"])
        torch.cuda.synchronize()
        service.append(time.perf_counter() - t0)
        sp.close()
    ctx.close()
    mu = ncal / sum(service)
    base = np.array([r["gap"] for r in reqs])  # unit-rate Poisson arrival times
    out = {"metric": METRIC, "mode": "serving", "nreq": len(reqs), "max_strings": args.max_count,
           "fp64_service_rate_per_s": mu, "calibration_requests": ncal, "rates": []}
    for mult in [float(x) for x in args.rates.split(",")]:
        lam = mult * mu
        arrivals = base / lam
        r64, m64 = _replay(tb, reqs, arrivals, False, max_active=1, fuse_sigma=-1)
        rmx, mmx = _replay(tb, reqs, arrivals, args.serving_mixed)
        diffs = [float(np.max(np.abs(np.array(a["energies"]) - np.array(b["energies"])))) for a, b in zip(rmx, r64)]
        out["rates"].append({
            "arrival_rate_per_s": lam, "x_fp64_rate": mult,
            "fp64_one_at_a_time": _latency_summary(r64, m64),
            "mixed_batched": dict(_latency_summary(rmx, mmx), sigma_mode=args.serving_mixed),
            "energy_diff_vs_fp64_Eh": {"max": max(diffs), "p50": float(np.median(diffs))}})
    if print_line:
        print(json.dumps(out), flush=True)
    return out


def run_selection_study(args):
    """Bitstring selection loop (Sec. III.B) and coefficient distributions (Fig. 3)
    on a synthetic Hamiltonian with the recipe's two-electron scale 0.1 (the
    default 0.3 spreads the ground-state weight evenly over the strings): the
    full string space of norb 14, 7+7 electrons (11.8M determinants) is solved,
    its strings are weighed and selected at each delta, and each selected TPB
    space is solved again. Reports sizes, energies (and their distance from the
    full-space energy), solve times and the |c_K / c_HF| histograms."""
    import torch
    import paper_2503_10335_gb300 as tb
    from tbsci_inputs import synth_hamiltonian
    n, N = args.sel_norb, args.sel_norb // 2
    h, eri, ecore = synth_hamiltonian(n, seed=1014, scale=0.1)
    ctx = tb.Context(0)
    full = tb.Space(ctx, n, N, N, h, eri, ecore)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_full, info, X = full.davidson(1, want_vectors=True, mixed=1)
    t_full = time.perf_counter() - t0
    c0 = X[0].contiguous()
    c_hf = float(torch.max(torch.abs(c0)))
    ratios, counts = full.coefficient_histogram(c0, c_hf, lo=-12, hi=0)
    out = {"metric": METRIC, "mode": "selection_study", "norb": n, "nelec": [N, N], "two_electron_scale": 0.1,
           "full": {"ndet": full.ndet, "energy": float(e_full[0]), "seconds": t_full,
                    "iterations": info["iterations"], "histogram": counts.tolist()},
           "bin_edges_c_over_c_hf": ratios.tolist(), "runs": []}
    for delta in [float(x) for x in args.deltas.split(",")]:
        ka, kb = full.select_by_weight(c0, delta)
        sub = tb.Space(ctx, n, N, N, h, eri, ecore, alpha=ka, beta=kb)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e, inf, Xs = sub.davidson(1, want_vectors=True, mixed=1)
        dt = time.perf_counter() - t0
        xs = Xs[0].contiguous()
        _, hs = sub.coefficient_histogram(xs, float(torch.max(torch.abs(xs))), lo=-12, hi=0)
        out["runs"].append({"delta": delta, "n_alpha": len(ka), "n_beta": len(kb), "ndet": sub.ndet,
                            "fraction_of_full": sub.ndet / full.ndet, "energy": float(e[0]),
                            "minus_full_Eh": float(e[0] - e_full[0]), "seconds": dt,
                            "iterations": inf["iterations"], "histogram": hs.tolist()})
        sub.close()
        del Xs, xs
    full.close()
    ctx.close()
    print(json.dumps(out), flush=True)


def run_precision_study(args):
    """Davidson on one workload with every low-precision sigma type: the energy
    reached by the low-precision phase, its error against the final FP64-refined
    energy, sigma counts and wall time per mode."""
    import torch
    import paper_2503_10335_gb300 as tb
    wl = WORKLOADS[args.workload]
    h, eri, ecore = wl.hamiltonian()
    ctx = tb.Context(0)
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=wl.alpha_selection(),
                  beta=wl.beta_selection())
    names = {0: "f64", 1: "f32", 2: "f32+tf32x3 tensor", 3: "f32+bf16 tensor"}
    modes = [int(x) for x in args.modes.split(",")]
    tuned = {}
    if not args.no_autotune:
        # set-up, untimed: launch shapes of the SIMT sigma kernels the solves use
        g = torch.Generator(device="cuda").manual_seed(wl.seed_vec)
        for dt, tdt, name in ((tb.TBSCI_F32, torch.float32, "f32"), (tb.TBSCI_F32_TC_TF32, torch.float32, "tc"),
                              (tb.TBSCI_F64, torch.float64, "f64")):
            if dt == tb.TBSCI_F32 and 1 not in modes:
                continue
            if dt == tb.TBSCI_F32_TC_TF32 and not any(m in (2, 3) for m in modes):
                continue  # one tuning serves both tensor-core types (same SIMT pass)
            C = torch.randn((1, sp.la, sp.lb), generator=g, device="cuda", dtype=torch.float32).to(tdt)
            S = torch.empty_like(C)
            tuned[name + "_sigma_ms"] = tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, S, 1, dt)
            del C, S
        torch.cuda.empty_cache()
    out = {"metric": METRIC, "mode": "precision_study", "workload": wl.notes, "ndet": sp.ndet,
           "nroots": wl.nroots, "counts": sp.counts(), "autotuned_sigma_ms": tuned, "runs": []}
    for m in modes:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e, info = sp.davidson(wl.nroots, mixed=m, max_iter=args.max_iter, check=False,
                              basis_f32=bool(args.basis_f32 and m), max_subspace=args.max_subspace,
                              restart_keep=args.restart_keep)
        dt = time.perf_counter() - t0
        e_low = info["energy_f32"][:wl.nroots] if m else None
        out["runs"].append({"sigma": names[m], "basis": "f32" if (args.basis_f32 and m) else "f64",
                            "seconds": dt, "iterations": info["iterations"],
                            "iterations_lowp": info["iterations_f32"], "nsigma": info["nsigma"],
                            "nsigma_lowp": info["nsigma_f32"], "energies": [float(x) for x in e],
                            "converged": info["converged"], "status": info["status"],
                            "seconds_sigma": info["seconds_sigma"],
                            "seconds_sigma_lowp": info["seconds_sigma_f32"],
                            "energy_lowp_phase": e_low,
                            "lowp_phase_error_Eh": (max(abs(a - b) for a, b in zip(e_low, e)) if m else 0.0)})
    ref = out["runs"][0]["energies"]
    for r in out["runs"]:
        r["final_vs_first_mode_Eh"] = max(abs(a - b) for a, b in zip(r["energies"], ref))
    sp.close()
    ctx.close()
    print(json.dumps(out), flush=True)


def _sigma_leg(tb, ctx, wl, dtype, nvec, steps, warmup, dev, stream, autotune=True, clocks=False,
               count_alpha=None):
    """Times `steps` sigma evaluations of `nvec` vectors on one workload (device
    buffers, CUDA events on the launching stream). Returns the leg's record and
    the space with its device vectors (for the callers' e2e and baseline legs)."""
    import torch
    h, eri, ecore = wl.hamiltonian()
    asel = wl.alpha_selection()
    if count_alpha is not None:
        asel = selected_strings(wl.norb, wl.nalpha, count_alpha, wl.seed_sel)
    t_setup = time.perf_counter()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=asel, beta=wl.beta_selection())
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    tdt = torch.float64 if dtype == "f64" else torch.float32
    sdt = {"f64": tb.TBSCI_F64, "f32": tb.TBSCI_F32, "tf32tc": tb.TBSCI_F32_TC_TF32,
           "bf16tc": tb.TBSCI_F32_TC_BF16}[dtype]
    g = torch.Generator(device=dev).manual_seed(wl.seed_vec)
    C = torch.randn((nvec, sp.la, sp.lb), generator=g, device=dev, dtype=torch.float64).to(tdt)
    S = torch.empty_like(C)
    tuned_ms = None
    if autotune:
        # set-up, untimed: pick the launch shape of the SIMT kernel for this space
        tuned_ms = tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, S, nvec, sdt, stream)
    for _ in range(warmup):
        sp.sigma(C, S, stream=stream, dtype=sdt)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index) if clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    # the library's kernel trace brackets each of its launches with events on
    # the launching stream: per-kernel device times of the timed steps
    tb.tbsci_trace_read(ctx.handle)
    tb.tbsci_trace_enable(ctx.handle, True)
    ev[0].record(stream)
    for k in range(steps):
        sp.sigma(C, S, stream=stream, dtype=sdt)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    tb.tbsci_trace_enable(ctx.handle, False)
    trace, dropped = tb.tbsci_trace_read(ctx.handle)
    clk = sampler.stop() if sampler else None
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    counts = sp.counts()  # after tuning: carries the chosen launch shape
    n1a, n2a = tb.tbsci_tables_counts(sp.ta)
    n1b, n2b = tb.tbsci_tables_counts(sp.tb)
    kernels = _kernel_table(trace, steps, dict(counts, n1a=n1a, n2a=n2a, n1b=n1b, n2b=n2b, la=sp.la, lb=sp.lb,
                                               norb=wl.norb), nvec, dtype)
    dom = max(kernels, key=lambda r: r["ms_per_step"])
    step_flops = 2.0 * counts["nnz"] * nvec
    traffic = _traffic(wl.name, dtype, dom["kernel"], counts, nvec)
    roofline = {"bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"], "unit": dom["unit"],
                "frac": dom["frac"], "traffic": traffic, "kernel": dom["kernel"],
                "launches_per_step": dom["launches_per_step"], "ms_per_launch": dom["ms_per_launch"],
                "share_of_step": dom["share"], "peak_source": dom["peak_source"],
                "algorithmic_per_launch": dom["work_per_launch"], "algorithmic_rule": dom["rule"],
                "timing": "library kernel trace: CUDA events around each launch on its stream, timed steps",
                "step": {"achieved": step_flops / (total_ms / steps * 1e-3) / 1e12, "unit": "TFLOP/s",
                         "peak": FP64_NOMINAL_TFLOPS if dtype == "f64" else FP32_NOMINAL_TFLOPS,
                         "rule": "2 flops per non-zero H_IJ per vector over the whole step"}}
    roofline["step"]["frac"] = roofline["step"]["achieved"] / roofline["step"]["peak"]
    launches_per_step = len(trace) / steps if steps else 0
    rec = {"value": nvec * sp.ndet / (total_ms / steps * 1e-3) / 1e9, "ms_per_step": total_ms / steps,
           "step_ms_min": min(per_step), "step_ms_max": max(per_step), "roofline": roofline,
           "kernels": kernels, "trace_dropped": dropped, "gpu_launches": len(trace),
           "launches_per_step": launches_per_step, "counts": counts, "setup_seconds": t_setup,
           "autotune_ms": tuned_ms, "config": _config(wl, nvec, dtype, la=sp.la, lb=sp.lb), "clocks": clk}
    return rec, sp, C, S, sdt


def _e2e_leg(tb, ctx, sp, C, nvec, steps, world):
    """The same metric through tbsci_sigma_host with pinned HOST buffers: the
    host->device copy of c and the device->host copy of sigma are inside the
    timed region of every step. Returns the record and the pinned host c."""
    import torch
    hc = C.cpu().pin_memory()
    hs = torch.empty_like(hc).pin_memory()
    hcn, hsn = hc.numpy(), hs.numpy()
    tb.tbsci_sigma_host(ctx.handle, sp.ham, sp.ta, sp.tb, hcn, hsn, nvec)  # warm the device buffers
    t0 = time.perf_counter()
    for _ in range(steps):
        tb.tbsci_sigma_host(ctx.handle, sp.ham, sp.ta, sp.tb, hcn, hsn, nvec)
    dt = (time.perf_counter() - t0) / steps
    nbytes = nvec * sp.ndet * 8
    del hs
    return ({"value": world * nvec * sp.ndet / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": nbytes,
             "d2h_bytes_per_step": nbytes, "ms_per_step": dt * 1e3, "steps": steps, "api": "tbsci_sigma_host"},
            hcn)


def _davidson_leg(tb, ctx, wl):
    """Davidson to |dE| < 1e-9, ||r|| < 1e-5 per root, FP64 and mixed precision."""
    import torch
    h, eri, ecore = wl.hamiltonian()
    sp = tb.Space(ctx, wl.norb, wl.nalpha, wl.nbeta, h, eri, ecore, alpha=wl.alpha_selection(),
                  beta=wl.beta_selection())
    dav = {"workload": wl.notes, "nroots": wl.nroots}
    for mode, mixed in (("f64", 0), ("mixed", 1), ("mixed_tc", 2)):
        if mixed == 2:
            # set-up, untimed: tune the tensor-core sigma type's pass for the
            # same-spin classes on one FP32 vector, as a user would once per space
            C = torch.randn((1, sp.la, sp.lb), device="cuda", dtype=torch.float32)
            S = torch.empty_like(C)
            tb.tbsci_sigma_autotune(ctx.handle, sp.ham, sp.ta, sp.tb, C, S, 1, tb.TBSCI_F32_TC_TF32)
            del C, S
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e, info = sp.davidson(wl.nroots, mixed=mixed, tol_energy=1e-9, tol_residual=1e-5)
        dt = time.perf_counter() - t0
        dav[mode] = {"seconds": dt, "iterations": info["iterations"], "nsigma": info["nsigma"],
                     "nsigma_f32": info["nsigma_f32"], "energies": [float(x) for x in e],
                     "converged": info["converged"], "seconds_sigma": info["seconds_sigma"],
                     "seconds_outside_sigma": dt - info["seconds_sigma"]}
    for mode in ("mixed", "mixed_tc"):
        dav[mode + "_minus_f64_max_abs"] = max(abs(a - b) for a, b in zip(dav[mode]["energies"],
                                                                          dav["f64"]["energies"]))
    dav["modes"] = {"f64": "FP64 sigma throughout", "mixed": "FP32 sigma, then FP64 refinement",
                    "mixed_tc": "FP32 sigma with split-TF32 tensor-core alpha-beta and same-spin products "
                                "(autotuned once, untimed), then FP64 refinement"}
    dav["target"] = "time to |dE| < 1e-9 and ||r|| < 1e-5 per root (energies within 1e-8 Eh)"
    sp.close()
    return dav


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--workload", default="sel24", choices=sorted(WORKLOADS))
    ap.add_argument("--count-alpha", type=int, default=None,
                    help="use this many selected alpha strings (a smaller case of the workload, for profiling)")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "tf32tc", "bf16tc"])
    ap.add_argument("--ref-rows", type=int, default=0, help="reference arm: oracle rows per step (0: sized)")
    ap.add_argument("--no-davidson", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the norb=16 selected-space sigma leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-stream leg of the default run")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--serving", action="store_true", help="serving stream instead of the sigma bench")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune-cache", default=None,
                    help="tune-cache file loaded into the context (with --no-autotune: pins the launch shape)")
    ap.add_argument("--precision-study", action="store_true")
    ap.add_argument("--selection-study", action="store_true",
                    help="bitstring selection loop and coefficient histograms")
    ap.add_argument("--sel-norb", type=int, default=14)
    ap.add_argument("--deltas", default="1e-2,1e-3,1e-4,1e-5")
    ap.add_argument("--modes", default="1,2,3", help="Davidson mixed modes for --precision-study")
    ap.add_argument("--max-iter", type=int, default=0)
    ap.add_argument("--basis-f32", action="store_true", help="--precision-study: FP32-stored Davidson basis")
    ap.add_argument("--max-subspace", type=int, default=0)
    ap.add_argument("--restart-keep", type=int, default=0)
    ap.add_argument("--nreq", type=int, default=512)
    ap.add_argument("--rates", default="2", help="serving: arrival rates as multiples of the FP64 service rate")
    ap.add_argument("--calibrate", type=int, default=64, help="serving: requests timed for the FP64 rate")
    ap.add_argument("--serving-mixed", type=int, default=1, help="serving: low-precision sigma mode (1, 2, 3)")
    ap.add_argument("--max-count", type=int, default=3000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)
    if args.precision_study:
        return run_precision_study(args)
    if args.selection_study:
        return run_selection_study(args)

    import torch
    import paper_2503_10335_gb300 as tb

    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    nvec = wl.nvec
    ctx = tb.Context(local, tune_cache=args.tune_cache) if args.tune_cache else tb.Context(local)
    stream = torch.cuda.current_stream()
    if dist:
        dist.barrier()
    rec, sp, C, S, sdt = _sigma_leg(tb, ctx, wl, args.dtype, nvec, args.steps, args.warmup, dev, stream,
                                    autotune=not args.no_autotune, clocks=True, count_alpha=args.count_alpha)
    ms_step = rec["ms_per_step"]
    if dist:
        dist.barrier()
        ms_step = max_over_ranks(ms_step, dist, dev)
    value = replica_throughput(ws, nvec * sp.ndet, ms_step * 1e-3) / 1e9
    del S

    e2e, hc = None, None
    if args.dtype == "f64" and args.e2e_steps > 0:
        e2e, hc = _e2e_leg(tb, ctx, sp, C, nvec, args.e2e_steps, ws)
    del C
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        if hc is None:
            hc = np.ascontiguousarray(random_vectors(nvec, sp.la, sp.lb, seed=wl.seed_vec))
        cpu = cpu_baseline(wl, nvec, C=hc.reshape(nvec, -1), count_alpha=args.count_alpha)
    del hc
    sp.close()
    torch.cuda.empty_cache()

    extra = None
    if rank == 0 and not args.no_extra and args.workload != "sel16":
        # the norb=16, 3,000 x 3,000 selected space (9.0M determinants, 3 vectors), FP64
        r16, sp16, C16, S16, _ = _sigma_leg(tb, ctx, WORKLOADS["sel16"], "f64", 3, max(5, args.steps // 2),
                                           args.warmup, dev, stream, autotune=not args.no_autotune)
        extra = {k: r16[k] for k in ("value", "ms_per_step", "roofline", "kernels", "config", "launches_per_step")}
        extra["unit"] = UNIT
        sp16.close()
        del C16, S16
        torch.cuda.empty_cache()

    dav = None
    if not args.no_davidson and rank == 0:
        dav = _davidson_leg(tb, ctx, WORKLOADS["sel16"])

    serving = None
    if not args.no_serving and rank == 0 and ws == 1:
        serving = run_serving(args, print_line=False)
        serving.pop("metric", None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": dict(rec["config"], parallelism="replicas" if ws > 1 else "single"),
            "roofline": rec["roofline"], "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": rec["gpu_launches"], "kernels": rec["kernels"],
            "clocks": rec["clocks"], "sel16_sigma": extra, "davidson": dav, "serving": serving,
            "counts": rec["counts"], "setup_seconds": rec["setup_seconds"], "autotune_ms": rec["autotune_ms"],
            "step_ms_min": rec["step_ms_min"], "step_ms_max": rec["step_ms_max"],
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
