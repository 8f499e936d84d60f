"""Benchmark: binned FFT KDE with an unconstrained bandwidth on GB300.

One step = the whole hot path on one batch: linear binning of the n samples
(kde_bin), the kernel grid and its spectrum (kde_kernel_grid, including the
host-side factorisation of H) and the FFT evaluation (kde_fft_eval).  Inputs
are resident in HBM when the timed region starts; L2 is flushed (a 256 MB
write) between timed steps.  Rank 0 prints one JSON line.  With no
--workload the line is the 1024^2 FP32 grid (n = 10^6) and carries, under
"kde3d_256_f32", the same record for the 256^3 FP32 grid (n = 10^7).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, timed on host cores
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("grid points/s and samples/s of FFT KDE at <=1e-5 rel err vs FP64; % HBM roofline")
DEFAULT_WORKLOAD = "kde2d_1024_f32"
SECOND_WORKLOAD = "kde3d_256_f32"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=None,
                    help="one workload; default: kde2d_1024_f32 with a kde3d_256_f32 record")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--learned-batch", type=int, default=256,
                    help="datasets per preparation, search and selection call (learned2d_256)")
    ap.add_argument("--e2e-graph-stages", type=int, default=2,
                    help="pipeline stages (datasets) captured per CUDA graph in the e2e stream")
    ap.add_argument("--bin-method", default="auto", choices=["auto", "direct", "tiled"])
    ap.add_argument("--counts", default="zeroed_per_step", choices=["zeroed_per_step", "kept_zero"],
                    help="zeroed_per_step: kde_bin zeroes them before binning; kept_zero: "
                         "binning adds (kde_bin_accumulate) and the evaluation clears the counts "
                         "(kde_fft_eval_consume), measured slower with L2 flushed between steps")
    ap.add_argument("--range", default="corrected", choices=["corrected", "per_axis"],
                    help="support of the kernel grid: the corrected range of Eq. 15 or the "
                         "per-axis (diagonal) range")
    ap.add_argument("--layout", default="corrected", choices=["corrected", "wand"],
                    help="kernel-grid layout: corrected (all signed lags) or Wand's (k_|l|)")
    ap.add_argument("--P-min", type=int, nargs="*", default=None,
                    help="smallest padded length per axis (the plan takes the smallest "
                         "supported size at or above it and at or above M + L)")
    ap.add_argument("--dft", default="fft", choices=["fft", "tc"],
                    help="first pass: mixed-radix FFT, or split-TF32 DFT matrix on the tensor cores")
    ap.add_argument("--slab", default="off", choices=["off", "on"],
                    help="3-D: last two axes slab by slab on thread-block clusters (one "
                         "launch each way) instead of separate row and column passes")
    ap.add_argument("--lscv", default="autocorr", choices=["autocorr", "spectrum"],
                    help="lscv2d_512_f32: pair sums from the counts' autocorrelation, or from "
                         "the count spectrum against per-candidate kernel spectra")
    ap.add_argument("--train-sets", type=int, default=100_000,
                    help="learned2d_256: training datasets labelled by the plain search")
    ap.add_argument("--eval-sets", type=int, default=10_000,
                    help="learned2d_256: held-out datasets both methods select for")
    ap.add_argument("--cpu-oracle", default=None, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# Algorithmic bytes per launch of each kernel: one read of every array a pass
# consumes and one write of every array it produces (zero padding is never
# stored).  cs = complex bytes, r = real bytes, Q = P_last/2 + 1.  Kernels
# that do the same pass under another name (the tensor-core first pass)
# carry the same figure.
# ---------------------------------------------------------------------------
def algorithmic_bytes(info, n, x_itemsize):
    d = info.d
    r = 4 if info.precision == "f32" else 8
    cs = 2 * r
    M, L, P, Q = info.M, info.L, info.P, info.Q
    cells = int(np.prod(M))
    # zeroing the counts before the atomic adds is overhead, not algorithmic
    # traffic: its time counts in the step, its bytes do not
    b = {"kde_bin_kernel": n * d * x_itemsize + 8 * cells, "kde_zero_counts_kernel": 0}
    # the tiled binning's algorithmic bytes are the same: the samples read
    # once (count kernel) and the counts written once (accumulation); its
    # second read of the samples and its records are overhead
    b.update({"kde_bin_count_kernel": n * d * x_itemsize, "kde_bin_scatter_kernel": 0,
              "kde_bin_accum_kernel": 8 * cells})
    if d == 1:
        b["kde_rows_r2c_kgen_kernel"] = Q * r
        b["kde_line1d_kernel"] = 8 * cells + Q * r + cells * r
    elif d == 2:
        w0 = 2 * L[0] + 1
        b["kde_rows_r2c_kgen_kernel"] = w0 * Q * cs
        b["kde_cols_kgen_real_kernel"] = w0 * Q * cs + P[0] * Q * r
        b["kde_rows_r2c_counts_kernel"] = 8 * cells + M[0] * Q * cs
        b["kde_cols_mid_kernel"] = 2 * M[0] * Q * cs + P[0] * Q * r
        b["kde_rows_c2r_kernel"] = M[0] * Q * cs + cells * r
    else:
        w0, w1 = 2 * L[0] + 1, 2 * L[1] + 1
        b["kde_rows_r2c_kgen_kernel"] = w0 * w1 * Q * cs
        b["kde_cols_kgen_kernel"] = w0 * w1 * Q * cs + w0 * P[1] * Q * cs
        b["kde_cols_kgen_real_kernel"] = w0 * P[1] * Q * cs + P[0] * P[1] * Q * r
        b["kde_rows_r2c_counts_kernel"] = 8 * cells + M[0] * M[1] * Q * cs
        b["kde_cols_fwd_kernel"] = M[0] * M[1] * Q * cs + M[0] * P[1] * Q * cs
        b["kde_cols_mid_kernel"] = 2 * M[0] * P[1] * Q * cs + P[0] * P[1] * Q * r
        b["kde_cols_inv_kernel"] = M[0] * P[1] * Q * cs + M[0] * M[1] * Q * cs
        b["kde_rows_c2r_kernel"] = M[0] * M[1] * Q * cs + cells * r
        # slab passes: axes 2 and 1 in one launch each way, the half spectra
        # between them kept on chip
        b["kde_fx_slab_fwd_kernel"] = 8 * cells + M[0] * P[1] * Q * cs
        b["kde_fx_slab_inv_kernel"] = M[0] * P[1] * Q * cs + cells * r
    if "kde_rows_r2c_counts_kernel" in b:
        b["kde_rows_r2c_tc_kernel"] = b["kde_rows_r2c_counts_kernel"]
    # the two-phase FFT passes do the same passes as the Stockham ones
    for k in list(b):
        if k.startswith(("kde_rows_", "kde_cols_")) and k != "kde_rows_r2c_tc_kernel":
            b[k.replace("kde_", "kde_fx_", 1)] = b[k]
    return b


def step_bytes(alg, prof, steps):
    """Algorithmic bytes of one step: every kernel that ran in the profiled
    steps, counted once per launch it made per step (a kernel that did not
    run, such as the pass the tensor-core first pass replaces, counts
    nothing)."""
    total, missing = 0.0, []
    for k, (_, launches) in prof.items():
        if k in alg:
            total += alg[k] * launches / steps
        else:
            missing.append(k)
    return total, missing


# ---------------------------------------------------------------------------
# Replicas (one process per GPU): the slowest rank times the job.
# ---------------------------------------------------------------------------
def rank_max(value, device=None):
    """Max of a per-rank scalar over all ranks of the default process group
    (the value itself when there is no group or one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, ms_step):
    """Whole-job rate: every rank's units over the slowest rank's step time."""
    return world * units_per_rank / (ms_step * 1e-3)


# FP32 ALU roofline: 152 SMs x 128 FP32 lanes x 2 flops (FMA) at the SM clock.
def fp32_peak_tflops(sm_mhz=2070.0, sms=152):
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def ac_flops(L):
    """Lag terms of the half-plane autocorrelation sum of one matrix with
    support L (rows 0..L_0, all 2 L_1 + 1 columns), 8 flops each: the
    exponent in completed squares along the row, D_1 (m + b l_0)^2 + e_0
    (5: two adds, a multiply and an FMA), exp (1), times R and accumulate
    (2)."""
    return 8.0 * (L[0] + 1) * (2 * L[1] + 1)


def fft_flops(n_lines, N):
    """The conventional 5 N log2 N flops of a complex FFT of length N."""
    return n_lines * 5.0 * N * np.log2(N)


def source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1508_02766_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, kernel):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as fh:
            t = json.load(fh)
        e = t.get(workload, {})
        if e.get("source_digest") != source_digest():
            return None
        v = e.get("kernels", {}).get(kernel)
        return None if v is None else float(v)
    except Exception:
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        busy = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": float(np.median(busy)) if busy else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(
                    (float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ---------------------------------------------------------------------------
# CPU oracle: the FP64 oracle as it stands, timed on a bounded sample of a
# workload on the host cores.  It runs in a child process (no CUDA context;
# its pool of workers is started with "spawn").  One timed sample is the
# oracle's binning of n_bin samples and Eq. 7 summed at n_nodes random
# nodes; with workers > 1 both are split into equal contiguous chunks over a
# process pool (the oracle's own functions, unchanged, on each chunk).
# ---------------------------------------------------------------------------
_CPU = {}


def _cpu_init(barrier):
    _CPU["barrier"] = barrier


def _cpu_load(path):
    """Loads one sample's arrays into this worker, then waits until every
    worker has done the same (so each worker takes exactly one of these
    tasks)."""
    z = np.load(path, allow_pickle=False)
    _CPU.update({k: z[k] for k in z.files})
    _CPU["barrier"].wait(timeout=120)
    return 1


def _cpu_bin_chunk(r):
    from oracle import kde_oracle as O
    a, b = r
    O.bin_linear(_CPU["sub"][a:b], _CPU["lo"], _CPU["hi"], tuple(int(m) for m in _CPU["M"]))
    return b - a


def _cpu_nodes_chunk(r):
    from oracle import kde_oracle as O
    a, b = r
    L = tuple(int(x) for x in _CPU["L"])
    return O.binned_direct_at(_CPU["c"], _CPU["k"], L, _CPU["nodes"][a:b])


def _chunks(n, parts):
    edges = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(edges[i]), int(edges[i + 1])) for i in range(parts) if edges[i + 1] > edges[i]]


def cpu_oracle_child(spec_json):
    """Child-process body: times the oracle on `reps` samples and prints JSON."""
    spec = json.loads(spec_json)
    from oracle import kde_oracle as O
    from paper_1508_02766_gb300 import workloads as W
    w = W.WORKLOADS[spec["workload"]]()
    n_bin, n_nodes, workers = spec["n_bin"], spec["n_nodes"], spec["workers"]
    counts, _ = O.bin_linear(w.X, w.lo, w.hi, w.M)          # set-up, not timed
    L = O.support_L(w.H, w.lo, w.hi, w.M, w.tau, spec["range"])
    k = O.kernel_weights(w.H, w.lo, w.hi, w.M, L, w.n, spec["layout"])
    c = O.counts_to_c(counts)
    pool, tmp = None, None
    if workers > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        tmp = tempfile.mktemp(prefix="kde_cpu_", suffix=".npz")
        pool = ctx.Pool(workers, initializer=_cpu_init, initargs=(ctx.Barrier(workers),))
    reps = []
    for rep in range(spec["reps"]):
        rng = np.random.default_rng(spec["seed"] + rep)
        sub = w.X[rng.choice(w.n, size=min(n_bin, w.n), replace=False)]
        nodes = np.stack([rng.integers(0, m, n_nodes) for m in w.M], axis=1)
        if workers == 1:
            t0 = time.perf_counter()
            O.bin_linear(sub, w.lo, w.hi, w.M)
            t_bin = time.perf_counter() - t0
            t0 = time.perf_counter()
            ref = O.binned_direct_at(c, k, L, nodes)
            t_nodes = time.perf_counter() - t0
        else:
            np.savez(tmp, sub=sub, lo=np.asarray(w.lo), hi=np.asarray(w.hi),
                     M=np.asarray(w.M), L=np.asarray(L), c=c, k=k, nodes=nodes)
            pool.map(_cpu_load, [tmp] * workers, chunksize=1)   # not timed
            t0 = time.perf_counter()
            pool.map(_cpu_bin_chunk, _chunks(len(sub), workers))
            t_bin = time.perf_counter() - t0
            t0 = time.perf_counter()
            ref = np.concatenate(pool.map(_cpu_nodes_chunk, _chunks(n_nodes, workers)))
            t_nodes = time.perf_counter() - t0
        reps.append({"t_bin": t_bin, "t_nodes": t_nodes})
        if rep == 0 and spec.get("nodes_file"):
            np.save(spec["nodes_file"] + ".nodes.npy", nodes)
            np.save(spec["nodes_file"] + ".ref.npy", ref)
    if pool is not None:
        pool.terminate()
        os.unlink(tmp)
    cells = float(np.prod(w.M))
    out = {"reps": reps, "cells": cells, "n": w.n, "n_bin": int(min(n_bin, w.n)),
           "n_nodes": n_nodes, "workers": workers}
    if spec.get("o1_nodes"):
        # O1 (Eq. 1, the direct sum over every sample, no binning) at a few
        # random grid points
        rng = np.random.default_rng(spec["seed"] + 99)
        j = np.stack([rng.integers(0, m, spec["o1_nodes"]) for m in w.M], axis=1)
        lo, hi, M = (np.asarray(v, dtype=np.float64) for v in (w.lo, w.hi, w.M))
        pts = lo + j * ((hi - lo) / (M - 1.0))
        t0 = time.perf_counter()
        O.direct_kde(w.X, w.H, pts, chunk=1)
        out["o1_s"] = time.perf_counter() - t0
        out["o1_nodes"] = int(spec["o1_nodes"])
    if spec.get("o3"):
        # O3 (Eq. 10-14 with a plain separable DFT, the literal corrected
        # layout) on the whole grid, once
        t0 = time.perf_counter()
        O.fft_corrected(c, k, L)
        out["o3_s"] = time.perf_counter() - t0
    print(json.dumps(out))


def run_cpu_oracle(workload, n_bin, n_nodes, seed=0, workers=1, reps=1, nodes_file="",
                   range_mode="corrected", layout="corrected", o3=False, o1_nodes=0):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    spec = json.dumps({"workload": workload, "n_bin": n_bin, "n_nodes": n_nodes, "seed": seed,
                       "workers": workers, "reps": reps, "nodes_file": nodes_file,
                       "range": range_mode, "layout": layout, "o3": o3, "o1_nodes": o1_nodes})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-oracle", spec],
                       capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_rates(r, n):
    """Rates of one timed sample: seconds per binned sample and per node,
    and the grid-point rate they give for the full workload (all n samples
    binned, Eq. 7 at every node)."""
    t_bin = float(np.mean([x["t_bin"] for x in r["reps"]]))
    t_nodes = float(np.mean([x["t_nodes"] for x in r["reps"]]))
    per_sample = t_bin / r["n_bin"]
    per_node = t_nodes / r["n_nodes"]
    t_full = per_sample * n + per_node * r["cells"]
    return {"t_sample_s": t_bin + t_nodes, "t_full_s": t_full,
            "grid_points_per_s": r["cells"] / t_full}


# bounded samples (binned samples, nodes) of the CPU baseline per workload:
# about a second of single-core oracle work each
CPU_SAMPLE = {"kde2d_1024_f32": (1_000_000, 40_000), "kde2d_128_f64": (10_000, 16_384),
              "kde3d_256_f32": (1_000_000, 4_000)}
# grid points at which O1 (the direct sum over all samples) is timed
O1_NODES = {"kde2d_1024_f32": 16, "kde2d_128_f64": 64, "kde3d_256_f32": 2}


def cpu_baseline(workload, range_mode="corrected", layout="corrected", nodes_file=""):
    """The oracle on one core and on every host core, same sample; the first
    run also writes the sampled nodes and their oracle values."""
    n_bin, n_nodes = CPU_SAMPLE[workload]
    cores = host_cores()
    one = run_cpu_oracle(workload, n_bin, n_nodes, seed=123, workers=1, nodes_file=nodes_file,
                         range_mode=range_mode, layout=layout, o3=workload == "kde2d_128_f64",
                         o1_nodes=O1_NODES.get(workload, 0))
    allc = run_cpu_oracle(workload, n_bin, n_nodes, seed=123, workers=cores,
                          range_mode=range_mode, layout=layout) if cores > 1 else one
    r1, ra = oracle_rates(one, one["n"]), oracle_rates(allc, allc["n"])
    sample = (f"oracle binning of {one['n_bin']} samples and Eq. 7 summed at {one['n_nodes']} "
              f"random nodes; value = the full workload's grid points over the time those "
              f"rates give for binning every sample and summing Eq. 7 at every node")
    out = {"value": ra["grid_points_per_s"], "unit": "grid points/s", "cores": allc["workers"],
           "kind": "oracle", "sample": sample,
           "sample_seconds": ra["t_sample_s"], "extrapolated_full_step_s": ra["t_full_s"],
           "one_core": {"value": r1["grid_points_per_s"], "cores": 1,
                        "sample_seconds": r1["t_sample_s"],
                        "extrapolated_full_step_s": r1["t_full_s"]},
           "host_cores": cores}
    if "o1_s" in one:
        out["o1_direct_kde"] = {"seconds": one["o1_s"], "cores": 1, "nodes": one["o1_nodes"],
                                "grid_points_per_s": one["o1_nodes"] / one["o1_s"],
                                "what": "O1: Eq. 1 summed over every sample (no binning) at "
                                        "random grid points"}
    if "o3_s" in one:
        out["o3_naive_dft"] = {"seconds": one["o3_s"], "cores": 1,
                               "grid_points_per_s": one["cells"] / one["o3_s"],
                               "what": "O3: the literal corrected layout (Eq. 12-14) "
                                       "convolved by a plain separable DFT (Eq. 10), whole grid"}
    return out


# ---------------------------------------------------------------------------
# Reference arm: the oracle timed per step, each step a bounded sample of the
# workload on every host core.  ms_per_step is the time the sampled work
# took; value is the workload's grid points over the full-workload time
# that the sampled rates give (reported separately).
# ---------------------------------------------------------------------------
REF_SAMPLE = {"kde2d_1024_f32": (200_000, 8_000), "kde2d_128_f64": (10_000, 4_000),
              "kde3d_256_f32": (200_000, 800)}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    workload = args.workload or DEFAULT_WORKLOAD
    n_bin, n_nodes = REF_SAMPLE[workload]
    cores = host_cores()
    r = run_cpu_oracle(workload, n_bin, n_nodes, seed=0, workers=cores,
                       reps=args.warmup + args.steps)
    timed = r["reps"][args.warmup:]
    r_t = dict(r, reps=timed)
    rates = oracle_rates(r_t, r["n"])
    ms = 1e3 * float(np.mean([x["t_bin"] + x["t_nodes"] for x in timed]))
    value = rates["grid_points_per_s"]
    sample = (f"per step: oracle binning of {r['n_bin']} samples and Eq. 7 summed at "
              f"{n_nodes} random nodes over {r['workers']} host cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "grid points/s",
            "samples_per_s": r["n"] / rates["t_full_s"], "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "extrapolated_full_step_ms": 1e3 * rates["t_full_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload},
            "step_definition": "ms_per_step is the measured time of one sampled step; value is "
                               "the full workload's grid points over extrapolated_full_step_ms",
            "cpu_baseline": {"value": value, "unit": "grid points/s", "cores": r["workers"],
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "grid points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GB300 arm.
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.cpu_oracle is not None:
        return cpu_oracle_child(args.cpu_oracle)
    if args.impl == "reference":
        return reference_arm(args)
    workload = args.workload or DEFAULT_WORKLOAD
    if workload.startswith("lscv"):
        return lscv_main(args)
    if workload.startswith("ragged"):
        return ragged_main(args)
    if workload.startswith("learned"):
        return learned_main(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1508_02766_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    line = kde_arm(args, workload, world, rank, local, dev)
    if args.workload is None:
        # the second target grid, same steps and timing rules, as its own record
        sub = kde_arm(args, SECOND_WORKLOAD, world, rank, local, dev)
        for k in ("metric", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
                  "vs_baseline", "data"):
            sub.pop(k, None)
        line[SECOND_WORKLOAD] = sub
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def kde_arm(args, workload, world, rank, local, dev):
    """One workload through bin -> kernel grid -> FFT evaluation: device-timed
    steps, per-kernel events, the end-to-end stream, the CPU baseline and the
    sampled accuracy.  Returns the JSON record."""
    import torch
    import torch.distributed as dist

    from paper_1508_02766_gb300 import kde
    from paper_1508_02766_gb300 import workloads as W

    w = W.WORKLOADS[workload]()
    stream = torch.cuda.Stream(device=dev)
    plan = kde.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau, dft=args.dft,
                    range_mode=args.range, layout=args.layout, P_min=args.P_min, slab=args.slab)
    info = plan.info
    X_host = torch.from_numpy(np.ascontiguousarray(w.X)).pin_memory()
    X = X_host.to(dev)
    # kept_zero: zeroed once here; every step then bins by adding and its
    # evaluation leaves them zeroed for the next step
    kept = args.counts == "kept_zero"
    counts = torch.zeros(w.M, dtype=torch.int64, device=dev)
    Ks = torch.empty(info.kspec_elems, dtype=plan.real_dtype(), device=dev)
    dens = torch.empty(w.M, dtype=plan.real_dtype(), device=dev)
    ws = plan.workspace(dev)
    # Binning method: direct (64-bit atomics into counts) or tiled (counting
    # sort by grid tile, shared-memory accumulation; needs a workspace).
    method = args.bin_method
    if method == "auto":
        method = "direct"   # the faster of the two on every workload measured
    bws = kde.bin_workspace(w.n, w.d, w.M, dev) if method == "tiled" else None
    dens_host = torch.empty(w.M, dtype=plan.real_dtype()).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    # One step: the kernel grid (no dependence on the samples) runs on a side
    # stream while the samples are binned; the FFT evaluation waits for both.
    side = torch.cuda.Stream(device=dev, priority=-1)
    step_dev = kde.PreparedPath(plan, X, counts, Ks, dens, ws, bin_workspace=bws, stream=stream,
                                kgen_stream=side, counts_kept_zero=kept)
    Xe = torch.empty_like(X)
    step_e2e = kde.PreparedPath(plan, Xe, counts, Ks, dens, ws, bin_workspace=bws, stream=stream,
                                kgen_stream=side, counts_kept_zero=kept)
    fork = torch.cuda.Event()
    join = torch.cuda.Event()

    def enqueue(path):
        # the kernel grid needs no samples: it runs beside the binning
        fork.record(stream)
        side.wait_event(fork)
        path.kernel_grid()
        path.bin()
        join.record(side)
        stream.wait_event(join)
        path.fft_eval()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            enqueue(step_dev)
    torch.cuda.synchronize()
    kde.plan_check(plan, stream)   # every bounded device wait completed

    # The step captured once as a CUDA graph and replayed.
    graph = None
    per_step_launches = 0
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        l0 = kde.launch_count()
        with torch.cuda.graph(graph, stream=stream):
            enqueue(step_dev)
        per_step_launches = kde.launch_count() - l0
        with torch.cuda.stream(stream):
            graph.replay()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = kde.launch_count()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            if graph is not None:
                graph.replay()
            else:
                enqueue(step_dev)
            ends[i].record(stream)
    torch.cuda.synchronize()
    launches = (kde.launch_count() - l0) if graph is None else per_step_launches * args.steps
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    kde.plan_check(plan, stream)
    per_step = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = rank_max(sum(per_step), dev)
    ms_step = ms / args.steps
    ms_median = float(np.median(per_step))
    # the same steps launched call by call, without the graph
    ms_plain = None
    if graph is not None:
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                starts[i].record(stream)
                enqueue(step_dev)
                ends[i].record(stream)
        torch.cuda.synchronize()
        ms_plain = float(np.median([s.elapsed_time(e) for s, e in zip(starts, ends)]))
    cells = int(np.prod(w.M))
    value = job_throughput(world, cells, ms_step)
    samples_s = job_throughput(world, w.n, ms_step)

    # Per-kernel durations: the same steps launched one by one on one stream
    # (no overlap, so each event pair measures its kernel alone) with the
    # library's event pairs around every kernel (graph replays carry none).
    step_serial = kde.PreparedPath(plan, X, counts, Ks, dens, ws, bin_workspace=bws, stream=stream,
                                   counts_kept_zero=kept)
    kde.profile_enable(True)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            step_serial()
    torch.cuda.synchronize()
    prof = kde.profile_read()
    kde.profile_enable(False)

    # End to end through the public API with host buffers, as a stream of
    # datasets.  One pipeline stage uploads the next step's samples from
    # pinned memory (upload stream), runs this step's three calls (compute
    # stream; kernel grid beside the binning) and reads the previous step's
    # density back to pinned memory (read-back stream); two sample and two
    # density buffers alternate between stages.  G stages are captured per
    # CUDA graph (one graph per starting buffer parity) and replayed back to
    # back: every step still makes one upload, one evaluation and one
    # read-back, and the graph launches are G times fewer (measured at
    # 1024²: 56.6 µs per step with one stage per graph, 51.0 with two, no
    # better with four or eight).
    e2e_steps = max(3, min(args.steps, 50))
    up_s = torch.cuda.Stream(device=dev)
    down_s = torch.cuda.Stream(device=dev)
    Xb = [Xe, torch.empty_like(X)]
    Db = [dens, torch.empty_like(dens)]
    Hb = [dens_host, torch.empty(w.M, dtype=plan.real_dtype()).pin_memory()]
    paths = [step_e2e, kde.PreparedPath(plan, Xb[1], counts, Ks, Db[1], ws, bin_workspace=bws,
                                        stream=stream, kgen_stream=side, counts_kept_zero=kept)]
    ev_fork, ev_up, ev_down = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()

    def stage(b):
        ev_fork.record(stream)
        up_s.wait_event(ev_fork)
        down_s.wait_event(ev_fork)
        with torch.cuda.stream(up_s):
            Xb[1 - b].copy_(X_host, non_blocking=True)        # next step's samples
        with torch.cuda.stream(down_s):
            Hb[1 - b].copy_(Db[1 - b], non_blocking=True)     # previous step's density
        ev_up.record(up_s)
        ev_down.record(down_s)
        enqueue(paths[b])                                      # this step
        stream.wait_event(ev_up)
        stream.wait_event(ev_down)

    with torch.cuda.stream(stream):
        Xb[0].copy_(X_host, non_blocking=True)
        for i in range(4):
            stage(i % 2)
    torch.cuda.synchronize()
    # G stages per graph (parities alternating inside it); one graph per
    # starting parity, so that consecutive replays keep alternating
    G = max(1, args.e2e_graph_stages) if graph is not None else 1
    e2e_steps = -(-e2e_steps // G) * G
    stage_graphs = []
    if graph is not None:
        for b in range(2):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for j in range(G):
                    stage((b + j) % 2)
            stage_graphs.append(g)
        torch.cuda.synchronize()

    def e2e_step(i):
        # step i of the stream; a graph covers steps i .. i + G - 1
        if stage_graphs:
            if i % G == 0:
                stage_graphs[i % 2].replay()
        else:
            stage(i % 2)

    e_s = torch.cuda.Event(enable_timing=True)
    e_e = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        Xb[0].copy_(X_host, non_blocking=True)
        for i in range(2):
            e2e_step(i)
        e_s.record(stream)
        for i in range(e2e_steps):
            e2e_step(i)
        e_e.record(stream)
    torch.cuda.synchronize()
    e2e_ms = rank_max(e_s.elapsed_time(e_e) / e2e_steps, dev)

    # End to end without copies: the binning kernel reads the samples in
    # place from the pinned host buffer and the output-row pass writes the
    # density in place into pinned host memory (page-locked host memory is
    # device-accessible under unified addressing; on a Grace-Blackwell node
    # those loads and stores cross the NVLink-C2C link).  The same three
    # C-ABI calls, captured once and replayed per step; nothing is cached
    # between steps (the counts and spectra are rewritten each step).
    dens_zc = torch.empty(w.M, dtype=plan.real_dtype()).pin_memory()
    path_zc = kde.PreparedPath(plan, X_host, counts, Ks, dens_zc, ws, bin_workspace=bws,
                               stream=stream, kgen_stream=side, counts_kept_zero=kept)
    with torch.cuda.stream(stream):
        for _ in range(2):
            enqueue(path_zc)
    torch.cuda.synchronize()
    zc_graph = None
    if graph is not None:
        zc_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(zc_graph, stream=stream):
            enqueue(path_zc)
        torch.cuda.synchronize()
    z_s = torch.cuda.Event(enable_timing=True)
    z_e = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        z_s.record(stream)
        for i in range(e2e_steps):
            if zc_graph is not None:
                zc_graph.replay()
            else:
                enqueue(path_zc)
        z_e.record(stream)
    torch.cuda.synchronize()
    zc_ms = rank_max(z_s.elapsed_time(z_e) / e2e_steps, dev)
    zc_err = float((dens_zc.to(dev) - dens).abs().max().item()) if rank == 0 else 0.0

    # Roofline of the dominant kernel, and of the whole step.
    alg = algorithmic_bytes(info, w.n, w.X.dtype.itemsize)
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                   "share": v[0] / max(1e-12, sum(x[0] for x in prof.values())),
                   "algorithmic_bytes_per_launch": alg.get(k)}
               for k, v in prof.items()}
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    peak, peak_kind = peaks()
    ach = alg.get(dom, 0) / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": f"{peak_kind} (hbm_gbs, copy bandwidth)",
                "traffic": measured_traffic(workload, dom),
                "algorithmic_bytes": alg.get(dom, 0)}
    sbytes, missing = step_bytes(alg, prof, args.steps)
    path_roof = {"algorithmic_bytes_per_step": sbytes,
                 "achieved_GBps": sbytes / (ms_step * 1e-3) / 1e9,
                 "frac": sbytes / (ms_step * 1e-3) / 1e9 / peak,
                 "what": "every kernel that ran in one step (per-kernel event pass), each "
                         "counted once per launch, over the device-timed step"}
    if missing:
        path_roof["kernels_without_byte_model"] = missing

    line = {"metric": METRIC, "value": value, "unit": "grid points/s", "samples_per_s": samples_s,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "ms_per_step_median": ms_median, "ms_per_step_without_graph_median": ms_plain,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if info.precision == "f32" else "f64", "data": "synthetic",
            "config": {"workload": workload, "d": w.d, "n": w.n, "grid": list(w.M),
                       "L": list(info.L), "P": list(info.P), "precision": info.precision,
                       "l2": "flushed between timed steps (256 MB write)",
                       "launch": "CUDA graph replay per step" if graph is not None else "stream launches",
                       "streams": "kernel grid on a side stream, concurrent with binning",
                       "binning": method, "range": args.range, "layout": args.layout,
                       "counts": ("kept at zero between steps: binning adds into them "
                                  "(kde_bin_accumulate) and the evaluation's second pass clears "
                                  "them once its first pass has read them (kde_fft_eval_consume); "
                                  "zeroed once before the first step") if kept else
                                 "zeroed by kde_bin before every binning",
                       "first_pass": "split-TF32 DFT matrix on the tensor cores" if args.dft == "tc"
                       else "FFT",
                       **({"slab_passes": "last two axes per slab on 8-block clusters"}
                          if info.slab_passes else {}),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "path_roofline": path_roof, "kernels": kernels,
            "kernel_timing": "CUDA events around each kernel, over the same K steps launched "
                             "one by one on one stream right after the timed region",
            "gpu_launches": launches,
            "e2e": {"value": job_throughput(world, cells, e2e_ms), "unit": "grid points/s",
                    "overlap": "step i+1's upload and step i-1's read-back run beside step i's "
                               "kernels (two sample and two density buffers, two copy streams, "
                               f"{G} stage(s) captured per CUDA graph, one graph per starting "
                               "buffer parity, replayed back to back)",
                    "graph_stages": G,
                    "l2": "not flushed between the steps of the stream: every array a step "
                          "reads is written within that step (its samples by its own upload; "
                          "counts, kernel spectrum and spectra by its kernels); only the plan's "
                          "twiddle tables persist",
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": int(X.numel() * X.element_size()),
                    "d2h_bytes_per_step": int(dens.numel() * dens.element_size()),
                    "in_place_host_buffers": {
                        "value": job_throughput(world, cells, zc_ms), "unit": "grid points/s",
                        "ms_per_step": zc_ms,
                        "how": "the same calls on pinned host buffers: binning reads the samples "
                               "and the output rows write the density in place over the host link",
                        "h2d_bytes_per_step": int(X.numel() * X.element_size()),
                        "d2h_bytes_per_step": int(dens.numel() * dens.element_size()),
                        "max_abs_diff_vs_device_buffers": zc_err}},
            "clocks": clocks}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tmp = tempfile.mktemp(prefix="kde_nodes_")
        line["cpu_baseline"] = cpu_baseline(workload, range_mode=args.range, layout=args.layout,
                                            nodes_file=tmp)
        nodes = np.load(tmp + ".nodes.npy")
        ref = np.load(tmp + ".ref.npy")
        for suf in (".nodes.npy", ".ref.npy"):
            os.unlink(tmp + suf)
        with torch.cuda.stream(stream):
            enqueue(step_dev)
        torch.cuda.synchronize()
        got = dens.cpu().numpy()[tuple(nodes.T)]
        line["accuracy"] = {"max_rel_err_vs_oracle_sampled": float(
            np.max(np.abs(got - ref)) / np.max(np.abs(ref))), "nodes": int(len(ref)),
            "oracle": "Eq. 7 (binned direct sum, FP64) at random nodes"}
    if rank == 0 and (args.range != "corrected" or args.layout != "corrected"):
        # what the per-axis range or Wand's layout changes: this estimate
        # against the corrected one from the same counts (Sec. 4.2, Fig. 1)
        pc = kde.Plan(w.M, w.lo, w.hi, w.H, precision=w.precision, tau=w.tau)
        wsc = pc.workspace(dev)
        with torch.cuda.stream(stream):
            enqueue(step_dev)
            # the same samples' counts (the step's own are cleared by its evaluation)
            cc = kde.kde_bin(X, w.lo, w.hi, w.M, stream=stream)
            Kc = kde.kde_kernel_grid(pc, w.n, workspace=wsc)
            dc = kde.kde_fft_eval(pc, cc, Kc, workspace=wsc)
        torch.cuda.synchronize()
        line["vs_corrected"] = {
            "max_rel_diff": float((dens - dc).abs().max() / dc.abs().max()),
            "L": list(info.L), "L_corrected": list(pc.info.L)}
    return line


# ---------------------------------------------------------------------------
# Ragged batch: 64 independent datasets of different sizes, one graph replay.
# ---------------------------------------------------------------------------
RAGGED_METRIC = "datasets/s and grid points/s of a ragged batch of 2-D FFT KDEs"


def ragged_main(args):
    import torch
    from paper_1508_02766_gb300 import build as B
    from paper_1508_02766_gb300 import kde
    from paper_1508_02766_gb300 import workloads as W
    if not os.path.exists(B.LIB):
        B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    problems = W.ragged64_f32()
    bp = kde.BatchPlan([(w.M, w.lo, w.hi, w.H, w.n) for w in problems], precision="f32")
    stream = torch.cuda.Stream(device=dev)
    X = torch.from_numpy(np.ascontiguousarray(np.concatenate([w.X for w in problems]))).to(dev)
    dens = torch.empty(bp.density_elems, dtype=torch.float32, device=dev)
    # room for the longer paddings the tuner may choose, and at least 256 MB
    # so that the tuner can start each timed run with the caches cold
    ws = torch.empty(max(2 * bp.workspace_bytes, 256 << 20), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tuned_ms = bp.tune(X, dens, ws, reps=3, stream=stream)
    tuned_mode, tuned_shape = bp.mode(), bp.shape()
    pad, order, Ps, queue = bp.config(len(problems))

    def timed(mode, shape):
        """K graph replays of one evaluation in the given mode (L2 flushed)."""
        bp.set_mode(mode)
        bp.set_shape(*shape)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                bp.eval(X, dens, ws, stream=stream)
        torch.cuda.synchronize()
        bp.check(stream)
        graph = torch.cuda.CUDAGraph()
        l0 = kde.launch_count()
        with torch.cuda.graph(graph, stream=stream):
            bp.eval(X, dens, ws, stream=stream)
        per_step = kde.launch_count() - l0
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                starts[i].record(stream)
                graph.replay()
                ends[i].record(stream)
        torch.cuda.synchronize()
        bp.check(stream)
        return float(sum(a.elapsed_time(b) for a, b in zip(starts, ends))) / args.steps, per_step

    other = "staged" if tuned_mode == "persistent" else "persistent"
    other_shape = (tuned_shape[0], tuned_shape[0]) if other == "persistent" else tuned_shape
    ms_other, launches_other = timed(other, other_shape)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ms_step, per_step = timed(tuned_mode, tuned_shape)
    clocks = sampler.stop()
    kde.profile_enable(True)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            bp.eval(X, dens, ws, stream=stream)
    torch.cuda.synchronize()
    prof = kde.profile_read()
    kde.profile_enable(False)
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                   "share": v[0] / max(1e-12, sum(x[0] for x in prof.values()))}
               for k, v in prof.items()}
    cells = sum(int(np.prod(w.M)) for w in problems)
    # algorithmic bytes of each pass summed over the problems (the same
    # per-problem formulas as the single-problem path)
    alg = {}
    for w in problems:
        pi = kde.kde_plan_info_compute(w.M, w.lo, w.hi, w.H, precision="f32", tau=w.tau)
        b = algorithmic_bytes(pi, w.n, 4)
        for src, dst in (("kde_bin_kernel", "kde_batch_bin_kernel"),
                         ("kde_rows_r2c_kgen_kernel", "kde_batch_krows_kernel"),
                         ("kde_cols_kgen_real_kernel", "kde_batch_kcols_kernel"),
                         ("kde_rows_r2c_counts_kernel", "kde_batch_rows_kernel"),
                         ("kde_cols_mid_kernel", "kde_batch_mid_kernel"),
                         ("kde_rows_c2r_kernel", "kde_batch_c2r_kernel")):
            alg[dst] = alg.get(dst, 0) + b[src]
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    peak, peak_kind = peaks()
    ach = alg.get(dom, 0) / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": peak_kind, "traffic": None,
                "algorithmic_bytes": alg.get(dom, 0)}
    line = {"metric": RAGGED_METRIC, "value": len(problems) / (ms_step * 1e-3), "unit": "datasets/s",
            "grid_points_per_s": cells / (ms_step * 1e-3),
            "samples_per_s": sum(w.n for w in problems) / (ms_step * 1e-3), "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "ragged64_f32", "datasets": len(problems),
                       "grids": sorted({w.M[0] for w in problems}), "total_samples": int(X.shape[0]),
                       "launch": "one CUDA graph replay per step",
                       "tuner": {"mode": tuned_mode, "queue_order": queue,
                                 "threads_per_line": list(tuned_shape),
                                 "padding": pad, "radix_order": order,
                                 "padded_lengths": [list(p) for p in Ps], "tuned_ms": tuned_ms},
                       "l2": "flushed between timed steps (256 MB write)"},
            "other_mode": {"mode": other, "threads_per_line": list(other_shape),
                           "ms_per_step": ms_other, "value": len(problems) / (ms_other * 1e-3),
                           "launches_per_step": launches_other},
            "roofline": roofline, "kernels": kernels, "gpu_launches": per_step * args.steps,
            "clocks": clocks}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# Bandwidth selection: bin once, count spectrum once, LSCV for every candidate.
# ---------------------------------------------------------------------------
LSCV_METRIC = "LSCV candidates/s (binned FFT KDE, batched kernel spectra)"


def lscv_main(args):
    import torch
    from paper_1508_02766_gb300 import build as B
    from paper_1508_02766_gb300 import kde
    from paper_1508_02766_gb300 import workloads as W
    if not os.path.exists(B.LIB):
        B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = W.lscv2d_512_f32()
    lam = [np.linalg.eigvalsh(h).max() for h in w.H]
    big = 2.0 * w.H[int(np.argmax(lam))]
    pinfo = kde.kde_plan_info_compute(w.M, w.lo, w.hi, big, precision=w.precision, tau=w.tau)
    plan = kde.Plan(w.M, w.lo, w.hi, big, precision=w.precision, tau=w.tau, P_min=pinfo.P)
    info = plan.info
    stream = torch.cuda.Stream(device=dev)
    X = torch.from_numpy(np.ascontiguousarray(w.X)).to(dev)
    counts = torch.empty(w.M, dtype=torch.int64, device=dev)
    Wsp = torch.empty(info.kspec_elems, dtype=plan.real_dtype(), device=dev)
    ws = plan.workspace(dev)
    lws = torch.empty(max(256, kde.kde_lscv_workspace_bytes(plan)), dtype=torch.uint8, device=dev)
    scores = torch.empty(len(w.H), dtype=torch.float64, device=dev)
    pair = torch.empty(2 * len(w.H), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    R = torch.empty(info.P[0], info.P[1], dtype=plan.real_dtype(), device=dev)
    acws = torch.empty(kde.kde_lscv_autocorr_workspace_bytes(plan), dtype=torch.uint8, device=dev)
    # the candidates' FP64 factorisations, once (set-up, like the plan)
    cand_set = kde.LscvCands(plan, w.H)

    def step():
        kde.kde_bin(X, w.lo, w.hi, w.M, counts=counts, method="direct", stream=stream)
        if args.lscv == "spectrum":
            kde.kde_power_spectrum(plan, counts, W=Wsp, workspace=ws, stream=stream)
            kde.kde_lscv(plan, w.n, w.H, Wsp, lscv=scores, pair_sums=pair, workspace=lws,
                         stream=stream)
        else:
            kde.kde_autocorrelation(plan, counts, R=R, workspace=acws, stream=stream)
            cand_set.score(w.n, R, lscv=scores, pair_sums=pair, workspace=acws, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    torch.cuda.synchronize()
    # the autocorrelation step is launches only: captured once as a CUDA
    # graph and replayed (the spectrum path copies host parameters per call)
    graph, per_step_launches = None, 0
    if not args.no_graph and args.lscv == "autocorr":
        graph = torch.cuda.CUDAGraph()
        l0 = kde.launch_count()
        with torch.cuda.graph(graph, stream=stream):
            step()
        per_step_launches = kde.launch_count() - l0
        with torch.cuda.stream(stream):
            graph.replay()
        torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    l0 = kde.launch_count()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            if graph is not None:
                graph.replay()
            else:
                step()
            ends[i].record(stream)
    torch.cuda.synchronize()
    launches = per_step_launches * args.steps if graph is not None else kde.launch_count() - l0
    clocks = sampler.stop()
    ms_step = float(sum(a.elapsed_time(b) for a, b in zip(starts, ends))) / args.steps
    # per-kernel durations: the same steps launched one by one right after
    kde.profile_enable(True)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            step()
    torch.cuda.synchronize()
    prof = kde.profile_read()
    kde.profile_enable(False)
    value = len(w.H) / (ms_step * 1e-3)
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                   "share": v[0] / max(1e-12, sum(x[0] for x in prof.values()))}
               for k, v in prof.items()}
    # FFT flops (5 N log2 N per complex line) of the batched kernel-spectrum
    # passes, per launch: every chunk holds 64 matrices (H_i and 2 H_i).
    P0, P1, Q = info.P[0], info.P[1], info.Q
    Ls = [kde.kde_plan_info_compute(w.M, w.lo, w.hi, A, precision=w.precision, tau=w.tau).L
          for h in w.H for A in (h, 2 * h)]
    nlaunch = max(1, max(prof.get("kde_cols_kgen_dot_kernel", (0, 1))[1],
                         prof.get("kde_lscv_ac_kernel", (0, 1))[1]) // args.steps)
    flops = {"kde_rows_kgen_batch_kernel": sum(fft_flops(L[0] + 1, P1) for L in Ls) / nlaunch,
             "kde_cols_kgen_dot_kernel": len(Ls) * (fft_flops((Q + 1) // 2, P0) + 2.0 * P0 * Q) / nlaunch,
             "kde_lscv_ac_kernel": sum(ac_flops(L) for L in Ls) / nlaunch}
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / prof[dom][1]
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    if dom == "kde_bin_kernel":
        # binning: HBM-bound model, X read once and the counts written once
        hbm, src = peaks()
        nbytes = w.n * w.d * w.X.dtype.itemsize + 8 * int(np.prod(w.M))
        ach = nbytes / (dom_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"
                    if src == "measured" else "fallback 6.8 TB/s",
                    "traffic": None, "bytes_per_launch": nbytes}
    else:
        peak = fp32_peak_tflops(sm_max)
        ach = flops.get(dom, 0.0) / (dom_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x SM max clock",
                    "traffic": None, "flops_per_launch": flops.get(dom, 0.0),
                    "flop_model": "5 N log2 N per complex FFT line + 2 per dot-product term; "
                                  "8 per lag term of the autocorrelation sum (exp counted as 1)"}
    line = {"metric": LSCV_METRIC, "value": value, "unit": "candidates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": info.precision, "data": "synthetic",
            "config": {"workload": w.name, "d": w.d, "n": w.n, "grid": list(w.M),
                       "candidates": len(w.H), "P": list(info.P),
                       "pair_sums": "counts' autocorrelation, candidates prepared once "
                                    "(kde_lscv_cands: host FP64 factorisations outside the loop)"
                       if args.lscv == "autocorr"
                       else "count spectrum x per-candidate kernel spectra",
                       "launch": "CUDA graph replay per step" if graph is not None
                       else "stream launches",
                       "l2": "flushed between timed steps (256 MB write)"},
            "roofline": roofline, "kernels": kernels, "gpu_launches": launches, "clocks": clocks}
    line["densities"] = multi_density_record(args, w, counts, stream, flush)
    if not args.no_cpu_baseline:
        # the oracle's spectral pair sums for a few candidates, timed, and the
        # GPU's values for the same candidates compared with them
        code = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import kde_oracle as O
from paper_1508_02766_gb300 import workloads as W
w = W.lscv2d_512_f32()
counts = np.load(sys.argv[2])
P = tuple(int(x) for x in sys.argv[3].split(","))
idx = [int(x) for x in sys.argv[4].split(",")]
c = O.counts_to_c(counts)
t0 = time.perf_counter()
out = []
for i in idx:
    for A in (w.H[i], 2 * w.H[i]):
        L = O.support_L(A, w.lo, w.hi, w.M, w.tau)
        out.append(O.binned_pair_sum_dft(c, A, w.lo, w.hi, w.M, L, P))
print(json.dumps({"t": time.perf_counter() - t0, "S": out}))
"""
        tmp = tempfile.mktemp(prefix="kde_counts_") + ".npy"
        np.save(tmp, counts.cpu().numpy())
        idx = [0, 100, 500]
        env = dict(os.environ)
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = "1"
        r = subprocess.run([sys.executable, "-c", code, ROOT, tmp,
                            ",".join(str(p) for p in info.P), ",".join(str(i) for i in idx)],
                           capture_output=True, text=True, env=env)
        os.unlink(tmp)
        res = json.loads(r.stdout.strip().splitlines()[-1])
        got = pair.cpu().numpy()
        want = np.array(res["S"])
        have = np.array([got[2 * i + h] for i in idx for h in (0, 1)])
        line["cpu_baseline"] = {"value": len(idx) / res["t"], "unit": "candidates/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"oracle spectral pair sums (plain DFT) for {len(idx)} "
                                          f"candidates ({res['t']:.1f} s)"}
        line["accuracy"] = {"max_rel_err_pair_sums_vs_oracle": float(np.max(np.abs(have - want) / np.abs(want)))}
    print(json.dumps(line))


def multi_density_record(args, w, counts, stream, flush):
    """Density grids for every candidate bandwidth from one count spectrum
    (kde_fft_eval_multi) against the per-bandwidth path (kde_kernel_grid +
    kde_fft_eval per H, plans made beforehand) on the same GPU, same counts,
    same padding; L2 flushed before each timed step."""
    import torch
    from paper_1508_02766_gb300 import kde
    dev = counts.device
    big = max(w.H, key=lambda h: np.linalg.eigvalsh(h).max())
    pinfo = kde.kde_plan_info_compute(w.M, w.lo, w.hi, big, precision="f32", tau=w.tau)
    plan = kde.Plan(w.M, w.lo, w.hi, big, precision="f32", tau=w.tau, P_min=pinfo.P)
    info = plan.info
    nH = len(w.H)
    dens = torch.empty((nH,) + tuple(w.M), dtype=torch.float32, device=dev)
    mws = torch.empty(kde.kde_fft_eval_multi_workspace_bytes(plan), dtype=torch.uint8, device=dev)
    steps = max(3, min(args.steps, 10))
    with torch.cuda.stream(stream):
        for _ in range(2):
            kde.kde_fft_eval_multi(plan, w.n, w.H, counts, dens, mws, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            kde.kde_fft_eval_multi(plan, w.n, w.H, counts, dens, mws, stream=stream)
            b.record(stream)
    torch.cuda.synchronize()
    ms_multi = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    kde.profile_enable(True)
    with torch.cuda.stream(stream):
        kde.kde_fft_eval_multi(plan, w.n, w.H, counts, dens, mws, stream=stream)
    torch.cuda.synchronize()
    prof = kde.profile_read()
    kde.profile_enable(False)
    # the per-bandwidth path
    plans = [kde.Plan(w.M, w.lo, w.hi, h, precision="f32", tau=w.tau, P_min=info.P) for h in w.H]
    ws = plan.workspace(dev)
    Ks = torch.empty(info.kspec_elems, dtype=torch.float32, device=dev)
    ref = torch.empty_like(dens)

    def per_h():
        for i, ph in enumerate(plans):
            kde.kde_kernel_grid(ph, w.n, Kspec=Ks, workspace=ws, stream=stream)
            kde.kde_fft_eval(ph, counts, Ks, density=ref[i], workspace=ws, stream=stream)

    with torch.cuda.stream(stream):
        per_h()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        flush.zero_()
        a.record(stream)
        per_h()
        b.record(stream)
    torch.cuda.synchronize()
    ms_per_h = a.elapsed_time(b)
    diff = float(((dens - ref).abs().amax(dim=(1, 2)) / ref.abs().amax(dim=(1, 2))).max())
    # algorithmic bytes: the count spectra once, then per bandwidth its kernel
    # rows and spectrum, middle axis and output rows (same model as the
    # single-problem path)
    total = 0.0
    for i, h in enumerate(w.H):
        hi = kde.kde_plan_info_compute(w.M, w.lo, w.hi, h, precision="f32", tau=w.tau,
                                       P_min=info.P)
        bb = algorithmic_bytes(hi, w.n, 4)
        total += sum(bb[k] for k in ("kde_rows_r2c_kgen_kernel", "kde_cols_kgen_real_kernel",
                                     "kde_cols_mid_kernel", "kde_rows_c2r_kernel"))
    total += algorithmic_bytes(info, w.n, 4)["kde_rows_r2c_counts_kernel"]
    peak, kind = peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    return {"value": nH / (ms_multi * 1e-3), "unit": "densities/s", "ms_per_step": ms_multi,
            "candidates": nH, "grid": list(w.M), "P": list(info.P),
            "per_bandwidth_path": {"value": nH / (ms_per_h * 1e-3), "unit": "densities/s",
                                   "ms": ms_per_h},
            "speedup": ms_per_h / ms_multi,
            "max_rel_diff_vs_per_bandwidth": diff,
            "path_roofline": {"algorithmic_bytes_per_step": total,
                              "achieved_GBps": total / (ms_multi * 1e-3) / 1e9,
                              "frac": total / (ms_multi * 1e-3) / 1e9 / peak,
                              "peak_source": kind},
            "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items()},
            "dominant_kernel": dom,
            "what": "one count spectrum, then 64 bandwidths per launch: kernel-grid rows, kernel "
                    "spectrum, middle axis and output rows (kde_fft_eval_multi); bandwidth "
                    "factorisations on the host inside the timed call"}


# ---------------------------------------------------------------------------
# Learned bandwidth proposal vs the plain batched LSCV search.
# ---------------------------------------------------------------------------
LEARN_METRIC = ("bandwidth selections/s of the learned proposal (scored and refined by FFT LSCV) "
                "vs the plain batched LSCV search, same grid and accuracy")


def _learn_chunk(job):
    """Worker of the dataset pool: one chunk of the learned workload's
    datasets (no CUDA in the workers)."""
    from paper_1508_02766_gb300 import workloads as W
    seed, chunk, count, n = job
    return W.mixture_dataset_chunk(seed, chunk, count, n)


def _learn_stream(pool, seed, total, chunk, n):
    """The datasets of one seed in chunks (count x n x 2), drawn by the pool
    in order."""
    jobs = [(seed, c, min(chunk, total - c * chunk), n) for c in range((total + chunk - 1) // chunk)]
    return pool.imap(_learn_chunk, jobs)


def learned_main(args):
    import multiprocessing as mp
    # the dataset pool starts before any CUDA call (spawned workers)
    workers = max(1, min(16, (os.cpu_count() or 1) - 1))
    pool = mp.get_context("spawn").Pool(workers)
    import torch
    from paper_1508_02766_gb300 import build as B
    from paper_1508_02766_gb300 import kde
    from paper_1508_02766_gb300 import learned as Lm
    if not os.path.exists(B.LIB):
        B.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n, chunk, Bsel = 10_000, 1024, args.learned_batch
    n_train, n_eval = args.train_sets, args.eval_sets
    sc = Lm.LscvScorer(n)
    # labels: the plain search (every candidate) on every training dataset,
    # in batches of Bsel datasets per preparation and search call
    feats = np.empty((n_train, kde.FEAT_DIM), dtype=np.float32)
    theta = np.empty((n_train, 3))
    t_label, t_gen, i0 = 0.0, 0.0, 0
    tg = time.perf_counter()
    for Xc in _learn_stream(pool, 31, n_train, chunk, n):
        t_gen += time.perf_counter() - tg
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for b0 in range(0, Xc.shape[0], Bsel):
            part = Xc[b0:b0 + Bsel]
            off = np.arange(part.shape[0] + 1, dtype=np.int64) * n
            Xd = torch.from_numpy(part.reshape(-1, 2)).to(dev)
            F, Rs, ns = sc.prepare_batch(Xd, off)
            th, _ = sc.search_batch(Rs, ns)
            k = part.shape[0]
            theta[i0:i0 + k] = th
            feats[i0:i0 + k] = F.cpu().numpy()
            i0 += k
        torch.cuda.synchronize()
        t_label += time.perf_counter() - t0
        tg = time.perf_counter()
    # training, with the library's per-kernel events
    mlp = kde.MLP(in_dim=kde.FEAT_DIM, hidden=256, out_dim=3, max_batch=256, seed=0)
    epochs, batch = 40, 256
    kde.profile_enable(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = Lm.train(mlp, feats, theta, epochs=epochs, batch=batch, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    prof_train = kde.profile_read()
    kde.profile_enable(False)
    steps_train = epochs * (n_train // batch)
    Bp, hid, din = 256, 256, kde.FEAT_DIM
    gemm_flops_step = 2.0 * Bp * (din * hid + hid * hid + hid * 16) + 2.0 * (
        hid * 16 * Bp + Bp * hid * 64 + hid * hid * Bp + Bp * hid * hid + hid * din * Bp)
    g_ms, g_n = prof_train.get("kde_gemm_tc_kernel", (0.0, 1))
    peak_bf16 = 1897.8
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as fh:
            peak_bf16 = float(json.load(fh).get("bf16_tflops", peak_bf16))
    gemm_tf = gemm_flops_step * steps_train / (g_ms * 1e-3) / 1e12 if g_ms > 0 else 0.0
    # held-out datasets (resident on the host, pinned: each batch is one copy)
    evals = np.concatenate(list(_learn_stream(pool, 32, n_eval + Bsel, chunk, n)))
    pool.close()
    pool.join()
    pinned = torch.from_numpy(evals.reshape(-1, 2)).pin_memory()
    warm, evals_t = pinned[:Bsel * n], pinned[Bsel * n:]
    K = n_eval

    todo = [(b0, min(Bsel, K - b0)) for b0 in range(0, K, Bsel)]
    bufs = [torch.empty(Bsel * n, 2, dtype=torch.float32, device=dev) for _ in range(2)]
    copy_stream = torch.cuda.Stream()

    def batches():
        """Each batch's samples as a device tensor: batch i + 1 is copied on a
        copy stream while batch i is processed (two buffers; a buffer is
        refilled only after the work that read it)."""
        ready = [torch.cuda.Event() for _ in range(2)]
        freed = [torch.cuda.Event() for _ in range(2)]

        def upload(i):
            b0, k = todo[i]
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(freed[i % 2])
                bufs[i % 2][:k * n].copy_(evals_t[b0 * n:(b0 + k) * n], non_blocking=True)
                ready[i % 2].record(copy_stream)

        upload(0)
        for i, (b0, k) in enumerate(todo):
            if i + 1 < len(todo):
                upload(i + 1)
            torch.cuda.current_stream().wait_event(ready[i % 2])
            yield b0, k, bufs[i % 2][:k * n]
            freed[i % 2].record()

    off_full = np.arange(Bsel + 1, dtype=np.int64) * n
    # warm-up of both methods
    Xd = warm.to(dev, non_blocking=True)
    F, Rs, ns = sc.prepare_batch(Xd, off_full)
    sc.search_batch(Rs, ns)
    Lm.select_batch(sc, mlp, Xd, offsets=off_full)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    # plain method: batched preparation, every candidate scored, argmin per dataset
    l0 = kde.launch_count()
    t0 = time.perf_counter()
    best = np.empty(K)
    for b0, k, Xd in batches():
        F, Rs, ns = sc.prepare_batch(Xd, off_full[:k + 1])
        best[b0:b0 + k] = sc.search_batch(Rs, ns)[1]
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    launches_plain = kde.launch_count() - l0
    # learned method, batches of Bsel datasets: batched preparation, one
    # network pass per batch, 28 scored candidates each, fallback rule
    scored = []
    torch.cuda.synchronize()
    l0 = kde.launch_count()
    t0 = time.perf_counter()
    got, fell, ncand = np.empty(K), 0, 0
    # batch i + 1 is enqueued before batch i's results are read back, so the
    # host's work on one batch overlaps the GPU's on the next
    def collect(b0, k, job):
        nonlocal fell, ncand
        th, v, c, fb = Lm.select_collect(sc, job, as_arrays=True)
        got[b0:b0 + k] = v
        fell += int(fb.sum())
        ncand += int(c.sum())

    prev = None
    for b0, k, Xd in batches():
        job = Lm.select_submit(sc, mlp, Xd, off_full[:k + 1])
        if prev is not None:
            collect(*prev)
        prev = (b0, k, job)
    collect(*prev)
    torch.cuda.synchronize()
    t_learn = time.perf_counter() - t0
    launches_learn = kde.launch_count() - l0
    clocks = sampler.stop()
    # per-kernel times from a separate pass over the first batches with the
    # library's event pairs on (they cost host time, so not in the loops above)
    nprof = min(K, 8 * Bsel)
    kde.profile_enable(True)
    for b0 in range(0, nprof, Bsel):
        k = min(Bsel, nprof - b0)
        Xd = evals_t[b0 * n:(b0 + k) * n].to(dev)
        F, Rs, ns = sc.prepare_batch(Xd, off_full[:k + 1])
        sc.search_batch(Rs, ns)
    torch.cuda.synchronize()
    prof_plain = kde.profile_read()
    kde.profile_enable(False)
    kde.profile_enable(True)
    for b0 in range(0, nprof, Bsel):
        k = min(Bsel, nprof - b0)
        Xd = evals_t[b0 * n:(b0 + k) * n].to(dev)
        Lm.select_collect(sc, Lm.select_submit(sc, mlp, Xd, off_full[:k + 1]), scored=scored,
                          as_arrays=True)
    torch.cuda.synchronize()
    prof = kde.profile_read()
    kde.profile_enable(False)
    # the method without the network: the normal-reference bandwidth refined
    # over the same neighbourhood (first 512 held-out datasets)
    reg_ref = []
    for i in range(min(512, K)):
        sc.prepare(evals_t[i * n:(i + 1) * n].to(dev))
        ref = Lm.normal_reference_theta(n)
        s_ref = sc.scores(np.stack([Lm.theta_to_H(t) for t in Lm.neighbourhood(ref)])).cpu().numpy()
        reg_ref.append((s_ref.min() - best[i]) / abs(best[i]))
    rel_regret = (got - best) / np.abs(best)
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1],
                   "share": v[0] / max(1e-12, sum(x[0] for x in prof.values()))}
               for k, v in prof.items()}
    # roofline of the selection loop's dominant kernel
    info = sc.plan.info
    # supports of every scored H and 2H (Eq. 15, corrected range), vectorised
    Hs = np.asarray(scored, dtype=np.float64).reshape(-1, 2, 2)
    Hs = np.concatenate([Hs, 2.0 * Hs])
    lam = 0.5 * (Hs[:, 0, 0] + Hs[:, 1, 1]) + np.sqrt(
        0.25 * (Hs[:, 0, 0] - Hs[:, 1, 1]) ** 2 + Hs[:, 0, 1] ** 2)
    Mg = np.array(sc.M, dtype=np.float64)
    dlt = (np.array(sc.hi) - np.array(sc.lo)) / (Mg - 1.0)
    Lv = np.minimum(Mg - 1.0, np.ceil(sc.tau * np.sqrt(lam)[:, None] / dlt[None, :]))
    # every matrix scored in the profiled pass (its first nprof datasets)
    ac_total = float(np.sum(8.0 * (Lv[:, 0] + 1.0) * (2.0 * Lv[:, 1] + 1.0)))
    flops = {"kde_lscv_ac_kernel": ac_total, "kde_lscv_theta_sums_kernel": ac_total,
             "kde_gemm_tc_kernel": nprof * 2.0 * 128 * (din * hid + hid * hid + hid * 16)}
    dom = max(prof, key=lambda k: prof[k][0])
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    cells = Lm.GRID_M * Lm.GRID_M
    P0, P1, Q = info.P[0], info.P[1], info.Q
    # per-launch algorithmic bytes of the batched preparation (Bsel datasets)
    nbytes = {"kde_standardize2_sets_kernel": Bsel * 16.0 * n,
              "kde_bin_sets_kernel": Bsel * (8.0 * n + 8.0 * cells),
              "kde_features2_sets_kernel": Bsel * (8.0 * cells + 4.0 * kde.FEAT_DIM),
              "kde_rows_r2c_counts_kernel": Bsel * (8.0 * cells + Lm.GRID_M * Q * 8.0),
              "kde_cols_auto_kernel": Bsel * (Lm.GRID_M * Q * 8.0 + P0 * Q * 8.0),
              "kde_rows_c2r_kernel": Bsel * (P0 * Q * 8.0 + P0 * P1 * 4.0)}
    # the same passes on the two-phase engine
    for k in ("kde_rows_r2c_counts_kernel", "kde_cols_auto_kernel", "kde_rows_c2r_kernel"):
        nbytes[k.replace("kde_", "kde_fx_", 1)] = nbytes[k]
    hbm, hbm_kind = peaks()
    if dom == "kde_gemm_tc_kernel":
        ach = flops[dom] / (prof[dom][0] * 1e-3) / 1e12
        roofline = {"bound": "tensor", "kernel": dom, "achieved": ach, "peak": peak_bf16,
                    "unit": "TFLOP/s", "frac": ach / peak_bf16, "traffic": None,
                    "peak_source": "measured (bf16 burst)",
                    "flops_per_launch": flops[dom] / prof[dom][1]}
    elif dom in flops:
        ach = flops[dom] / (prof[dom][0] * 1e-3) / 1e12
        peak = fp32_peak_tflops(sm_max)
        roofline = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x SM max clock",
                    "flops_per_launch": flops[dom] / prof[dom][1]}
    elif dom in nbytes:
        ach = nbytes[dom] / (prof[dom][0] / prof[dom][1] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "peak_source": hbm_kind, "traffic": None,
                    "algorithmic_bytes": nbytes[dom]}
    else:
        roofline = {"bound": None, "kernel": dom, "achieved": None, "peak": None,
                    "unit": None, "frac": None, "traffic": None}
    line = {"metric": LEARN_METRIC, "value": K / t_learn, "unit": "datasets/s",
            "n_gpus": 1, "steps": K, "warmup": Bsel, "ms_per_step": 1e3 * t_learn / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic",
            "config": {"workload": "learned2d_256", "grid": [256, 256], "n": n,
                       "train_datasets": n_train, "test_datasets": K,
                       "candidates_plain": int(len(sc.cand)), "P": list(info.P),
                       "mlp": f"{kde.FEAT_DIM}-256-256-3 ReLU, BF16 operands, FP32 accumulation",
                       "timing": "wall clock around the loop with device synchronisation; each "
                                 "batch's samples copied from pinned host memory inside it, on a "
                                 "copy stream beside the previous batch's work",
                       "batch": Bsel, "dataset_workers": workers},
            "plain_search": {"value": K / t_plain, "unit": "datasets/s",
                             "ms_per_dataset": 1e3 * t_plain / K,
                             "gpu_launches": launches_plain,
                             "kernel_ms_per_dataset": {k: v[0] / nprof for k, v in prof_plain.items()}},
            "speedup_vs_plain": t_plain / t_learn,
            "quality": {"mean_rel_regret": float(rel_regret.mean()),
                        "p95_rel_regret": float(np.percentile(rel_regret, 95)),
                        "fraction_exact_best": float(np.mean(rel_regret <= 1e-12)),
                        "fallbacks": fell, "mean_candidates": ncand / K,
                        "normal_reference_refined_mean_rel_regret": float(np.mean(reg_ref))},
            "labels": {"datasets_per_s": n_train / t_label, "seconds": t_label,
                       "generation_wait_s": t_gen},
            "training": {"samples_per_s": steps_train * batch / t_train, "epochs": epochs,
                         "seconds": t_train, "loss_first_last": [hist[0], hist[-1]],
                         "gemm_tflops": gemm_tf, "gemm_frac_of_bf16_peak": gemm_tf / peak_bf16},
            "roofline": roofline, "kernels": kernels, "gpu_launches": launches_learn,
            "clocks": clocks}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
