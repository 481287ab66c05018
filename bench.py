#!/usr/bin/env python
"""Benchmark of the LRDM Gateaux-derivative hot path on GB300.

Metric: Gateaux derivatives per second at a 96^3 grid (884,736 points),
N_s = 4096, K = 16 directions (one derivative = one (system, direction) f_k).
One step = one pass of the whole path over one batch of K directions:
Hartree + LDA kernel, projection GEMM, mu' and Loewner scaling, response GEMM
with the f = drho - v epilogue (lrdm_gateaux_batch), the K x K least-squares
step and update (lrdm_apply), and the hand-written adjoint of the response
map and of the eigenvalue / occupation inputs for one cotangent per direction
(lrdm_backward).  The forward call alone (one CUDA-graph replay of
lrdm_gateaux_batch) is timed separately and reported under "forward_only",
with and without the Poisson (cuFFT) step.  A periodic workload sampled at
4 Brillouin-zone points (48^3 grid, N_s = 512 complex states per point, K = 8,
same precision; lrdm_kp_gateaux) is timed after the main step and reported under
"kpoint" with its own roofline and oracle baseline (--kpoint-only runs it
alone).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x3|tf32|fp32|fp64]
  python bench.py --impl reference ...     (the FP64 CPU oracle, timed on the host)

Inputs are seeded and synthetic (workloads/), resident in HBM when the timed
region starts and larger than L2 (the Psi operand copies are ~29 GB).  With
torchrun (N > 1) every rank runs an independent system (weak scaling, no
data-path collective); value = all ranks' derivatives / max-over-ranks time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gateaux derivatives/sec at 96^3 grid, N_s=4096, K=16; tensor-pipe % vs FP64 plain form"
GRID = (96, 96, 96)
H = (0.5, 0.5, 0.5)
NS = 4096
KDIR = 16
NE = 3700.0
KT = 0.005
# The paper's own results (whole SCF, not this step; context only)
PAPER_CONTEXT = {
    "hardware": "NERSC Perlmutter Phase 1 nodes (4x A100 + 64-core AMD Milan); some runs on OLCF Summit (6x V100)",
    "scf_iterations_lrdm": "22-31 on the benchmark systems (3-5x fewer than Anderson / Kerker / Broyden-TFW)",
    "scf_cost_reduction_vs_kerker": "up to 3.4x (213.30 -> 63.5 GPU node-hours, Pt+GaAs+SiO2H 40 layers)",
    "lrdma_rank_reduction": "1.5-1.8x lower average rank",
    "gateaux_step_rate": "not reported",
}
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="bf16x3", choices=["bf16x3", "tf32", "fp32", "fp64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="use the default launch shape instead of tuning at create")
    p.add_argument("--no-fp64-plain", action="store_true",
                   help="skip timing the plain FP64 GPU form")
    p.add_argument("--grid", type=int, default=96, help="grid edge (96 = the benchmark workload)")
    p.add_argument("--ns", type=int, default=NS)
    p.add_argument("--fwd-reps", type=int, default=20,
                   help="graph replays of the forward call timed for forward_only")
    p.add_argument("--no-kpoint", action="store_true",
                   help="skip the Brillouin-zone-sampled (k-point) leg")
    p.add_argument("--kpoint-only", action="store_true",
                   help="run only the k-point leg and print its JSON")
    p.add_argument("--jsonl", default=None,
                   help="also append the result line (with a UTC timestamp and the host) to this JSONL file")
    p.add_argument("--config", type=int, default=0, choices=[0, 1, 2, 3, 4],
                   help="instead of the benchmark step, time the forward call of another workload "
                        "(1: 16^3 toy model, 2: 48^3 / 512, 3: the uneven batch with its spin pair, "
                        "4: 72^3 / 2048 with near-degenerate pairs) in its precisions, with the FP64 "
                        "oracle timed on the host cores in full and the error of every precision")
    p.add_argument("--prec-list", default="",
                   help="with --config: comma-separated precisions instead of the config's own")
    p.add_argument("--shard", default="replicas", choices=["replicas", "directions", "rows"],
                   help="N > 1: an independent system per rank (weak scaling); one system whose "
                        "K directions are split over the ranks, f all-gathered before the "
                        "least-squares step on every rank; or one system whose grid rows are "
                        "split over the ranks (lrdm_create_rows: the Poisson input, X_k and the "
                        "least-squares sums summed by NCCL) (both strong scaling)")
    p.add_argument("--no-batched", action="store_true",
                   help="skip timing the uneven batch (64 derivatives per call) after the main step")
    p.add_argument("--compare-fp64", action="store_true",
                   help="time the plain FP64 GPU form (torch, Psi X' materialised) and the "
                        "library's FP64 path on a 48^3 slice instead of the benchmark step")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


TC_SOURCES = ("paper_2211_07894_gb300/csrc/k_tc.cu", "paper_2211_07894_gb300/csrc/tc_ptx.cuh",
              "paper_2211_07894_gb300/csrc/tc_problem.h")


def tc_source_hash():
    """SHA-256 of the tensor-core kernel sources (the DRAM counters recorded
    under profiles/ are valid only for the sources they were taken with)."""
    import hashlib
    h = hashlib.sha256()
    for rel in TC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_value(record, field, kernel, workload, shape, same_tile=False):
    """A per-launch ncu figure of `kernel` on `workload` in launch shape
    `shape` (the kernel's own tuning fields, e.g. 'g1_nb=256,g1_dpt=1') from
    the summaries under profiles/ (lines '<record>: kernel=... workload=...
    shape=... source_sha256=... <field>=...'), or None when no record matches
    the current kernel sources and shape.  same_tile: a record whose shape
    differs only after its first field (the tile width; the rest orders the
    work items) also matches, when no exact one does."""
    import glob
    want = tc_source_hash()
    near = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for line in fh:
                line = line.strip().strip("`")
                if not line.startswith(record + ":"):
                    continue
                f = dict(kv.split("=", 1) for kv in line.split()[1:] if "=" in kv)
                if (f.get("kernel") != kernel or f.get("workload") != workload
                        or f.get("source_sha256") != want or field not in f):
                    continue
                if f.get("shape") == shape:
                    return float(f[field])
                if (same_tile and shape and f.get("shape", "").split(",")[0] == shape.split(",")[0]
                        and near is None):
                    near = float(f[field])
    return near


def recorded_traffic(kernel, workload, shape):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)."""
    return recorded_value("traffic-record", "dram_bytes_per_launch", kernel, workload, shape)


def recorded_tensor_pipe(kernel, workload, shape):
    """sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_elapsed, %
    (a record of the same tile width when the work-item order differs)."""
    return recorded_value("tensor-pipe-record", "pct_of_elapsed", kernel, workload, shape, same_tile=True)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and --impl reference)
# ---------------------------------------------------------------------------

ORACLE_SAMPLE_GRID = (24, 24, 24)


def oracle_sample_system():
    """A bounded sample of the benchmark workload for the FP64 CPU oracle: the
    same N_s = 4096 subspace size, kT, filling and recipes on a 24^3 grid
    (1/64 of the 96^3 rows), one direction.  Both contractions scale linearly
    with the number of grid rows, so GD/s at 96^3 = 1 / (t_sample * 64)."""
    import numpy as np
    import oracle
    import workloads
    n = ORACLE_SAMPLE_GRID
    rng = workloads.rng_for(5, 50)
    psi = workloads.random_subspace(n, H, NS, rng)
    eps = workloads.random_eigenvalues(NS, rng)
    mu = oracle.solve_mu([eps], NE, KT, 2.0)
    rho = oracle.density(psi, oracle.fermi(eps, mu, KT), 2.0, 1e-3)
    sysm = oracle.System(n=n, h=H, psi=[psi], eps=[eps], rho=[rho], n_electrons=NE, kT=KT, g=2.0)
    V = workloads.smooth_directions(n, H, 1, 1, workloads.rng_for(5, 51))
    R = workloads.smooth_field(n, H, 0.1, workloads.rng_for(5, 52))[None, :]
    scale = float(np.prod(GRID)) / float(np.prod(n))
    return sysm, V, R, scale


def oracle_step(sysm, V, R):
    import oracle
    res = oracle.gateaux(sysm, V)
    oracle.lrdm_apply(R, V, res["F"], sysm.w, 0.5, rho=sysm.rho[0][None, :])
    oracle.backward(sysm, res["F"], res)


# the same oracle step on one host core: a 16^3 sample (the smallest grid that
# holds N_s = 4096 orthonormal states; 1/216 of the 96^3 rows)
ORACLE_1T_GRID = (16, 16, 16)


def one_thread_child(path):
    """Runs in a child process whose BLAS pools have one thread: loads the
    sample written by time_oracle_one_thread, times one oracle step, prints
    the seconds."""
    import numpy as np
    import oracle
    d = np.load(path)
    n = tuple(int(x) for x in d["n"])
    sysm = oracle.System(n=n, h=H, psi=[d["psi"]], eps=[d["eps"]], rho=[d["rho"]], n_electrons=NE,
                         kT=KT, g=2.0)
    t0 = time.perf_counter()
    oracle_step(sysm, d["V"], d["R"])
    print(time.perf_counter() - t0)


def time_oracle_one_thread():
    """The oracle step on one core, beside the all-cores figure: the sample
    is built here with every core, the step is timed in a child process with
    OPENBLAS / OMP / MKL threads = 1.  GD/s scaled by the row ratio; None
    when the child fails."""
    import tempfile
    import numpy as np
    global ORACLE_SAMPLE_GRID
    saved = ORACLE_SAMPLE_GRID
    ORACLE_SAMPLE_GRID = ORACLE_1T_GRID
    try:
        sysm, V, R, scale = oracle_sample_system()
    finally:
        ORACLE_SAMPLE_GRID = saved
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "sample.npz")
        np.savez(path, n=np.asarray(ORACLE_1T_GRID), psi=sysm.psi[0], eps=sysm.eps[0], rho=sysm.rho[0],
                 V=V, R=R)
        try:
            r = subprocess.run([sys.executable, "-c", f"import bench; bench.one_thread_child({path!r})"],
                               cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
            sec = float(r.stdout.strip().splitlines()[-1])
        except Exception:
            return None
    return {"value": 1.0 / (sec * scale), "unit": "GD/s", "cores": 1, "seconds": sec,
            "sample": f"oracle.gateaux + lrdm_apply + backward, K=1, N_s={NS}, grid {ORACLE_1T_GRID[0]}^3 "
                      f"(1/{int(scale)} of the 96^3 rows), one BLAS thread; GD/s scaled by the row ratio"}


def cpu_model():
    """The host CPU's model name (lscpu), else what platform reports."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# Brillouin-zone-sampled response (lrdm_kp_gateaux): a periodic workload of
# nk k-points with complex subspaces, timed beside the main step.
KP_GRID = (48, 48, 48)
KP_NS, KP_NK, KP_K, KP_NE, KP_KT = 512, 4, 8, 800.0, 0.01
KP_SAMPLE_GRID = (24, 24, 24)


def kp_weights(nk):
    raw = [1.0 + 2.0 * min(i, nk - 1 - i) for i in range(nk)]
    return [x / sum(raw) for x in raw]


def time_kpoint(torch, rank, prec, autotune=True, reps=5, warmup=2):
    """K = 8 real directions through lrdm_kp_gateaux on a 48^3 grid with 4
    k-points of N_s = 512 complex states each (tensor-core precisions: the
    real contractions on the stacked 2 N_s = 1024-column operand); the
    projection kernel's roofline from the library's own event timing."""
    import workloads
    from paper_2211_07894_gb300 import KpContext
    rng = workloads.rng_for(80, rank)
    pr, pi = [], []
    for q in range(KP_NK):
        a, b = workloads.random_subspace_complex_torch(KP_GRID, H, KP_NS, 2211078940 + 80 + 10 * rank + q,
                                                       "cuda")
        pr.append(a)
        pi.append(b)
    eps = [torch.as_tensor(workloads.random_eigenvalues(KP_NS, rng) + 0.02 * q, device="cuda")
           for q in range(KP_NK)]
    ctx = KpContext(KP_GRID, H, pr, pi, eps, kp_weights(KP_NK), KP_NE, KP_KT, rho_floor=1e-3,
                    prec=prec, io_dtype=torch.float32, k_max=KP_K, autotune=autotune)
    tuning = ctx.tuning() if prec in ("bf16x3", "tf32") else None
    split = ctx.split(KP_K)
    del pr, pi
    V = torch.as_tensor(workloads.smooth_directions(KP_GRID, H, KP_K, 1, workloads.rng_for(80, 100 + rank))[:, 0],
                        dtype=torch.float32, device="cuda").contiguous()
    F = torch.empty_like(V)
    dmu = torch.empty(KP_K, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        ctx.gateaux(V, out=F, dmu=dmu)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.gateaux(V, out=F, dmu=dmu)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_read(reset=True)
    ms = e0.elapsed_time(e1) / reps
    if ctx.status() != 0:
        raise RuntimeError("device status not ok after the k-point calls")
    ctx.close()
    ng = int(KP_GRID[0] * KP_GRID[1] * KP_GRID[2])
    # the projection work of one call (all k-points): per k-point and
    # direction the upper triangle of the complex N_s x N_s product, 8 real
    # flops per (row, i <= j), = the symmetric half of the stacked real
    # (2 N_s)^2 Gram, 2 flops per (row, i, j) / 2
    alg = KP_NK * KP_K * 4.0 * ng * KP_NS * KP_NS
    per_call = prof["gemm1_ms"] / max(prof["gemm1_launches"], 1) / 1e3   # one event per call
    peaks, src = load_peaks()
    peak, bound, issue, note = dtype_peak(prec, peaks)
    issued = issue * alg
    if prec in ("bf16x3", "tf32"):
        kname = "k_gemm1_pair" if tuning and tuning["g1_nb"] == 512 else "k_gemm1_tc"
    else:
        kname = "k_kp_gemm1<float>" if prec == "fp32" else "k_kp_gemm1<double>"
    achieved = issued / per_call / 1e12
    traffic = None
    if tuning:
        traffic = recorded_traffic(kname, f"{KP_GRID[0]}^3/kp{KP_NK}x{KP_NS}/K{KP_K}/{prec}",
                                   f"g1_nb={tuning['g1_nb']},g1_dpt={tuning['g1_dpt']},split={split}")
    return {"workload": f"{KP_GRID[0]}^3 grid, {KP_NK} k-points x N_s={KP_NS} complex, K={KP_K}, {prec}",
            "value": KP_K / (ms / 1e3), "unit": "GD/s", "ms_per_call": ms, "reps": reps,
            "launch_shape": tuning, "projection_row_ranges": split,
            "gemm1_ms_per_call": prof["gemm1_ms"] / reps, "gemm2_ms_per_call": prof["gemm2_ms"] / reps,
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                         "gemm1_ms_per_call": per_call * 1e3, "alg_flop_per_call": alg,
                         "peak_source": f"{src}; {note}"}}


def time_kpoint_oracle():
    """The oracle's gateaux_kpoints on a bounded sample of the k-point
    workload: the same 4 k-points x N_s = 512, one direction, a 24^3 grid (1/8
    of the rows); both contractions scale linearly with the rows."""
    import numpy as np
    import oracle
    import workloads
    n = KP_SAMPLE_GRID
    rng = workloads.rng_for(81, 0)
    psi = [workloads.random_subspace_complex(n, H, KP_NS, rng) for _ in range(KP_NK)]
    eps = [workloads.random_eigenvalues(KP_NS, rng) + 0.02 * q for q in range(KP_NK)]
    kw = kp_weights(KP_NK)
    ks = oracle.KpointSystem(n=n, h=H, psi=psi, eps=eps, k_weights=kw, rho=np.zeros(int(np.prod(n))),
                             n_electrons=KP_NE, kT=KP_KT)
    mu = oracle.solve_mu_kpoints(eps, kw, KP_NE, KP_KT, 2.0)
    ks.rho = oracle.density_kpoints(ks, mu, 1e-3)
    V = workloads.smooth_directions(n, H, 1, 1, workloads.rng_for(81, 1))[:, 0]
    t0 = time.perf_counter()
    oracle.gateaux_kpoints(ks, V)
    dt = time.perf_counter() - t0
    scale = float(np.prod(KP_GRID)) / float(np.prod(n))
    return {"value": 1.0 / (dt * scale), "unit": "GD/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"oracle.gateaux_kpoints, K=1, {KP_NK} k-points x N_s={KP_NS}, grid {n[0]}^3 "
                      f"(1/{int(scale)} of the {KP_GRID[0]}^3 rows); GD/s scaled by the row ratio"}


def append_jsonl(path, line):
    """One run record per line: the bench line plus when and where it ran."""
    import platform
    rec = dict(line)
    rec["time_utc"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    rec["host"] = {"machine": platform.machine(), "cores": os.cpu_count(), "python": platform.python_version()}
    with open(path, "a") as fh:
        fh.write(json.dumps(rec) + "\n")


def cpu_cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            try:
                return int(os.environ[var])
            except ValueError:
                pass
    return os.cpu_count()


def time_oracle(steps, warmup):
    sysm, V, R, scale = oracle_sample_system()
    for _ in range(warmup):
        oracle_step(sysm, V, R)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_step(sysm, V, R)
    dt = (time.perf_counter() - t0) / max(steps, 1)
    gds = 1.0 / (dt * scale)     # one direction per step, scaled to 96^3 rows
    sample = (f"oracle.gateaux + lrdm_apply + backward, K=1, N_s={NS}, grid {ORACLE_SAMPLE_GRID[0]}^3 "
              f"(1/{int(scale)} of the 96^3 rows), {steps} step(s); GD/s scaled by the row ratio")
    return gds, dt, sample


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    if (world > 1 and "numpy" not in sys.modules and os.environ.get("OMP_NUM_THREADS") == "1"
            and not os.environ.get("OPENBLAS_NUM_THREADS")):
        # torchrun starts every rank with one OpenMP thread; rank 0 is the only
        # rank working here, so its BLAS gets the host's cores (an explicit
        # OPENBLAS_NUM_THREADS is left as set)
        n = str(os.cpu_count() or 1)
        os.environ["OMP_NUM_THREADS"] = n
        os.environ["OPENBLAS_NUM_THREADS"] = n
    steps = max(1, args.steps)
    gds, dt, sample = time_oracle(steps, max(0, min(args.warmup, 1)))
    line = {"impl": "reference", "metric": METRIC, "value": gds, "unit": "GD/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"96^3 grid, N_s={NS}, K={KDIR} (oracle on a bounded sample)",
                       "grid": list(GRID), "n_s": NS, "K": KDIR},
            "cpu_baseline": {"value": gds, "unit": "GD/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model(),
                             "one_thread": time_oracle_one_thread()},
            "e2e": {"value": gds, "unit": "GD/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

# Peaks that MEASURED_PEAKS does not carry, measured on the GB300s
# with the same method (torch.matmul, CUDA events; best of 10 for the burst
# figure, back to back for 4 s for the sustained one): TF32 8192^3 1022 TF/s
# burst, 909 sustained; FP64 4096^3 1.10 (burst = sustained); FP32 without
# tensor cores 69.8 (the roofline below uses the FMA peak instead).
PEAK_TF32_SUSTAINED = 908.7
PEAK_FP64 = 1.10


def dtype_peak(prec, peaks):
    """(peak TF/s, bound, issued products per algorithmic product, note)
    of a contraction in precision prec."""
    bf = peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
    if prec == "bf16x3":
        return bf, "tensor", 3.0, "bf16x3 issues 3 bf16 MMAs per product; achieved = issued bf16 rate"
    if prec == "tf32":
        if PEAK_TF32_SUSTAINED:
            return (PEAK_TF32_SUSTAINED, "tensor", 1.0,
                    "tf32 peak = measured torch TF32 matmul, sustained (8192^3, 4 s)")
        return 0.5 * bf, "tensor", 1.0, "tf32 peak = bf16 sustained x 1/2 (nominal ratio)"
    if prec == "fp32":
        return 152 * 128 * 2 * 2.07e9 / 1e12, "alu", 1.0, "FP32 FMA peak = 152 SMs x 128 lanes x 2 x 2.07 GHz"
    return PEAK_FP64, "alu", 1.0, f"FP64 peak = measured torch FP64 matmul ({PEAK_FP64} TF/s)"


def oracle_system_for(cfg):
    """oracle.System of a workloads config: occupations, mu and the density
    g sum f psi^2 + floor from the oracle itself."""
    import numpy as np
    import oracle
    g = cfg["g"]
    mu = oracle.solve_mu(cfg["eps"], cfg["n_electrons"], cfg["kT"], g)
    occ = [oracle.fermi(e, mu, cfg["kT"]) for e in cfg["eps"]]
    rho = [oracle.density(p, o, g, cfg["rho_floor"]) for p, o in zip(cfg["psi"], occ)]
    return oracle.System(n=cfg["n"], h=cfg["h"], psi=[np.asarray(p, dtype=np.float64) for p in cfg["psi"]],
                         eps=[np.asarray(e, dtype=np.float64) for e in cfg["eps"]], rho=rho,
                         n_electrons=cfg["n_electrons"], kT=cfg["kT"], g=g)


CONFIG_LEGS = {
    1: ("16^3 FD toy model (8 Gaussian wells, dense eigenpairs), N_s=32, N_e=24, kT=0.01, K=4",
        ["fp64"]),
    2: ("48^3 grid, N_s=512, N_e=460, kT=0.005, K=8 (random subspace under a smooth envelope)",
        ["fp64", "fp32", "tf32", "bf16x3"]),
    3: ("6 uneven systems (32^3/256/K4 .. 64^3/1024/K16) + spin pair (64^3, 768/704, K8): "
        "64 derivatives per call, FP32 storage", ["bf16x3", "tf32", "fp32"]),
    4: ("72^3 grid, N_s=2048, N_e=1800, kT=0.002, K=12, 5% near-degenerate pairs (gap 1e-9 Ha)",
        ["fp64", "fp32", "tf32", "bf16x3"]),
}


def config_inputs(n):
    import workloads
    if n == 1:
        return [workloads.config1()]
    if n == 2:
        return [workloads.config2()]
    if n == 3:
        return workloads.config3()
    return [workloads.config4()]


def time_forward(torch, ctx, V, reps_max=20, budget_s=10.0):
    """Median of CUDA-event timed forward calls (graph replays: the context
    is created with use_graph and the calls run on a non-default stream)."""
    stream = torch.cuda.current_stream()
    F = [torch.empty_like(v) for v in V]
    ctx.gateaux(V, out=F)              # captures the graph
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    ctx.gateaux(V, out=F)
    a1.record(stream)
    torch.cuda.synchronize()
    first = a0.elapsed_time(a1)
    reps = int(max(3, min(reps_max, budget_s * 1e3 / max(first, 1e-3))))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for b0, b1 in ev:
        b0.record(stream)
        ctx.gateaux(V, out=F)
        b1.record(stream)
    torch.cuda.synchronize()
    ms = sorted(b0.elapsed_time(b1) for b0, b1 in ev)
    return statistics.median(ms), reps, F


def gpu_config_run(torch, cfgs, prec, refs, peaks, autotune=True):
    """One precision of a config leg: forward GD/s (graph replays), the
    contractions' rates from one profiled (eager) call, the error of every
    direction against the oracle's results."""
    import numpy as np
    from paper_2211_07894_gb300 import Context
    io = torch.float64 if prec == "fp64" else torch.float32
    systems, V = [], []
    for c in cfgs:
        d = dict(n=c["n"], h=c["h"], n_electrons=c["n_electrons"], kT=c["kT"], g=c["g"],
                 rho_floor=c["rho_floor"], k_max=c["V"].shape[0])
        d["psi"] = [torch.as_tensor(np.ascontiguousarray(p), dtype=io, device="cuda") for p in c["psi"]]
        d["eps"] = [torch.as_tensor(np.ascontiguousarray(e), dtype=torch.float64, device="cuda")
                    for e in c["eps"]]
        systems.append(d)
        V.append(torch.as_tensor(np.ascontiguousarray(c["V"]), dtype=io, device="cuda"))
    tc = prec in ("bf16x3", "tf32")
    ctx = Context(systems, prec=prec, io_dtype=io, k_max=max(c["V"].shape[0] for c in cfgs),
                  use_graph=True, autotune=autotune and tc)
    del systems
    ms, reps, F = time_forward(torch, ctx, V)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    ctx.gateaux(V, out=F)
    torch.cuda.synchronize()
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    if ctx.status() != 0:
        raise RuntimeError(f"device status not ok ({prec})")
    errs = []
    for f, ref in zip(F, refs or []):
        fh = f.double().cpu().numpy()
        for k in range(fh.shape[0]):
            b = ref["F"][k]
            errs.append(float(np.sqrt(np.sum((fh[k] - b) ** 2) / np.sum(b * b))))
    ktot = sum(c["V"].shape[0] for c in cfgs)
    alg = sum(c["V"].shape[0] * int(np.prod(c["n"])) * sum(p.shape[1] ** 2 for p in c["psi"]) for c in cfgs)
    peak, bound, issue, note = dtype_peak(prec, peaks)
    rates = {}
    for key, t, n in (("projection", prof["gemm1_ms"], prof["gemm1_launches"]),
                      ("response", prof["gemm2_ms"], prof["gemm2_launches"])):
        r = issue * alg / (t / 1e3) / 1e12 if t > 0 else None
        rates[key] = {"ms": t, "launches": n, "achieved_tflops": r, "peak": peak,
                      "frac": r / peak if r else None}
    out = {"gd_s": ktot / (ms / 1e3), "ms_median": ms, "replays": reps, "graph": True,
           "err_f_max": max(errs) if errs else None,
           "err_f_median": statistics.median(errs) if errs else None,
           "bound": bound, "peak_source": note, "contractions": rates,
           "gpu_launches_per_call": prof["kernel_launches"],
           "launch_shape": ctx.tuning() if tc else None}
    ctx.close()
    torch.cuda.empty_cache()
    return out


def config_leg(args, torch):
    import numpy as np
    import oracle
    n = args.config
    desc, precs = CONFIG_LEGS[n]
    if args.prec_list:
        precs = [p for p in args.prec_list.split(",") if p]
    cfgs = config_inputs(n)
    ktot = sum(c["V"].shape[0] for c in cfgs)
    t0 = time.perf_counter()
    refs = [oracle.gateaux(oracle_system_for(c), c["V"]) for c in cfgs]
    t_or = time.perf_counter() - t0
    peaks, peak_src = load_peaks()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    gpu = {p: gpu_config_run(torch, cfgs, p, refs, peaks, autotune=not args.no_autotune) for p in precs}
    clocks = sampler.stop()
    line = {"leg": "config", "config_id": n, "workload": desc, "derivatives_per_call": ktot,
            "unit": "GD/s", "data": "synthetic",
            "oracle": {"gd_s": ktot / t_or, "seconds": t_or, "cores": cpu_cores(), "cpu_model": cpu_model(),
                       "kind": "oracle", "sample": "full run: oracle.gateaux over every direction"},
            "gpu": gpu, "clocks": clocks, "peaks_source": peak_src}
    print(json.dumps(line), flush=True)
    if args.jsonl:
        append_jsonl(args.jsonl, line)
    return 0

def build_problem(torch, rank, prec, edge, ns, autotune=True, rows=None):
    import numpy as np
    import workloads
    from paper_2211_07894_gb300 import Context
    n = (edge, edge, edge)
    ng = int(np.prod(n))
    if ng * ns <= 200_000_000:
        # small cases (profiling runs): the host QR of the same recipe
        psi = torch.as_tensor(workloads.random_subspace(n, H, ns, workloads.rng_for(5, 10 * rank + 3)),
                              dtype=torch.float32, device="cuda")
    else:
        psi = workloads.random_subspace_torch(n, H, ns, seed=2211078940 + 50 + rank, device="cuda")
    rng = workloads.rng_for(5, 10 * rank)
    eps = torch.as_tensor(workloads.random_eigenvalues(ns, rng), dtype=torch.float64,
                          device="cuda")
    V = torch.as_tensor(workloads.smooth_directions(n, H, KDIR, 1, workloads.rng_for(5, 10 * rank + 1)),
                        dtype=torch.float32, device="cuda")
    R = torch.as_tensor(workloads.smooth_field(n, H, 0.1, workloads.rng_for(5, 10 * rank + 2))[None, :],
                        dtype=torch.float32, device="cuda")
    ne = NE * ns / NS
    system = dict(n=n, h=H, psi=[psi], eps=[eps], n_electrons=ne, kT=KT, g=2.0,
                  rho_floor=1e-3, k_max=KDIR)
    io = torch.float32 if prec != "fp64" else torch.float64
    if io == torch.float64:
        system["psi"] = [psi.double()]
        V, R = V.double(), R.double()
    kw = {}
    if rows is not None:
        # grid rows [r0, r1) of the one shared system on this rank
        r0, r1, fn = rows
        system["psi"] = [system["psi"][0][r0:r1].contiguous()]
        V, R = V[:, :, r0:r1].contiguous(), R[:, r0:r1].contiguous()
        kw["rows"] = dict(row_begin=r0, n_rows=r1 - r0, allreduce=fn)
    ctx = Context([system], prec=prec, io_dtype=io, k_max=KDIR, use_graph=True,
                  autotune=autotune and prec in ("bf16x3", "tf32"), **kw)
    del psi, system
    torch.cuda.empty_cache()
    return ctx, V, R, ng


FP64_SAMPLE_GRID = (48, 48, 48)


def time_fp64_plain(torch, reps=1, with_library=False):
    """The plain FP64 GPU form: per direction, X = Psi^T (a o Psi) and
    drho = rowsum((Psi X') o Psi) with dense torch FP64 matmuls (Psi X'
    materialised), for one direction on a 48^3 grid with N_s = 4096 (1/8 of
    the 96^3 rows; both products are linear in the rows, so GD/s at 96^3 =
    1 / (8 t)).  The two dense products are > 99 % of the plain form's work;
    its element-wise steps are not timed.  with_library also times this
    library's FP64 path on the same slice."""
    import numpy as np
    import workloads
    from paper_2211_07894_gb300 import Context
    n = FP64_SAMPLE_GRID
    ng = int(np.prod(n))
    scale = float(np.prod(GRID)) / ng
    psi32 = workloads.random_subspace_torch(n, H, NS, seed=2211078940 + 60, device="cuda")
    psi = psi32.double()
    del psi32
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    a = torch.randn(ng, dtype=torch.float64, device="cuda", generator=g)
    Xp = torch.randn(NS, NS, dtype=torch.float64, device="cuda", generator=g)
    Xp = Xp + Xp.T

    def plain():
        X = psi.T @ (a[:, None] * psi)
        d = ((psi @ Xp) * psi).sum(dim=1)
        return X, d

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    out = {}
    t_plain = timed(plain)
    out["plain-fp64-gpu"] = t_plain
    if with_library:
        eps = torch.as_tensor(workloads.random_eigenvalues(NS, workloads.rng_for(5, 60)), device="cuda")
        V = torch.as_tensor(workloads.smooth_directions(n, H, 1, 1, workloads.rng_for(5, 61)),
                            dtype=torch.float64, device="cuda")
        ctx = Context([dict(n=n, h=H, psi=[psi], eps=[eps], n_electrons=NE, kT=KT, g=2.0,
                            rho_floor=1e-3, k_max=1)], prec="fp64", io_dtype=torch.float64, k_max=1)
        F = torch.empty_like(V)
        out["library-fp64"] = timed(lambda: ctx.gateaux([V], out=[F]))
        ctx.close()
    del psi, a, Xp
    torch.cuda.empty_cache()
    sample = (f"1 direction, {n[0]}^3 grid, N_s={NS}, {reps} timed rep(s); GD/s scaled by the "
              f"{int(scale)}x row ratio")
    return {k: (1.0 / (t * scale), t * scale) for k, t in out.items()}, sample


def compare_fp64(args):
    import torch
    torch.cuda.set_device(0)
    res, sample = time_fp64_plain(torch, reps=2, with_library=True)
    for impl, (gds, sec) in res.items():
        print(json.dumps({"impl": impl, "metric": METRIC, "value": gds, "unit": "GD/s",
                          "dtype": "f64", "sample": sample,
                          "seconds_per_direction_at_96^3": sec}), flush=True)
    return 0


def time_forward_calls(torch, ctx, V, F, dmu, prof, args, world):
    """The forward call alone (CUDA-graph replays of lrdm_gateaux_batch, K
    directions and one direction)."""
    stream = torch.cuda.current_stream()
    ctx.gateaux([V], out=[F], dmu=dmu)          # captures the graph
    torch.cuda.synchronize()
    reps = max(args.fwd_reps, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for a0, a1 in ev:
        a0.record(stream)
        ctx.gateaux([V], out=[F], dmu=dmu)
        a1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = sorted(a0.elapsed_time(a1) for a0, a1 in ev)
    fwd_med = statistics.median(fwd_ms)
    # Poisson per forward call (one solve per call; the backward makes one more)
    poisson_fwd = prof["poisson_ms"] / max(prof["poisson_calls"], 1)
    forward_only = {"value": KDIR * world / (fwd_med / 1e3), "unit": "GD/s",
                    "ms_median": fwd_med, "ms_min": fwd_ms[0], "replays": reps,
                    "graph": True, "poisson_ms": poisson_fwd,
                    "value_without_poisson": KDIR * world / ((fwd_med - poisson_fwd) / 1e3)}
    if ctx.status() != 0:
        raise RuntimeError("device status not ok after the forward-only replays")
    # one direction per call (the unit of the adaptive-rank LRDM / LRDMA steps)
    V1, F1 = V[:1].contiguous(), torch.empty_like(V[:1])
    dmu1 = torch.empty(1, dtype=torch.float64, device="cuda")
    ctx.gateaux([V1], out=[F1], dmu=dmu1)       # captures the K = 1 graph
    torch.cuda.synchronize()
    ev1 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for a0, a1 in ev1:
        a0.record(stream)
        ctx.gateaux([V1], out=[F1], dmu=dmu1)
        a1.record(stream)
    torch.cuda.synchronize()
    k1_med = statistics.median(a0.elapsed_time(a1) for a0, a1 in ev1)
    forward_k1 = {"K": 1, "value": world / (k1_med / 1e3), "unit": "GD/s", "ms_median": k1_med,
                  "graph": True}
    if ctx.status() != 0:
        raise RuntimeError("device status not ok after the one-direction replays")

    return forward_only, forward_k1


def time_e2e(torch, ctx, step, bwd, V, R, fbar, rho_out, coeff, srel, ns, k_local, steps, total_gd, dist):
    """The timed step through the public API with the inputs copied from
    pinned host buffers and the results read back inside the timed region."""
    stream = torch.cuda.current_stream()
    Vh = V.cpu().pin_memory()
    Rh = R.cpu().pin_memory()
    Fbh = fbar.cpu().pin_memory()
    out_h = torch.empty_like(rho_out, device="cpu").pin_memory()
    coef_h = torch.empty(KDIR, dtype=torch.float64).pin_memory()
    srel_h = torch.empty(1, dtype=torch.float64).pin_memory()
    vbar_h = torch.empty((k_local,) + tuple(V.shape[1:]), dtype=V.dtype).pin_memory()
    ebar_h = torch.empty(ns, dtype=torch.float64).pin_memory()
    obar_h = torch.empty(ns, dtype=torch.float64).pin_memory()
    Vd = torch.empty_like(V)
    Rd = torch.empty_like(R)
    Fbd = torch.empty_like(fbar)

    def e2e_step():
        Vd.copy_(Vh, non_blocking=True)
        Rd.copy_(Rh, non_blocking=True)
        Fbd.copy_(Fbh, non_blocking=True)
        step(Vd, Rd, Fbd)
        vbar, eb, ob = bwd()
        out_h.copy_(rho_out, non_blocking=True)
        coef_h.copy_(coeff, non_blocking=True)
        srel_h.copy_(srel, non_blocking=True)
        vbar_h.copy_(vbar[0], non_blocking=True)
        ebar_h.copy_(eb[0], non_blocking=True)
        obar_h.copy_(ob[0], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(steps):
        e2e_step()
    a1.record(stream)
    torch.cuda.synchronize()
    ems = a0.elapsed_time(a1)
    if dist:
        t = torch.tensor([ems], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ems = float(t.item())
    nb = lambda x: x.numel() * x.element_size()
    h2d = nb(Vh) + nb(Rh) + nb(Fbh)
    d2h = nb(out_h) + nb(coef_h) + nb(srel_h) + nb(vbar_h) + nb(ebar_h) + nb(obar_h)
    e2e = {"value": total_gd / (ems / 1e3), "unit": "GD/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}
    if ctx.status() != 0:
        raise RuntimeError("device status not ok after the end-to-end steps")
    return e2e


def main():
    args = parse()
    if args.compare_fp64:
        return compare_fp64(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    # every library call runs on a dedicated stream: the forward call's CUDA
    # graph is captured and replayed only on a stream other than the legacy
    # default one
    torch.cuda.set_stream(torch.cuda.Stream())
    if args.config:
        from paper_2211_07894_gb300 import build as _build
        _build.build()
        return config_leg(args, torch) if rank == 0 else 0
    if args.kpoint_only:
        from paper_2211_07894_gb300 import build as _build
        _build.build()
        kp = time_kpoint(torch, rank, args.prec, autotune=not args.no_autotune)
        if rank == 0 and not args.no_cpu_baseline:
            kp["cpu_baseline"] = time_kpoint_oracle()
        print(json.dumps(kp), flush=True)
        return 0
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2211_07894_gb300 import build as _build
    _build.build()

    directions = args.shard == "directions"
    rows_mode = args.shard == "rows"
    shared = directions or rows_mode
    seed_rank = 0 if shared else rank              # one shared system when it is split
    rows = None
    if rows_mode:
        from paper_2211_07894_gb300 import torch_allreduce
        from paper_2211_07894_gb300.sharding import shard_bounds
        r0, r1 = shard_bounds(args.grid ** 3, world, rank)
        rows = (r0, r1, torch_allreduce() if dist else (lambda t, st: None))
    ctx, V, R, ng = build_problem(torch, seed_rank, args.prec, args.grid, args.ns,
                                  autotune=not args.no_autotune, rows=rows)
    ng_local = rows[1] - rows[0] if rows else ng
    ns = args.ns
    tuning = ctx.tuning() if args.prec in ("bf16x3", "tf32") else None
    F = torch.empty_like(V)
    rho_out = torch.empty_like(R)
    coeff = torch.empty(KDIR, dtype=torch.float64, device="cuda")
    srel = torch.empty(1, dtype=torch.float64, device="cuda")
    dmu = torch.empty(KDIR, dtype=torch.float64, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2211078940 + 70 + seed_rank)
    fbar = torch.randn(V.shape, dtype=V.dtype, device="cuda", generator=gen)
    bwd_out = None
    stream = torch.cuda.current_stream()
    k_lo, k_hi = 0, KDIR                       # the directions this rank evaluates
    if directions:
        from paper_2211_07894_gb300.sharding import shard_bounds, sharded_step
        k_lo, k_hi = shard_bounds(KDIR, world, rank)

    def step(Vs, Rs, Fb):
        nonlocal bwd_out
        if directions:
            # this rank's slice forward, all-gather of f, the K x K step on every rank
            sharded_step(ctx, Vs, Rs, 0.0, rho=rho_out, coeff=coeff, s_rel=srel)
            bwd_out = ctx.backward([Fb[k_lo:k_hi]], out=bwd_out)
            return
        ctx.gateaux([Vs], out=[F], dmu=dmu)
        ctx.apply(0, Rs, Vs, F, 0.0, rho=rho_out, coeff=coeff, s_rel=srel)
        bwd_out = ctx.backward([Fb], out=bwd_out)

    for _ in range(max(args.warmup, 0)):
        step(V, R, fbar)
    torch.cuda.synchronize()
    if ctx.status() != 0:
        raise RuntimeError("device status not ok after warm-up")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(V, R, fbar)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    steps = max(args.steps, 1)
    ms_step = ms / steps
    total_gd = KDIR * steps * (1 if shared else world)
    value = total_gd / (ms / 1e3)
    if ctx.status() != 0:
        raise RuntimeError("device status not ok after the timed region")
    forward_only = forward_k1 = None
    apply_ms = None
    if not shared:
        forward_only, forward_k1 = time_forward_calls(torch, ctx, V, F, dmu, prof, args, world)
        # the least-squares step alone (Gram, K x K solve, update) on the step's own derivatives
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        rho_tmp = rho_out.clone()
        a0.record(stream)
        for _ in range(10):
            ctx.apply(0, R, V, F, 0.0, rho=rho_tmp, coeff=coeff, s_rel=srel)
        a1.record(stream)
        torch.cuda.synchronize()
        apply_ms = a0.elapsed_time(a1) / 10
        del rho_tmp

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = time_e2e(torch, ctx, step, lambda: bwd_out, V, R, fbar, rho_out, coeff, srel, ns,
                       k_hi - k_lo, steps, total_gd, dist)

    # roofline of the dominant contraction
    peaks, peak_src = load_peaks()
    g1 = (prof["gemm1_ms"], prof["gemm1_launches"])
    g2 = (prof["gemm2_ms"], prof["gemm2_launches"])
    name, (tms, nl) = max((("projection GEMM (X_k)", g1), ("response GEMM (drho_k)", g2)),
                          key=lambda x: x[1][0])
    g1_kernel = "k_gemm1_pair" if tuning and tuning["g1_nb"] == 512 else "k_gemm1_tc"
    g2_kernel = "k_gemm2_pair" if tuning and tuning["g2_bn"] == 512 else "k_gemm2_tc"
    kname = g1_kernel if name.startswith("projection") else g2_kernel
    kshape = ((f"g1_nb={tuning['g1_nb']},g1_dpt={tuning['g1_dpt']}" if kname == g1_kernel
               else f"g2_bn={tuning['g2_bn']},g2_kgroup={tuning['g2_kgroup']}") if tuning else None)
    avg_s = tms / max(nl, 1) / 1e3
    alg_flops = (k_hi - k_lo) * ng_local * ns * ns   # one launch: this rank's directions and rows, symmetric half
    peak, bound, issue, note = dtype_peak(args.prec, peaks)
    issued = issue * alg_flops
    achieved = issued / avg_s / 1e12 if avg_s > 0 else None
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None,
                "traffic": recorded_traffic(kname, f"{args.grid}^3/{ns}/K{KDIR}/{args.prec}", kshape),
                "kernel": name, "avg_launch_ms": avg_s * 1e3, "launches": nl,
                "alg_flop_per_launch": alg_flops, "peak_source": f"{peak_src}; {note}"}

    # tensor-pipe use of both contractions: the issued rate against the
    # measured peak (live) and ncu's pipe-active share (recorded full-size capture)
    tensor_pipe = None
    if args.prec in ("bf16x3", "tf32"):
        tensor_pipe = {"source": "rate_frac: issued MMA rate / peak (as roofline), live; ncu_pct_of_elapsed: "
                                 "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_elapsed "
                                 "from a one-pass capture under profiles/ of this workload, else of the "
                                 "48^3 / N_s = 1024 small case (ncu_workload says which; null when no "
                                 "record matches the current sources and shape)"}
        for key, kn, (ms, n) in (("projection", g1_kernel, g1), ("response", g2_kernel, g2)):
            sh = ((f"g1_nb={tuning['g1_nb']},g1_dpt={tuning['g1_dpt']}" if kn == g1_kernel
                   else f"g2_bn={tuning['g2_bn']},g2_kgroup={tuning['g2_kgroup']}") if tuning else None)
            sec = ms / max(n, 1) / 1e3
            pct, wl = None, None
            for w in (f"{args.grid}^3/{ns}/K{KDIR}/{args.prec}", f"48^3/1024/K{KDIR}/{args.prec}"):
                pct = recorded_tensor_pipe(kn, w, sh)
                if pct is not None:
                    wl = w
                    break
            tensor_pipe[key] = {"rate_frac": issued / sec / 1e12 / peak if sec > 0 else None,
                                "ncu_pct_of_elapsed": pct, "ncu_workload": wl}

    # the uneven batch with its spin pair: 64 derivatives per call (one
    # grouped launch per contraction, graph replay), same precision
    batched = None
    if not args.no_batched and not shared and args.prec in ("bf16x3", "tf32", "fp32"):
        ctx.close()
        F = fbar = bwd_out = None
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        cfgs3 = config_inputs(3)
        gen_s = time.perf_counter() - t0
        batched = gpu_config_run(torch, cfgs3, args.prec, None, load_peaks()[0],
                                 autotune=not args.no_autotune)
        batched.update({"workload": CONFIG_LEGS[3][0], "derivatives_per_call": 64,
                        "value": batched["gd_s"] * world, "host_generation_s": gen_s})
        del cfgs3

    kpoint = None
    if not args.no_kpoint and not shared:
        ctx.close()
        F = fbar = bwd_out = None
        torch.cuda.empty_cache()
        kpoint = time_kpoint(torch, rank, args.prec, autotune=not args.no_autotune)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            kpoint["cpu_baseline"] = time_kpoint_oracle()

    fp64_plain = None
    if not args.no_fp64_plain and not shared:
        ctx.close()
        F = fbar = bwd_out = None
        torch.cuda.empty_cache()
        res, sample = time_fp64_plain(torch)
        gds, sec = res["plain-fp64-gpu"]
        fp64_plain = {"value": gds * world, "unit": "GD/s", "seconds_per_direction": sec,
                      "sample": sample,
                      "speedup_forward_only": forward_only["value"] / (gds * world),
                      "speedup_step": value / (gds * world)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gds, dt, sample = time_oracle(1, 0)
        cpu = {"value": gds, "unit": "GD/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": sample, "cpu_model": cpu_model(), "one_thread": time_oracle_one_thread()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GD/s", "n_gpus": world,
                "steps": steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "strong" if shared else "weak",
                "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
                "config": {"workload": f"{args.grid}^3 grid, N_s={ns}, K={KDIR}, FP32 Psi, "
                                       f"{args.prec} contractions",
                           "grid": [args.grid] * 3, "n_s": ns, "K": KDIR,
                           "precision": args.prec,
                           "l2": "inputs larger than L2 (Psi operand copies > 14 GB)",
                           "parallelism": f"{args.shard} x{world}"},
                "roofline": roofline, "tensor_pipe": tensor_pipe, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clocks,
                "gpu_launches": prof["kernel_launches"],
                "forward_only": forward_only, "forward_k1": forward_k1, "fp64_plain": fp64_plain,
                "kpoint": kpoint, "batched_uneven": batched,
                "paper_context": PAPER_CONTEXT,
                "launch_shape": tuning,
                "breakdown_ms": {"gemm1_per_step": prof["gemm1_ms"] / steps,
                                 "gemm2_per_step": prof["gemm2_ms"] / steps,
                                 "poisson_per_step": prof["poisson_ms"] / steps,
                                 "apply_per_call": apply_ms,
                                 "gemm1_launches_per_step": prof["gemm1_launches"] / steps,
                                 "gemm2_launches_per_step": prof["gemm2_launches"] / steps}}
        print(json.dumps(line), flush=True)
        if args.jsonl:
            append_jsonl(args.jsonl, line)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
