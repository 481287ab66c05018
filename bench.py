#!/usr/bin/env python
"""Benchmark of the LRDM Gateaux-derivative hot path on GB300.

Metric: Gateaux derivatives per second at a 96^3 grid (884,736 points),
N_s = 4096, K = 16 directions (one derivative = one (system, direction) f_k).
One step = one pass of the whole path over one batch of K directions:
Hartree + LDA kernel, projection GEMM, mu' and Loewner scaling, response GEMM
with the f = drho - v epilogue (lrdm_gateaux_batch), then the K x K
least-squares step and update (lrdm_apply).

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

METRIC = "Gateaux derivatives/sec at 96^3 grid, N_s=4096, K=16"
GRID = (96, 96, 96)
H = (0.5, 0.5, 0.5)
NS = 4096
KDIR = 16
NE = 3700.0
KT = 0.005
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
    p.add_argument("--grid", type=int, default=96, help="grid edge (96 = the benchmark workload)")
    p.add_argument("--ns", type=int, default=NS)
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
    sample = (f"oracle.gateaux + lrdm_apply, K=1, N_s={NS}, grid {ORACLE_SAMPLE_GRID[0]}^3 "
              f"(1/{int(scale)} of the 96^3 rows), {steps} step(s); GD/s scaled by the row ratio")
    return gds, dt, sample


def reference_arm(args, rank, world):
    if rank != 0:
        return 0
    steps = max(1, args.steps)
    gds, dt, sample = time_oracle(steps, max(0, min(args.warmup, 1)))
    line = {"impl": "reference", "metric": METRIC, "value": gds, "unit": "GD/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"96^3 grid, N_s={NS}, K={KDIR} (oracle on a bounded sample)",
                       "grid": list(GRID), "n_s": NS, "K": KDIR},
            "cpu_baseline": {"value": gds, "unit": "GD/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gds, "unit": "GD/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def build_problem(torch, rank, prec, edge, ns):
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
    ctx = Context([system], prec=prec, io_dtype=io, k_max=KDIR)
    del psi, system
    torch.cuda.empty_cache()
    return ctx, V, R, ng


def compare_fp64(args):
    """The plain FP64 GPU form: per direction, X = Psi^T (a o Psi) and
    drho = rowsum((Psi X') o Psi) with dense torch FP64 matmuls (Psi X'
    materialised), next to this library's FP64 path, both for one direction on
    a 48^3 grid with N_s = 4096 (1/8 of the 96^3 rows; both forms are linear in
    the rows, so GD/s at 96^3 = 1 / (8 t)).  The two dense products are > 99 %
    of the plain form's work; its element-wise steps are not timed."""
    import numpy as np
    import torch
    import workloads
    from paper_2211_07894_gb300 import Context
    torch.cuda.set_device(0)
    n = (48, 48, 48)
    ng = int(np.prod(n))
    scale = float(np.prod(GRID)) / ng
    psi32 = workloads.random_subspace_torch(n, H, NS, seed=2211078940 + 60, device="cuda")
    psi = psi32.double()
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    a = torch.randn(ng, dtype=torch.float64, device="cuda", generator=g)
    Xp = torch.randn(NS, NS, dtype=torch.float64, device="cuda", generator=g)
    Xp = Xp + Xp.T

    def plain():
        X = psi.T @ (a[:, None] * psi)
        d = ((psi @ Xp) * psi).sum(dim=1)
        return X, d

    def timed(fn, reps=2):
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

    t_plain = timed(plain)
    eps = torch.as_tensor(workloads.random_eigenvalues(NS, workloads.rng_for(5, 60)), device="cuda")
    V = torch.as_tensor(workloads.smooth_directions(n, H, 1, 1, workloads.rng_for(5, 61)),
                        dtype=torch.float64, device="cuda")
    ctx = Context([dict(n=n, h=H, psi=[psi], eps=[eps], n_electrons=NE, kT=KT, g=2.0,
                        rho_floor=1e-3, k_max=1)], prec="fp64", io_dtype=torch.float64, k_max=1)
    F = torch.empty_like(V)
    t_ours = timed(lambda: ctx.gateaux([V], out=[F]))
    for impl, t in (("plain-fp64-gpu", t_plain), ("library-fp64", t_ours)):
        print(json.dumps({"impl": impl, "metric": METRIC, "value": 1.0 / (t * scale),
                          "unit": "GD/s", "dtype": "f64",
                          "sample": "1 direction, 48^3 grid, N_s=4096; GD/s scaled by the 8x row ratio",
                          "seconds_per_direction_at_96^3": t * scale}), flush=True)
    return 0


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
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2211_07894_gb300 import build as _build
    _build.build()

    ctx, V, R, ng = build_problem(torch, rank, args.prec, args.grid, args.ns)
    ns = args.ns
    F = torch.empty_like(V)
    rho_out = torch.empty_like(R)
    coeff = torch.empty(KDIR, dtype=torch.float64, device="cuda")
    srel = torch.empty(1, dtype=torch.float64, device="cuda")
    dmu = torch.empty(KDIR, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        ctx.gateaux([V], out=[F], dmu=dmu)
        ctx.apply(0, R, V, F, 0.0, rho=rho_out, coeff=coeff, s_rel=srel)

    for _ in range(max(args.warmup, 0)):
        step()
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
        step()
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
    total_gd = KDIR * steps * world
    value = total_gd / (ms / 1e3)
    if ctx.status() != 0:
        raise RuntimeError("device status not ok after the timed region")

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Vh = V.cpu().pin_memory()
        Rh = R.cpu().pin_memory()
        out_h = torch.empty_like(rho_out, device="cpu").pin_memory()
        coef_h = torch.empty(KDIR, dtype=torch.float64).pin_memory()
        srel_h = torch.empty(1, dtype=torch.float64).pin_memory()
        Vd = torch.empty_like(V)
        Rd = torch.empty_like(R)

        def e2e_step():
            Vd.copy_(Vh, non_blocking=True)
            Rd.copy_(Rh, non_blocking=True)
            ctx.gateaux([Vd], out=[F], dmu=dmu)
            ctx.apply(0, Rd, Vd, F, 0.0, rho=rho_out, coeff=coeff, s_rel=srel)
            out_h.copy_(rho_out, non_blocking=True)
            coef_h.copy_(coeff, non_blocking=True)
            srel_h.copy_(srel, non_blocking=True)

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
        h2d = Vh.numel() * Vh.element_size() + Rh.numel() * Rh.element_size()
        d2h = (out_h.numel() * out_h.element_size() + coef_h.numel() * 8 + 8)
        e2e = {"value": total_gd / (ems / 1e3), "unit": "GD/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # roofline of the dominant contraction
    peaks, peak_src = load_peaks()
    g1 = (prof["gemm1_ms"], prof["gemm1_launches"])
    g2 = (prof["gemm2_ms"], prof["gemm2_launches"])
    name, (tms, nl) = max((("projection GEMM (X_k)", g1), ("response GEMM (drho_k)", g2)),
                          key=lambda x: x[1][0])
    avg_s = tms / max(nl, 1) / 1e3
    alg_flops = KDIR * ng * ns * ns           # one launch: K directions, symmetric half
    if args.prec == "bf16x3":
        issued = 3.0 * alg_flops
        peak = peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
        bound, note = "tensor", "bf16x3 issues 3 bf16 MMAs per product; achieved = issued bf16 rate"
    elif args.prec == "tf32":
        issued = alg_flops
        peak = 0.5 * peaks.get("bf16_tflops_sustained", FALLBACK_PEAKS["bf16_tflops_sustained"])
        bound, note = "tensor", "tf32 peak = bf16 sustained x 1/2 (nominal ratio)"
    elif args.prec == "fp32":
        issued = alg_flops
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        bound, note = "alu", "FP32 FMA peak = 152 SMs x 128 lanes x 2 x 2.07 GHz"
    else:
        issued = alg_flops
        peak = 1.10
        bound, note = "alu", "FP64 peak = measured torch FP64 matmul (1.10 TF/s)"
    achieved = issued / avg_s / 1e12 if avg_s > 0 else None
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": None,
                "kernel": name, "avg_launch_ms": avg_s * 1e3, "launches": nl,
                "alg_flop_per_launch": alg_flops, "peak_source": f"{peak_src}; {note}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gds, dt, sample = time_oracle(1, 0)
        cpu = {"value": gds, "unit": "GD/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GD/s", "n_gpus": world,
                "steps": steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.prec, "data": "synthetic",
                "config": {"workload": f"{args.grid}^3 grid, N_s={ns}, K={KDIR}, FP32 Psi, "
                                       f"{args.prec} contractions",
                           "grid": [args.grid] * 3, "n_s": ns, "K": KDIR,
                           "precision": args.prec,
                           "l2": "inputs larger than L2 (Psi operand copies > 14 GB)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": prof["kernel_launches"],
                "breakdown_ms": {"gemm1_per_step": prof["gemm1_ms"] / steps,
                                 "gemm2_per_step": prof["gemm2_ms"] / steps}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
