#!/usr/bin/env python3
"""Benchmark of the SFHK high-harmonic path on B300.

One step = the whole hot path over one batch: for the H2 workload at
molecular-axis angles 0/45/90 degrees (1e6 trajectories each; 800 nm,
3 cycles of sin^2, 1.5e14 W/cm^2, dt = 0.05, gamma = 0.5, prefactor filter
|C| > 1e4):
  device sampling of the initial ensemble (ionization step) for each angle,
  one persistent propagation launch over the three ensembles (trajectories,
  stability matrices, action, prefactor, fused dipole reduction),
  and the windowed Fourier transform of each dipole (three spectra).
The headline form is the mixed-precision path; the plain FP64 GPU path is
timed on the same workload for comparison, with the relative L2 difference
of their dipoles.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one rank per GPU, each rank on its own seeds
(weak scaling, no data-path collective).  `--impl reference` times the FP64
CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2608_13686_b300 import costs  # noqa: E402
from paper_2608_13686_b300 import workloads as W  # noqa: E402

METRIC = W.METRIC if hasattr(W, "METRIC") else (
    "trajectory-steps/sec and HHG spectra/sec at stated dipole error; p50/p99 latency")
UNIT = "trajectory-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-traj", type=int, default=W.H2_ANGLES["n_traj"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--block", type=int, default=0, help="pin the integrator's block size")
    ap.add_argument("--kernel-variant", type=int, default=0, help="pin the register-cap variant")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ CPU oracle
def oracle_sample_run(n_per_angle, angles, seed_base=0):
    """The oracle over the first n_per_angle trajectories of each angle:
    sampling, propagation and spectrum.  Returns (seconds, traj_steps)."""
    import oracle as O
    t, p = W.TARGETS["H2"], W.PULSE_800
    d = O.pulse_derived(p)
    t0 = time.perf_counter()
    steps = 0
    for k, ang in enumerate(angles):
        soa, _, _ = O.sample(t, p, W.fixed(ang), seed=seed_base, instance=k, n=n_per_angle)
        vz, fin, _ = O.propagate(t, p, soa, W.GAMMA, cutoff=W.CUTOFF, want_final=False,
                                 stab_cutoff=W.STAB_CUTOFF)
        O.spectrum(vz, d["dt"], d["t_origin"], 0.5 * d["Tp"], d["nt"] // 2)
        steps += int(np.sum(d["nt"] - 1 - soa[0]))
    return time.perf_counter() - t0, steps


def cpu_baseline(target_s, angles):
    import oracle as O
    O.build()
    n = 64
    sec, st = oracle_sample_run(n, angles)
    n = int(max(64, min(200000, n * target_s / max(sec, 1e-3))))
    sec, st = oracle_sample_run(n, angles)
    cores = os.cpu_count()
    return {"value": st / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"H2 workload, first {n} trajectories of each of {len(angles)} angles "
                      f"(sampling + FP64 RK4 propagation + dipole + DFT), {sec:.1f} s, "
                      f"OpenMP over {cores} host threads",
            "seconds": sec, "traj_steps": st}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    angles = W.H2_ANGLES["angles"]
    import oracle as O
    O.build()
    n = 64
    sec, _ = oracle_sample_run(n, angles)
    # each step a bounded sample sized so the whole run stays within minutes
    per_step_s = min(20.0, 150.0 / max(1, args.steps + args.warmup))
    n = int(max(32, min(100000, n * per_step_s / max(sec, 1e-3))))
    for _ in range(args.warmup):
        oracle_sample_run(n, angles)
    times, steps = [], 0
    for _ in range(args.steps):
        s, st = oracle_sample_run(n, angles)
        times.append(s)
        steps += st
    total = sum(times)
    value = steps / total
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W.H2_ANGLES["name"], "sample_per_angle": n,
                       "parallelism": "none (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {n} trajectories of each angle per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU path
def run_ours(args):
    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2608_13686_b300 import _build
    _build.build()
    from paper_2608_13686_b300 import sfhk as S

    cfg = W.H2_ANGLES
    angles = cfg["angles"]
    n = args.n_traj
    ctx = S.sfhk_create(local, 0)
    tgt = S.sfhk_create_target(ctx, W.TARGETS[cfg["target"]])
    pul = S.sfhk_set_pulse(ctx, cfg["pulse"])
    grid = S.sfhk_pulse_grid(pul)
    nt, dt, t_or, tau = grid["nt"], grid["dt"], grid["t_origin"], 0.5 * grid["Tp"]
    n_out = nt // 2
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    seed = cfg["seed"] + 1000 * rank
    ens = [S.sfhk_sample_initial(ctx, tgt, pul, W.fixed(a), n, seed, k, sp)
           for k, a in enumerate(angles)]
    spec = [torch.empty((3, n_out), dtype=torch.float64, device="cuda") for _ in angles]

    def step(opts, k_step):
        for k, a in enumerate(angles):
            S.sfhk_sample_into(ctx, ens[k], W.fixed(a), seed, k, sp)
        S.sfhk_propagate_batch(ctx, ens, opts, sp)
        for k in range(len(angles)):
            vz_ptr, _ = S.sfhk_dipole_device(ens[k])
            o = spec[k]
            S.sfhk_spectrum_device(vz_ptr, nt, dt, t_or, tau, o[0].data_ptr(), o[1].data_ptr(),
                                   o[2].data_ptr(), n_out, sp)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    mixed = S.run_opts(S.SFHK_MIXED, cfg["gamma"], W.CUTOFF, stab_cutoff=W.STAB_CUTOFF,
                       block_threads=args.block, kernel_variant=args.kernel_variant)
    # launch shape (block size x register-cap variant) chosen by the autotuner
    # on the first angle's ensemble, untimed
    tuned = None
    if not args.no_tune and not (args.block and args.kernel_variant):
        tuned = S.sfhk_autotune(ctx, ens[0], mixed, max_items=8192)
    for w in range(args.warmup):
        step(mixed, w)
    barrier()
    clock = ClockSampler(local)
    clock.start()
    l0 = S.sfhk_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    prop_ms = []
    barrier()
    ev[0].record(stream)
    for k in range(args.steps):
        step(mixed, k)
        ev[k + 1].record(stream)
    barrier()
    launches = (S.sfhk_launch_count() - l0)
    clk = clock.stop()
    ms_steps = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    st = [S.sfhk_stats_get(e) for e in ens]
    traj_steps = sum(s["traj_steps"] for s in st)       # per step (deterministic)
    prop_ms = st[0]["kernel_ms"]                        # the batch launch of the last step
    ms = float(np.mean(ms_steps))
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * traj_steps / (ms * 1e-3)
    spectra_per_s = world * len(angles) / (ms * 1e-3)
    vz_mixed = [S.sfhk_dipole(ctx, e, nt) for e in ens]

    # roofline of the propagation kernel (FP32 FMA pipe)
    flops = costs.FLOPS_PER_STEP[cfg["target"]] * traj_steps
    achieved = flops / (prop_ms * 1e-3) / 1e12
    peak = costs.fp32_peak_tflops()
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "k_propagate<mixed>", "kernel_ms": prop_ms,
            "flops_per_traj_step": costs.FLOPS_PER_STEP[cfg["target"]],
            "peak_basis": "148 SM x 128 FP32 lanes x 2 x 2032 MHz (unit counts, max clock)"}
    if clk.get("sm_mhz"):
        roof["peak_at_median_clock"] = costs.fp32_peak_tflops(clk["sm_mhz"])

    # e2e through the public API with host buffers (dipole and spectrum to host)
    def e2e_step():
        for k, a in enumerate(angles):
            S.sfhk_sample_into(ctx, ens[k], W.fixed(a), seed, k, sp)
        S.sfhk_propagate_batch(ctx, ens, mixed, sp)
        for k in range(len(angles)):
            vz = S.sfhk_dipole(ctx, ens[k], nt)
            S.sfhk_spectrum(vz, dt, t_or, tau, n_out)

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = len(angles) * (nt * 8 + 24) + 48
    d2h = len(angles) * (nt * 8 + 3 * n_out * 8)
    e2e = {"value": world * traj_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3}

    # the plain FP64 GPU path on the same workload, and the dipole difference
    fp64 = None
    if not args.no_fp64:
        o64 = S.run_opts(S.SFHK_FP64, cfg["gamma"], W.CUTOFF, stab_cutoff=W.STAB_CUTOFF)
        step(o64, 0)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(o64, 1)
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1)
        st64 = [S.sfhk_stats_get(e) for e in ens]
        ts64 = sum(s["traj_steps"] for s in st64)
        vz64 = [S.sfhk_dipole(ctx, e, nt) for e in ens]
        errs = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(vz_mixed, vz64)]
        fp64 = {"value": world * ts64 / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "kernel_ms": st64[0]["kernel_ms"], "steps": 1, "warmup": 1,
                "dipole_rel_l2_mixed_vs_fp64": errs,
                "speedup_mixed_over_fp64": (traj_steps / ms) / (ts64 / ms64)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds, angles)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64 (mixed: f32 state, two-float action/phase, f64 reduction)",
                "data": "synthetic",
                "config": {"workload": cfg["name"], "target": cfg["target"],
                           "angles_deg": list(angles), "n_traj_per_angle": n,
                           "nt": nt, "dt": dt, "gamma": cfg["gamma"],
                           "prefactor_cutoff": W.CUTOFF, "stability_cutoff": W.STAB_CUTOFF,
                           "traj_steps_per_step": traj_steps,
                           "l2": "inputs larger than L2 (trajectory SoA 3 x 96 MB)",
                           "parallelism": f"replicas x{world}"},
                "spectra_per_s": spectra_per_s,
                "ms_per_step_all": ms_steps,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "fp64_path": fp64, "gpu_launches": launches // args.steps,
                "autotuned": tuned,
                "clocks": clk,
                "filtered_frac": sum(s["n_filtered"] + s["n_unstable"] for s in st)
                / (len(angles) * n)}
        print(json.dumps(line), flush=True)
    for e in ens:
        S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(pul)
    S.sfhk_destroy_target(tgt)
    S.sfhk_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
