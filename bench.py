#!/usr/bin/env python
"""Benchmark of the CF-DQMC sweep: autocorrelation-corrected effective
samples per second on the N_phi = 36 torus.

Workload (one step = one sweep of every chain): torus N_phi = 36 (N = 72
single-particle states per spin block, N_q = 333 momenta, 1332 real fields
per slice), beta = 36, dtau = 0.1 (L = 360 slices), eight chains at couplings
u = linspace(0.5, 2.0, 8), seeds 0..7, restabilisation every 10 slices.
Default path: mixed precision (FP32 eigensolver bulk and drift transforms,
FP64 propagators, ratios and updates) with learned-proposal sweeps and a
Langevin sweep every 4th step; --mode plain --precision 0 is the plain FP64
Langevin sweep.

value = sum over chains of K / (2 tau_int) divided by the device time of the
K timed sweeps, tau_int = max over {m^2, E} of Sokal's windowed estimate on
the chain's recorded series.

Multi-GPU: one process per GPU, each running its own eight chains (seeds
offset by 8 * rank): independent replicas, weak scaling, no collective on the
data path.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (no GPU work).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NPHI, BETA, DTAU, NCH, NSTAB = 36, 36.0, 0.1, 8, 10
COUPLINGS = np.linspace(0.5, 2.0, NCH)
EPS0 = 0.45
METRIC = "effective samples/s (autocorr-corrected) at N_phi=36 torus vs plain FP64 sweep"
UNIT = "effective samples/s"
# FP64 pipe peak of a GB300: 1.25 TFLOP/s nominal = 152 SMs x 2 DFMA/clk x
# 2 flop x 2.07 GHz (derivation and measurement in the design notes)
FP64_PEAK_TFLOPS = 1.25
# dram bytes (read + write) of one FP64 GEMM launch from the ncu capture
# summarised in profiles/k_zgemm_fp64_n36_full.md (n = 36, batch 32; the
# N = 72 batch-8 products move the same 2 MB of operands)
TRAFFIC_PER_LAUNCH = 1338624
# oracle sample: one sweep of an L_SAMPLE-slice chain at the same N_phi, one
# process per chain, scaled to L = 360
L_SAMPLE = 10
# learned mode: one Langevin sweep per LANGEVIN_EVERY steps
LANGEVIN_EVERY = 4


def workload_config(extra=None):
    cfg = {
        "workload": f"CF-DQMC sweep, torus N_phi=36 (N=72, N_q=333), beta={BETA:g}, dtau=0.1 "
                    f"(L={int(round(BETA / DTAU))}), 8 chains u=linspace(0.5,2,8) seeds 0-7 "
                    "(+8*rank), n_stab=10",
        "n_chains_per_gpu": NCH,
        "L": int(round(BETA / DTAU)),
        "l2": "inputs larger than L2: 8 chains x 360 slices x (B, B^-1) = 478 MB resident",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks --
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------- replicas -----
def replica_seeds(rank):
    """Seeds of rank `rank`'s chains: disjoint across ranks, so the ranks are
    independent replicas of the eight-chain workload."""
    return np.arange(NCH) + NCH * rank


def combine_over_ranks(dist, t_s, wall, ess, device):
    """Whole-job figures: the slowest rank's timed seconds and end-to-end wall
    clock (max over ranks) and the effective samples of all ranks (sum)."""
    if dist is None:
        return t_s, wall, ess
    import torch
    tt = torch.tensor([t_s, wall], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    es = torch.tensor([ess], device=device, dtype=torch.float64)
    dist.all_reduce(es)
    return float(tt[0]), float(tt[1]), float(es[0])


# ------------------------------------------------------------- tau / ESS ---
def tau_per_chain(series, tau_fn):
    """max over m^2 (col 0) and E (col 12) of the windowed tau_int"""
    return [max(tau_fn(series[c, :, 0]), tau_fn(series[c, :, 12])) for c in range(series.shape[0])]


# ------------------------------------------------------------ CPU oracle ---
def _oracle_sample(u, seed):
    """Time one sweep of an L_SAMPLE-slice oracle chain at N_phi = 36 and one
    measurement; return seconds per slice update and per measurement."""
    from oracle import model as M
    from oracle import oracle as O
    m = M.Model(M.TORUS, NPHI)
    ch = O.Chain(M.TORUS, NPHI, L_SAMPLE * DTAU, DTAU, u, 0.0, seed, n_stab=NSTAB, eps0=EPS0, model=m)
    t0 = time.perf_counter()
    ch.measure()
    t_meas = time.perf_counter() - t0
    t0 = time.perf_counter()
    ch.sweep(1)
    t_sw = time.perf_counter() - t0
    return (t_sw - t_meas) / L_SAMPLE, t_meas, t_sw


def oracle_sweeps_per_s(nproc=NCH):
    """Aggregate oracle chain-sweeps/s at L = 360 over nproc parallel chains
    (one process, one thread each), from a bounded sample."""
    from oracle import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(nproc) as pool:
        res = pool.starmap(_oracle_sample, [(float(COUPLINGS[c % NCH]), c) for c in range(nproc)])
    wall = time.perf_counter() - t0
    L = int(round(BETA / DTAU))
    t_full = [L * r[0] + r[1] for r in res]   # seconds per L=360 sweep per chain
    return sum(1.0 / t for t in t_full), t_full, wall, res


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, bounded
    sample per step (one L_SAMPLE-slice sweep of each of the eight chains in
    parallel processes), reported as effective samples/s at L = 360 with
    tau_int = 1/2 (the oracle's own tau cannot be measured in minutes: an
    upper bound of its rate)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    L = int(round(BETA / DTAU))
    step_rates = []
    with ctx.Pool(NCH) as pool:
        for k in range(args.warmup + args.steps):
            res = pool.starmap(_oracle_sample, [(float(COUPLINGS[c]), c) for c in range(NCH)])
            if k >= args.warmup:
                step_rates.append(sum(1.0 / (L * r[0] + r[1]) for r in res))
    sweeps_per_s = float(np.mean(step_rates))
    value = sweeps_per_s / (2 * 0.5)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * NCH / sweeps_per_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (fields drawn from the chains' own Philox streams)",
        "config": workload_config({"sample": f"one L={L_SAMPLE} sweep per chain per step, "
                                             f"scaled to L={L}; tau_int taken as 1/2"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": NCH, "kind": "oracle",
                         "sample": f"per step: one sweep of an L={L_SAMPLE} N_phi=36 oracle chain "
                                   f"per coupling, {NCH} processes x 1 thread, scaled to L={L}, "
                                   "tau_int=1/2 upper bound"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ours ------
def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle pool is spawned before the first GPU call
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, t_full, wall, _ = oracle_sweeps_per_s()
        cpu = {"sweeps_per_s": rate, "t_full": t_full, "wall": wall}
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2605_03700_gb300 import build as B
    B.build()
    import paper_2605_03700_gb300 as P

    stream = torch.cuda.Stream()
    wall0 = time.perf_counter()
    seeds = replica_seeds(rank)
    ch = P.Chain(P.QMC_TORUS, NPHI, BETA, DTAU, 0.0, 0.0, 0, n_chains=NCH, couplings=COUPLINGS,
                 seeds=seeds, n_stab=NSTAB, eps0=EPS0, series_capacity=4096,
                 precision=args.precision,
                 drift=P.QMC_DRIFT_FIRST if args.drift == "first" else P.QMC_DRIFT_EXACT)
    ch.set_stream(stream.cuda_stream)
    # learned mode: whole-slice moves around the network's Gaussian
    # (qmc_sweep_learned, rho = 0), a Langevin sweep every LANGEVIN_EVERY-th
    # step as the fallback; the network is at its prior initialisation
    # (mu = 0, sigma = 1), which held-out NLL early stopping keeps at this
    # workload (training does not improve it; see the design notes)
    net = P.Net(4 * ch.n_q, 256, 16, 1 + rank) if args.mode == "learned" else None

    def step(k):
        if net is None or k % LANGEVIN_EVERY == LANGEVIN_EVERY - 1:
            ch.sweep(1)
        else:
            ch.sweep_learned(net, 1, 0.0)

    pinned = torch.empty((args.steps, NCH, P.QMC_NOBS), dtype=torch.float64, pin_memory=True)
    for k in range(args.warmup):
        step(k)
    ch.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    launches0 = P.qmc_launch_count()
    P.qmc_profile_gemm(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
        ch.copy_latest_async(pinned[k].data_ptr())
    e1.record(stream)
    ch.sync()
    gemm_ms, gemm_n, gemm_flops = P.qmc_profile_gemm(False)
    launches = P.qmc_launch_count() - launches0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    series = ch.series()[:, args.warmup:, :]
    wall_e2e = time.perf_counter() - wall0
    taus = tau_per_chain(series, P.qmc_tau_int)
    learned_steps = [k for k in range(args.steps)
                     if net is not None and (args.warmup + k) % LANGEVIN_EVERY != LANGEVIN_EVERY - 1]
    acc_learned = float(series[:, learned_steps, 13].mean()) if learned_steps else None
    acc_langevin = float(np.delete(series[:, :, 13], learned_steps, axis=1).mean())
    ess = sum(args.steps / (2.0 * t) for t in taus)
    t_s = ms / 1000.0
    t_s, wall_e2e, ess = combine_over_ranks(dist, t_s, wall_e2e, ess, "cuda")
    value = ess / t_s
    e2e = ess / wall_e2e
    # roofline of the GEMM class (event-timed over the timed region)
    gemm_tflops = gemm_flops / (gemm_ms / 1000.0) / 1e12 if gemm_ms > 0 else 0.0
    roof = {"bound": "alu", "achieved": gemm_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": gemm_tflops / FP64_PEAK_TFLOPS,
            "traffic": TRAFFIC_PER_LAUNCH, "kernel": "k_zgemm<double> (batched complex FP64 GEMM; FP32 products excluded)",
            "launches": gemm_n, "ms_total": gemm_ms, "share_of_step_time": gemm_ms / ms,
            "peak_note": "nominal FP64 pipe rate (no measured FP64 peak exists for this part): "
                         "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26 TFLOP/s"}
    if rank != 0:
        ch.close()
        if dist:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f32+f64",
        "data": "synthetic (fields drawn from the chains' own Philox streams)",
        "config": workload_config({"parallelism": f"replicas x{world}",
                                   "precision": ["fp64", "mixed fp32/fp64"][args.precision],
                                   "mode": args.mode,
                                   "drift": args.drift,
                                   "schedule": ("plain Langevin sweeps" if args.mode == "plain" else
                                                f"learned sweeps (rho 0), every {LANGEVIN_EVERY}th "
                                                "step a Langevin sweep"),
                                   "acceptance_learned": acc_learned,
                                   "acceptance_langevin": acc_langevin,
                                   "tau_int": [round(t, 3) for t in taus],
                                   "tau_series_len": int(series.shape[1]),
                                   "sweeps_per_s_per_gpu": NCH * args.steps / t_s / world}),
        "roofline": roof,
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": NCH * P.QMC_NOBS * 8,
                "note": "wall clock through the C ABI from qmc_create to the last D2H of the "
                        "records, warm-up included; a sweep takes no host input"},
    }
    if cpu:
        ess_cpu = sum(1.0 / tf / (2.0 * t) for tf, t in zip(cpu["t_full"], taus))
        line["cpu_baseline"] = {
            "value": ess_cpu, "unit": UNIT, "cores": NCH, "kind": "oracle",
            "sample": f"one sweep of an L={L_SAMPLE} N_phi=36 oracle chain per coupling "
                      f"({NCH} processes x 1 thread), scaled to L=360; tau_int of the GPU "
                      f"chains (decision-identical Markov chains)",
            "sweeps_per_s": cpu["sweeps_per_s"]}
    print(json.dumps(line))
    ch.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="0: FP64 everywhere; 1: mixed (FP32 eigensolver + FP64 polish, FP32 "
                         "gradient transforms and wraps, FP64 propagators, ratios, updates)")
    ap.add_argument("--mode", default="learned", choices=["learned", "plain"],
                    help="learned: learned-proposal sweeps with a Langevin sweep every "
                         "4th step; plain: Langevin sweeps only")
    ap.add_argument("--drift", default="exact", choices=["exact", "first"],
                    help="Langevin drift: exact grad S, or the first-order drift (factors "
                         "treated as commuting; same target, no derivative chain)")
    ap.add_argument("--beta", type=float, default=BETA,
                    help="override beta (shorter imaginary-time axis, same kernels and matrix "
                         "sizes; used for profiler launch lists)")
    args = ap.parse_args()
    globals()["BETA"] = args.beta
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
