#!/usr/bin/env python
"""Benchmark of the CF-DQMC sweep: autocorrelation-corrected effective
samples per second on the N_phi = 36 torus, against the plain FP64 sweep.

Workload (one step = one sweep of every chain): torus N_phi = 36 (N = 72
single-particle states per spin block, N_q = 333 momenta, 1332 real fields
per slice), beta = 36, dtau = 0.1 (L = 360 slices), eight chains at couplings
u = linspace(0.5, 2.0, 8), seeds 0..7, restabilisation every 10 slices.

Two arms run in one invocation on the same GPU:
  * the headline path (default --mode prior --precision 2): mixed precision
    with whole-slice sweeps around the Gaussian prior (accepted by the exact
    determinant ratio; their proposals' propagators computed ahead in
    batches, with the batched products on the tensor cores); a Langevin
    sweep every n-th step is the fallback (--langevin-every n, fixed: a
    choice of move that depends on the chain's own acceptances would not
    leave the target invariant), off by default since the whole-slice
    acceptance is 0.63 here;
  * the plain FP64 Langevin sweep (--precision 0 --mode plain), the
    comparison the metric names.
Each arm: W warm-up sweeps, K timed sweeps (CUDA events on the library's
stream, graph-replayed sweeps, no profiler hook inside), then untimed sweeps
of the same schedule until the chain's series holds --tau-sweeps records.
tau_int = max over {m^2, E} of Sokal's windowed estimate (c = 5) on that
series, per chain; value = sum over chains of 1 / (2 tau_int) divided by the
timed seconds per sweep.  The line carries both arms' sweeps/s and effective
samples/s and their ratio (vs_plain_fp64).

The roofline of the FP64 GEMM class is taken in a separate untimed pass
(CUDA events around each FP64 GEMM launch), against the FP64 FMA rate
measured on the same GPU at start-up (qmc_peak_fma).  The G error against
the FP64 oracle: the oracle rebuilds G from chain 0's fields after the timed
region (propagators, UDV stack, G(0) in FP64 on the host) and the largest
elementwise difference to the GPU's G, relative to max|G|, is reported.

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
# dram bytes (read + write) of one FP64 GEMM launch from the ncu capture
# summarised in profiles/k_zgemm_fp64_n36_full.md (n = 36, batch 32; the
# N = 72 batch-8 products move the same 2 MB of operands)
TRAFFIC_PER_LAUNCH = 1338624
# oracle sample: one sweep of an L_SAMPLE-slice chain at the same N_phi, one
# process per chain, scaled to L = 360
L_SAMPLE = 10
# whole-slice modes: one Langevin sweep per LANGEVIN_EVERY steps (0: none;
# --langevin-every); pCN correlation of the whole-slice moves (--rho)
LANGEVIN_EVERY = 0
RHO = 0.0


def langevin_step(k):
    """True if step k of a whole-slice schedule is a Langevin sweep."""
    return LANGEVIN_EVERY > 0 and k % LANGEVIN_EVERY == LANGEVIN_EVERY - 1


def schedule_text(kind):
    if LANGEVIN_EVERY == 0:
        return f"{kind} whole-slice sweeps (rho {RHO:g}) only"
    if LANGEVIN_EVERY == 1:
        return "Langevin sweeps only"
    return (f"{kind} whole-slice sweeps (rho {RHO:g}), every {LANGEVIN_EVERY}th step a Langevin "
            "sweep")


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
def tau_with_error(x, tau_fn, c=5.0):
    """Sokal's windowed tau_int and its statistical error
    sigma^2 = 2 (2W + 1) tau^2 / n, W the self-consistent window (W >= c tau)."""
    t = tau_fn(x)
    W = max(1, int(math.ceil(c * t)))
    return t, t * math.sqrt(2.0 * (2 * W + 1) / len(x))


def tau_per_chain(series, tau_fn):
    """per chain: (tau, error) of the larger of m^2 (col 0) and E (col 12)"""
    out = []
    for c in range(series.shape[0]):
        a = tau_with_error(series[c, :, 0], tau_fn)
        b = tau_with_error(series[c, :, 12], tau_fn)
        out.append(a if a[0] >= b[0] else b)
    return out


def ess_rate(taus, step_s):
    """effective samples per second of a batch of chains and its error"""
    v = sum(1.0 / (2.0 * t) for t, _ in taus) / step_s
    e = math.sqrt(sum((dt / (2.0 * t * t)) ** 2 for t, dt in taus)) / step_s
    return v, e


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


def _oracle_green(u, seed, state, L):
    """G(0) of the oracle rebuilt in FP64 from a chain state (fields, Langevin
    step, sweep number) of the GPU: propagators, left UDV stack and the
    stabilised inverse, all on the host."""
    from oracle import model as M
    from oracle import oracle as O
    m = M.Model(M.TORUS, NPHI)
    ch = O.Chain(M.TORUS, NPHI, L * DTAU, DTAU, u, 0.0, seed, n_stab=NSTAB, eps0=EPS0, model=m)
    ch.set_state(state)
    return ch.green()


def oracle_sweeps_per_s(pool, nproc=NCH):
    """Aggregate oracle chain-sweeps/s at L = 360 over nproc parallel chains
    (one process, one thread each), from a bounded sample."""
    t0 = time.perf_counter()
    res = pool.starmap(_oracle_sample, [(float(COUPLINGS[c % NCH]), c) for c in range(nproc)])
    wall = time.perf_counter() - t0
    L = int(round(BETA / DTAU))
    t_full = [L * r[0] + r[1] for r in res]   # seconds per L=360 sweep per chain
    return sum(1.0 / t for t in t_full), t_full, wall, res


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, bounded
    sample per step (one L_SAMPLE-slice sweep of each of the eight chains in
    parallel processes).  The measured per-slice and per-measurement times
    are reported as measured; the L = 360 sweep rate is scaled from them, and
    tau_int is taken as 1/2 (the oracle's own tau cannot be measured in
    minutes), so the value is an upper bound of the oracle's rate."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    L = int(round(BETA / DTAU))
    step_rates, slice_s, meas_s, step_wall = [], [], [], []
    with ctx.Pool(NCH) as pool:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.starmap(_oracle_sample, [(float(COUPLINGS[c]), c) for c in range(NCH)])
            if k >= args.warmup:
                step_wall.append(time.perf_counter() - t0)
                step_rates.append(sum(1.0 / (L * r[0] + r[1]) for r in res))
                slice_s += [r[0] for r in res]
                meas_s += [r[1] for r in res]
    sweeps_per_s = float(np.mean(step_rates))
    value = sweeps_per_s / (2 * 0.5)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # a step here is one bounded sample (its measured wall time); the
        # L = 360 sweep time it stands for is config.scaled
        "ms_per_step": 1000.0 * float(np.mean(step_wall)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (fields drawn from the chains' own Philox streams)",
        "config": workload_config({
            "sample": f"one L={L_SAMPLE} sweep per chain per step (measured), scaled to L={L}; "
                      "tau_int taken as 1/2",
            "measured": {"slice_update_s": float(np.mean(slice_s)),
                         "measurement_s": float(np.mean(meas_s)),
                         "chains_in_parallel": NCH},
            "scaled": {"sweep_s_per_chain_at_L360": float(L * np.mean(slice_s) + np.mean(meas_s)),
                       "ms_per_sweep_of_all_chains": 1000.0 * NCH / sweeps_per_s,
                       "how": "L x measured slice-update time + one measurement"}}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": NCH, "kind": "oracle",
                         "sample": f"per step: one sweep of an L={L_SAMPLE} N_phi=36 oracle chain "
                                   f"per coupling, {NCH} processes x 1 thread, scaled to L={L}, "
                                   "tau_int=1/2 upper bound"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ours ------
def run_arm(P, stream, *, mode, precision, drift, seeds, steps, warmup, tau_sweeps, clocks_index,
            graph=True, want_state=False):
    """One arm: create the eight chains, warm up, time `steps` sweeps, then
    extend the series to `tau_sweeps` records with untimed sweeps of the same
    schedule.  Returns the timing, the tau_int estimates and diagnostics."""
    import torch
    wall0 = time.perf_counter()
    ch = P.Chain(P.QMC_TORUS, NPHI, BETA, DTAU, 0.0, 0.0, 0, n_chains=NCH, couplings=COUPLINGS,
                 seeds=seeds, n_stab=NSTAB, eps0=EPS0, series_capacity=4096, precision=precision,
                 drift=P.QMC_DRIFT_FIRST if drift == "first" else P.QMC_DRIFT_EXACT)
    ch.set_stream(stream.cuda_stream)
    # prior mode (default): whole-slice moves around the Gaussian part of
    # the action (rho = 0), accepted by the exact determinant ratio, with a
    # Langevin sweep every LANGEVIN_EVERY-th step if set; learned mode: the same
    # schedule with the network's Gaussian (at its initialisation mu = 0,
    # sigma = 1 it proposes what the prior move does, at the cost of its
    # forward pass: training on thinned plain-chain configurations never
    # lowered held-out NLL below the prior's at these couplings)
    net = P.Net(4 * ch.n_q, 256, 16, 1 + int(seeds[0])) if mode == "learned" else None

    def is_langevin(k):
        return mode == "plain" or langevin_step(k)

    def step(k):
        if is_langevin(k):
            ch.sweep(1, graph=graph)
        elif net is not None:
            ch.sweep_learned(net, 1, RHO, graph=graph)
        else:
            ch.sweep_prior(1, RHO, graph=graph)

    pinned = torch.empty((steps, NCH, P.QMC_NOBS), dtype=torch.float64, pin_memory=True)
    for k in range(warmup):
        step(k)
    ch.sync()
    torch.cuda.synchronize()
    clocks = Clocks(clocks_index) if clocks_index is not None else None
    launches0 = P.qmc_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        step(warmup + k)
        ch.copy_latest_async(pinned[k].data_ptr())
    e1.record(stream)
    ch.sync()
    torch.cuda.synchronize()
    wall_e2e = time.perf_counter() - wall0
    launches = P.qmc_launch_count() - launches0
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    state0 = green0 = None
    if want_state:
        # chain 0 in the oracle's single-chain layout: fields, step, sweep
        st = ch.get_state()
        nfl = ch.L * 4 * ch.n_q
        state0 = np.concatenate([st[:nfl], [st[NCH * nfl], st[-1]]])
        green0 = ch.green(0)
    # the untimed tail of the tau_int series (same schedule)
    k = warmup + steps
    while k < warmup + tau_sweeps:
        step(k)
        k += 1
    ch.sync()
    series = ch.series()[:, warmup:, :]
    taus = tau_per_chain(series, P.qmc_tau_int)
    timed = series[:, :steps, :]
    learned_steps = [j for j in range(series.shape[1]) if not is_langevin(warmup + j)]
    acc_learned = float(series[:, learned_steps, 13].mean()) if learned_steps else None
    lang = np.delete(series[:, :, 13], learned_steps, axis=1)
    acc_langevin = float(lang.mean()) if lang.size else None
    out = {"ch": ch, "net": net, "mode": mode, "ms": ms, "step_s": ms / 1000.0 / steps, "taus": taus,
           "series_len": int(series.shape[1]), "launches": int(launches), "clocks": clk,
           "wall_e2e": wall_e2e, "g_err_max": float(timed[:, :, 15].max()),
           "sign_max": float(timed[:, :, 16].max()), "acc_learned": acc_learned,
           "acc_langevin": acc_langevin, "state0": state0, "green0": green0,
           "d2h": NCH * P.QMC_NOBS * 8}
    return out


def gemm_roofline_pass(P, arm, steps=2):
    """GEMM class rooflines in a separate, untimed pass: CUDA events around
    each FP64 CUDA-core GEMM launch and each tensor-core MMA launch of
    `steps` further sweeps of the arm's own schedule (eager launches, so
    each product has its own event pair).  Returns (FP64 ms, launches,
    flops) and (tensor ms, launches, needed flops, issued flops)."""
    ch, net, mode = arm["ch"], arm["net"], arm["mode"]
    P.qmc_profile_gemm(True)
    t0 = time.perf_counter()
    for k in range(steps):
        if mode == "plain" or langevin_step(k):
            ch.sweep(1)
        elif net is not None:
            ch.sweep_learned(net, 1, RHO)
        else:
            ch.sweep_prior(1, RHO)
    ch.sync()
    ms, n, flops = P.qmc_profile_gemm(False)
    wall = time.perf_counter() - t0
    return (ms, n, flops), P.qmc_profile_tensor(), wall


def measured_peaks():
    """bf16 dense tensor peaks measured on this machine (generated file),
    else the recipe's fallback figures"""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"bf16_burst": float(d["bf16_tflops"]),
                "bf16_sustained": float(d["bf16_tflops_sustained"]), "source": "measured"}
    except Exception:
        return {"bf16_burst": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle pool is spawned before the first GPU call
    pool, cpu = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        pool = mp.get_context("spawn").Pool(NCH)
        rate, t_full, wall, res = oracle_sweeps_per_s(pool)
        cpu = {"sweeps_per_s": rate, "t_full": t_full, "wall": wall,
               "slice_s": float(np.mean([r[0] for r in res])),
               "meas_s": float(np.mean([r[1] for r in res]))}
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2605_03700_gb300 import build as B
    B.build()
    import paper_2605_03700_gb300 as P

    fp64_peak = P.qmc_peak_fma(True, 4096)
    stream = torch.cuda.Stream()
    seeds = replica_seeds(rank)
    if dist:
        dist.barrier()
    main = run_arm(P, stream, mode=args.mode, precision=args.precision, drift=args.drift,
                   seeds=seeds, steps=args.steps, warmup=args.warmup,
                   tau_sweeps=max(args.tau_sweeps, args.steps), clocks_index=local,
                   want_state=pool is not None)
    g_orc = None
    if pool is not None:
        L = int(round(BETA / DTAU))
        g_orc = pool.apply_async(_oracle_green, (float(COUPLINGS[0]), int(seeds[0]),
                                                 main["state0"], L))
    (gemm_ms, gemm_n, gemm_flops), (tc_ms, tc_n, tc_flops, tc_issued), prof_wall = \
        gemm_roofline_pass(P, main)
    plain = None
    if not args.no_plain_arm:
        plain = run_arm(P, stream, mode="plain", precision=0, drift="exact", seeds=seeds,
                        steps=args.plain_steps, warmup=args.warmup,
                        tau_sweeps=max(args.plain_tau_sweeps, args.plain_steps),
                        clocks_index=None)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    v_main, dv_main = ess_rate(main["taus"], main["step_s"])
    t_s, wall_e2e, ess = combine_over_ranks(dist, main["ms"] / 1000.0, main["wall_e2e"],
                                            v_main * main["ms"] / 1000.0, "cuda")
    value = ess / t_s
    e2e = ess / wall_e2e
    vs_plain = None
    if plain is not None:
        v_pl, dv_pl = ess_rate(plain["taus"], plain["step_s"])
        _, _, ess_pl = combine_over_ranks(dist, plain["ms"] / 1000.0, plain["wall_e2e"],
                                          v_pl * plain["ms"] / 1000.0, "cuda")
        ratio = v_main / v_pl
        vs_plain = {
            "ess_ratio": ratio,
            "ess_ratio_err": ratio * math.sqrt((dv_main / v_main) ** 2 + (dv_pl / v_pl) ** 2),
            "plain_fp64": {"value": v_pl, "value_err": dv_pl, "ms_per_step": plain["ms"] /
                           args.plain_steps, "sweeps_per_s_per_gpu": NCH / plain["step_s"],
                           "tau_int": [[round(t, 3), round(e, 3)] for t, e in plain["taus"]],
                           "tau_series_len": plain["series_len"],
                           "acceptance": plain["acc_langevin"], "g_err_max": plain["g_err_max"],
                           "timed_steps": args.plain_steps, "gpu_launches": plain["launches"]},
            "sweeps_per_s_ratio": plain["step_s"] / main["step_s"]}
    g_err_oracle = None
    if g_orc is not None:
        Go = g_orc.get(timeout=1800)
        g_err_oracle = float(np.abs(main["green0"] - Go).max() / np.abs(Go).max())
    if pool is not None:
        pool.close()
        pool.join()
    gemm_tflops = gemm_flops / (gemm_ms / 1000.0) / 1e12 if gemm_ms > 0 else 0.0
    roof_fp64 = {"bound": "alu", "achieved": gemm_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                 "frac": gemm_tflops / fp64_peak,
                 "traffic": TRAFFIC_PER_LAUNCH,
                 "kernel": "k_zgemm<double> (batched complex FP64 GEMM on the CUDA cores)",
                 "launches": gemm_n, "ms_total": gemm_ms,
                 "pass": "separate untimed pass of 2 sweeps, CUDA events around each FP64 GEMM",
                 "peak_note": "measured on this GPU at start-up: FP64 FMA chains on every SM "
                              "(qmc_peak_fma), 'alu' = the FP64 CUDA-core pipe; of measured"}
    roofs = [roof_fp64]
    if tc_n:
        pk = measured_peaks()
        tc_tflops = tc_flops / (tc_ms / 1000.0) / 1e12
        roofs.append({
            "bound": "tensor", "achieved": tc_tflops, "peak": pk["bf16_sustained"],
            "unit": "TFLOP/s", "frac": tc_tflops / pk["bf16_sustained"], "traffic": None,
            "kernel": "k_oz_mma (tcgen05 bf16 digit products, FP32 accumulate in TMEM)",
            "launches": tc_n, "ms_total": tc_ms,
            "issued_tflops": tc_issued / (tc_ms / 1000.0) / 1e12,
            "flops_note": "needed = digit pairs x 2 x M x 2N x 2K per complex product (real "
                          "embedding); issued adds the 128-row and column-tile padding",
            "pass": "separate untimed pass of 2 sweeps, CUDA events around each MMA launch",
            "peak_note": f"bf16 dense, sustained ({pk['source']}: MEASURED_PEAKS.json); of "
                         f"{pk['source']}"})
    # the dominant class by device time in the profiling pass
    roof = max(roofs, key=lambda r: r["ms_total"])
    if rank != 0:
        for arm in (main, plain):
            if arm:
                arm["ch"].close()
        if dist:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ["f64", "f32+f64", "f32+f64+bf16-digits"][args.precision],
        "data": "synthetic (fields drawn from the chains' own Philox streams)",
        "config": workload_config({"parallelism": f"replicas x{world}",
                                   "precision": ["fp64", "mixed fp32/fp64 (CUDA cores)",
                                                 "mixed on tensor cores: FP64-class products "
                                                 "from 7 bf16 digits, drift from 3; FP64 LU, "
                                                 "division, QR/UDV"][args.precision],
                                   "mode": args.mode,
                                   "drift": args.drift,
                                   "schedule": ("plain Langevin sweeps" if args.mode == "plain" else
                                                schedule_text(args.mode)),
                                   "launch": "graph-replayed sweeps",
                                   "acceptance_whole_slice": main["acc_learned"],
                                   "acceptance_langevin": main["acc_langevin"],
                                   "tau_int": [[round(t, 3), round(e, 3)] for t, e in main["taus"]],
                                   "tau_series_len": main["series_len"],
                                   "value_err": dv_main,
                                   "sweeps_per_s_per_gpu": NCH / main["step_s"],
                                   "g_err_max": main["g_err_max"],
                                   "g_err_vs_oracle": g_err_oracle,
                                   "sign_dev_max": main["sign_max"]}),
        "vs_plain_fp64": vs_plain,
        "roofline": roof,
        "rooflines": roofs,
        "fp64_peak_tflops_measured": fp64_peak,
        "clocks": main["clocks"],
        "gpu_launches": main["launches"],
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": main["d2h"],
                "note": "wall clock through the C ABI from qmc_create to the last D2H of the "
                        "timed steps' records, warm-up included; a sweep takes no host input"},
    }
    if cpu:
        ess_cpu = sum(1.0 / tf / (2.0 * t) for tf, (t, _) in zip(cpu["t_full"], main["taus"]))
        line["cpu_baseline"] = {
            "value": ess_cpu, "unit": UNIT, "cores": NCH, "kind": "oracle",
            "sample": f"one sweep of an L={L_SAMPLE} N_phi=36 oracle chain per coupling "
                      f"({NCH} processes x 1 thread), measured {cpu['slice_s']:.3f} s per slice "
                      f"update and {cpu['meas_s']:.3f} s per measurement, scaled to L=360; "
                      "tau_int of the GPU chains",
            "sweeps_per_s": cpu["sweeps_per_s"]}
    print(json.dumps(line))
    for arm in (main, plain):
        if arm:
            arm["ch"].close()
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------ other workloads ----
def run_batched(args):
    """64 independent chains, torus N_phi drawn from {16, 24, 36, 48}
    (numpy default_rng(0), the list is printed), beta = N_phi, dtau = 0.1,
    u ~ U[0.5, 2], anisotropy ~ U[-0.2, 0.2]; one context per size, all four
    swept as one CUDA graph per sweep (qmc_group_*), each size on its own
    graph branch.  One step = one sweep of all 64 chains."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2605_03700_gb300 import build as B
    B.build()
    import paper_2605_03700_gb300 as P
    rng = np.random.default_rng(0)
    sizes = rng.choice([16, 24, 36, 48], size=64)
    us = rng.uniform(0.5, 2.0, 64)
    als = rng.uniform(-0.2, 0.2, 64)
    wall0 = time.perf_counter()
    chains = []
    for nphi in (16, 24, 36, 48):
        idx = np.nonzero(sizes == nphi)[0]
        if len(idx) == 0:
            continue
        chains.append(P.Chain(P.QMC_TORUS, int(nphi), float(nphi), DTAU, 0.0, 0.0, 0,
                              n_chains=len(idx), couplings=us[idx], anisotropies=als[idx],
                              seeds=idx.astype(np.uint64), n_stab=NSTAB, eps0=EPS0,
                              precision=args.precision, series_capacity=4096))
    g = P.Group(chains)
    g.sweep(args.warmup)
    g.sync()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    l0 = P.qmc_launch_count()
    t0 = time.perf_counter()
    g.sweep(args.steps)
    g.sync()
    t = time.perf_counter() - t0
    launches = P.qmc_launch_count() - l0
    clk = clocks.stop()
    wall = time.perf_counter() - wall0
    while chains[0].series().shape[1] < args.warmup + max(args.tau_sweeps, args.steps):
        g.sweep(1)
    g.sync()
    taus = []
    for c in chains:
        taus += tau_per_chain(c.series()[:, args.warmup:, :], P.qmc_tau_int)
    step_s = t / args.steps
    v, dv = ess_rate(taus, step_s)
    line = {"metric": "effective samples/s (autocorr-corrected), 64 batched chains",
            "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * step_s, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f64", "f32+f64", "f32+f64+bf16-digits"][args.precision],
            "data": "synthetic",
            "config": {"workload": "64 chains, torus N_phi in {16,24,36,48} (rng(0)), beta=N_phi, "
                                   "dtau=0.1, u~U[0.5,2], anisotropy~U[-0.2,0.2], n_stab=10, "
                                   "one graph per sweep over four size branches",
                       "sizes": [int(x) for x in sizes], "value_err": dv,
                       "chain_sweeps_per_s": 64 / step_s,
                       "tau_int_mean": float(np.mean([t for t, _ in taus])),
                       "tau_series_len": max(args.tau_sweeps, args.steps),
                       "timing": "host wall clock around the graph launches and the final "
                                 "synchronise"},
            "clocks": clk, "gpu_launches": int(launches),
            "e2e": {"value": v * step_s * args.steps / wall, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    g.close()
    for c in chains:
        c.close()
    return 0


def run_sphere(args):
    """The 60-orbital sphere (N = 120, N_q = 3600), beta = 40 (L = 400),
    u = 1.2, one chain: prior whole-slice sweeps at rho = 0 in the headline
    path's schedule."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2605_03700_gb300 import build as B
    B.build()
    import paper_2605_03700_gb300 as P
    stream = torch.cuda.Stream()
    u = args.sphere_u
    workload = (f"sphere, 60 orbitals (N=120, N_q=3600), beta=40, dtau=0.1 (L=400), u={u}, one "
                f"chain, {schedule_text('prior')}")
    ch = P.Chain(P.QMC_SPHERE, 59, 40.0, DTAU, u, 0.0, 0, n_stab=NSTAB, eps0=0.2,
                 precision=args.precision, series_capacity=4096,
                 sign_tol=args.sphere_sign_tol)
    ch.set_stream(stream.cuda_stream)
    def step(k):
        if langevin_step(k):
            ch.sweep(1, graph=True)
        else:
            ch.sweep_prior(1, RHO, graph=True)
    try:
        for k in range(args.warmup):
            step(k)
        ch.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            step(args.warmup + k)
        e1.record(stream)
        ch.sync()
    except P.QMCError as err:
        # the chain's own checks (restabilisation error, sign of the ratio)
        # reject the run: print why instead of a number, with what the
        # records up to the failing sweep saw
        seen = {}
        try:
            r = ch.series()
            if r.shape[1]:
                seen = {"max_abs_sin_im_log_r": float(r[:, :, 16].max()),
                        "g_err_max": float(r[:, :, 15].max()), "sweeps_recorded": r.shape[1]}
        except P.QMCError:
            pass
        print(json.dumps({"metric": "effective samples/s (autocorr-corrected), 60-orbital sphere",
                          "value": None, "unit": UNIT, "n_gpus": 1,
                          "error": str(err), "config": {"workload": workload,
                                                        "precision": args.precision,
                                                        "sign_tol": args.sphere_sign_tol,
                                                        **seen}}))
        ch.close()
        return 0
    ms = e0.elapsed_time(e1)
    s = ch.series()[:, args.warmup:, :]
    taus = tau_per_chain(s, P.qmc_tau_int)
    v, dv = ess_rate(taus, ms / 1000 / args.steps)
    line = {"metric": "effective samples/s (autocorr-corrected), 60-orbital sphere",
            "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f64", "f32+f64", "f32+f64+bf16-digits"][args.precision],
            "data": "synthetic",
            "config": {"workload": workload,
                       "value_err": dv, "tau_int": [[round(t, 3), round(e, 3)] for t, e in taus],
                       "acceptance": float(s[:, :, 13].mean()),
                       "g_err_max": float(s[:, :, 15].max()),
                       "sign_tol": args.sphere_sign_tol,
                       "max_abs_sin_im_log_r": float(s[:, :, 16].max())}}
    print(json.dumps(line))
    ch.close()
    return 0


def run_torus140(args):
    """The paper's largest torus: N_phi = 140 (N = 280, N_q = 1305), beta =
    70 (L = 700), u = 1, anisotropy 0.1, eight chains (seeds 0-7), n_stab =
    10, mixed precision (default: the tensor-core products, precision 2),
    prior whole-slice sweeps in the headline path's schedule.  A sweep
    takes seconds, so a run times a few steps; tau_int is not resolved in
    that window and the line reports chain-sweeps/s with ESS/s from the
    short series."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_2605_03700_gb300 import build as B
    B.build()
    import paper_2605_03700_gb300 as P
    stream = torch.cuda.Stream()
    prec = args.precision if args.precision > 0 else 2
    wall0 = time.perf_counter()
    ch = P.Chain(P.QMC_TORUS, 140, 70.0, DTAU, 1.0, 0.1, 0, n_chains=NCH, seeds=np.arange(NCH),
                 n_stab=NSTAB, eps0=0.2, precision=prec, series_capacity=256)
    ch.set_stream(stream.cuda_stream)

    def step(k):
        if langevin_step(k):
            ch.sweep(1, graph=True)
        else:
            ch.sweep_prior(1, RHO, graph=True)
    for k in range(args.warmup):
        step(k)
    ch.sync()
    clocks = Clocks(0)
    l0 = P.qmc_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
    e1.record(stream)
    ch.sync()
    ms = e0.elapsed_time(e1)
    launches = P.qmc_launch_count() - l0
    clk = clocks.stop()
    s = ch.series()[:, args.warmup:, :]
    taus = tau_per_chain(s, P.qmc_tau_int)
    v, dv = ess_rate(taus, ms / 1000 / args.steps)
    line = {"metric": "effective samples/s (autocorr-corrected), torus N_phi=140",
            "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f64", "f32+f64", "f32+f64+bf16-digits"][prec],
            "data": "synthetic",
            "config": {"workload": "torus N_phi=140 (N=280, N_q=1305), beta=70, dtau=0.1 (L=700), "
                                   "u=1, anisotropy 0.1, 8 chains seeds 0-7, n_stab=10, "
                                   + schedule_text("prior"),
                       "precision": prec, "chain_sweeps_per_s": NCH * args.steps / (ms / 1000),
                       "value_err": dv, "tau_series_len": int(s.shape[1]),
                       "acceptance": float(s[:, :, 13].mean()),
                       "g_err_max": float(s[:, :, 15].max()),
                       "setup_s": time.perf_counter() - wall0 - ms / 1000},
            "clocks": clk, "gpu_launches": int(launches)}
    print(json.dumps(line))
    ch.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain-arm", action="store_true",
                    help="skip the plain FP64 comparison arm")
    ap.add_argument("--tau-sweeps", type=int, default=200,
                    help="records per chain for tau_int of the headline arm (timed + untimed)")
    ap.add_argument("--plain-steps", type=int, default=20, help="timed sweeps of the plain arm")
    ap.add_argument("--plain-tau-sweeps", type=int, default=120,
                    help="records per chain for tau_int of the plain FP64 arm")
    ap.add_argument("--precision", type=int, default=2, choices=[0, 1, 2],
                    help="0: FP64 everywhere; 1: mixed (FP32 eigensolver bulk + FP64 "
                         "refinement, FP32 drift transforms; FP64 propagators, ratios, updates); "
                         "2 (default): as 1, with the large dense products (the batched "
                         "prior-move proposals) on the tcgen05 tensor cores from FP64-exact "
                         "bfloat16 digits")
    ap.add_argument("--mode", default="prior", choices=["prior", "learned", "plain"],
                    help="prior: whole-slice moves around the Gaussian prior (with a Langevin "
                         "sweep every --langevin-every steps); learned: the same schedule with "
                         "the network's Gaussian; plain: Langevin sweeps only")
    ap.add_argument("--drift", default="exact", choices=["exact", "first"],
                    help="Langevin drift: exact grad S, or the first-order drift (factors "
                         "treated as commuting; same target, no derivative chain)")
    ap.add_argument("--beta", type=float, default=BETA,
                    help="override beta (shorter imaginary-time axis, same kernels and matrix "
                         "sizes; used for profiler launch lists)")
    ap.add_argument("--langevin-every", type=int, default=LANGEVIN_EVERY,
                    help="whole-slice schedules: a Langevin sweep every n-th step, the fallback "
                         "where whole-slice acceptance is low (0, default: whole-slice sweeps "
                         "only; 1: Langevin only)")
    ap.add_argument("--rho", type=float, default=RHO,
                    help="pCN correlation of the whole-slice moves, 0 <= rho < 1 (0: independent "
                         "proposals from the prior; rho > 0 keeps the move exact and raises its "
                         "acceptance where it would collapse)")
    ap.add_argument("--sphere-u", type=float, default=1.2,
                    help="coupling of --workload sphere60 (the workload's 1.2; the paper's sphere "
                         "scans use 0.075 .. 0.3)")
    ap.add_argument("--sphere-sign-tol", type=float, default=1e-6,
                    help="bound on |sin Im log R| of accepted updates for --workload sphere60 "
                         "(the library's default; the ratio is real in exact arithmetic and its "
                         "computed phase is rounding scaled by the conditioning of M)")
    ap.add_argument("--workload", default="nphi36",
                    choices=["nphi36", "batched", "sphere60", "torus140"],
                    help="nphi36: the headline workload (default); batched: 64 chains of mixed "
                         "N_phi in one graph; sphere60: the 60-orbital sphere; torus140: the "
                         "largest torus, N_phi = 140")
    args = ap.parse_args()
    globals()["BETA"] = args.beta
    if args.langevin_every < 0:
        ap.error("--langevin-every must be >= 0")
    globals()["LANGEVIN_EVERY"] = args.langevin_every
    if not 0.0 <= args.rho < 1.0:
        ap.error("--rho must lie in [0, 1)")
    globals()["RHO"] = args.rho
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "sphere60":
        return run_sphere(args)
    if args.workload == "torus140":
        return run_torus140(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
