"""Parity with the FP64 oracle at the benchmark's configuration.

The benchmark times torus N_phi = 36 (N = 72, N_q = 333, 1332 fields per
slice), n_stab = 10, eps0 = 0.45, couplings in [0.5, 2.0], in FP64 (the plain
sweep) and in mixed precision with learned whole-slice moves.  Here the same
kernels, sizes and schedule run with beta = 4 (L = 40): four restabilisations
per sweep, three of them interior, and left/right UDV stacks of four blocks,
for 400 updates per chain (10 sweeps).  The oracle chains run in spawned
worker processes while the GPU works.

 (a) FP64 Langevin sweeps: decision-identical over all 400 updates,
     log R within 1e-10, G within 1e-9 of max|G| after every sweep.
 (b) Mixed precision (FP32 drift transforms, FP32 Jacobi bulk with FP64
     refinement; everything in the MH ratio FP64-accurate), on the CUDA
     cores (precision 1) and in precision 2 (whose products at these batch
     sizes stay below the tensor-core threshold; (d) moves them all onto
     the tensor cores): the index of the first decision that differs from the
     oracle, and G against the oracle after every sweep up to it, within
     1e-6 (the G-error target of mixed runs).
 (c) Learned sweeps at rho = 0 with a seeded non-zero network of the
     benchmark's width (256), every fourth sweep a Langevin sweep, in both
     mixed modes.
 (d) The benchmark's default schedule: whole-slice moves around N(0, 1)
     only, their proposals computed ahead in batches (qmc_sweep_prior,
     graph-replayed), in FP64 (decision-identical, log R 1e-10, G 1e-9) and
     in precision 2, once with the default tensor-core threshold (at L = 40
     the stage's batches are small and stay on the CUDA cores) and once with
     every product on the tensor cores (QMC_OZ_MIN_WORK=1, in a fresh
     process): decisions tracking the oracle, G within 1e-6.
"""
import os
import subprocess
import sys
import multiprocessing as mp

import numpy as np
import pytest

from tests import oracle_runs as R
from tests.learned_inputs import random_params

pytestmark = pytest.mark.gpu

NPHI, BETA, DTAU, NSTAB, EPS0 = 36, 4.0, 0.1, 10, 0.45
COUPLINGS = (0.5, 2.0)
NSW = 10
SCHEDULE = "NNNPNNNPNN"   # the benchmark's --langevin-every 4: every fourth step Langevin
NET_H, NET_SEED = 256, 17


def _theta(nf):
    # non-zero output layer: mu and log sigma depend on the neighbouring
    # slices (|mu| ~ 0.05, sigma ~ e^{+-0.05})
    return random_params(nf, NET_H, NET_SEED, out_scale=0.05, logsig_bias=0.02)


@pytest.fixture(scope="module")
def oracle_results():
    """All oracle chains of this module, computed in parallel processes."""
    from oracle import oracle as O
    O.build()
    nf = 4 * 333
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(len(COUPLINGS) + 2)
    jobs = {("lang", c): pool.apply_async(R.langevin_chain,
                                          (NPHI, BETA, DTAU, u, 0.0, c, NSTAB, EPS0, NSW))
            for c, u in enumerate(COUPLINGS)}
    from oracle import model as M
    jobs[("prior", 0)] = pool.apply_async(
        R.plain_chain, (M.TORUS, NPHI, BETA, DTAU, 1.25, 0.0, 5, NSTAB, EPS0, NSW),
        dict(schedule="0" * NSW))
    jobs[("sched", 0)] = pool.apply_async(
        R.scheduled_chain, (NPHI, BETA, DTAU, 1.25, 0.0, 5, NSTAB, EPS0, SCHEDULE,
                            _theta(nf), NET_H, 0.0))
    pool.close()
    cache = {}

    def get(key):
        if key not in cache:
            cache[key] = jobs[key].get(timeout=1800)
        return cache[key]
    yield get
    pool.terminate()


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _gpu_langevin(qmc, precision):
    g = qmc.Chain(qmc.QMC_TORUS, NPHI, BETA, DTAU, 0.0, 0.0, 0, n_chains=len(COUPLINGS),
                  couplings=list(COUPLINGS), seeds=list(range(len(COUPLINGS))), n_stab=NSTAB,
                  eps0=EPS0, precision=precision, trace_capacity=NSW * 40)
    greens = []
    for _ in range(NSW):
        g.sweep(1)
        g.sync()
        greens.append([g.green(c) for c in range(len(COUPLINGS))])
    return g, greens


def test_fp64_langevin_decision_identical_at_benchmark_size(qmc, oracle_results):
    g, greens = _gpu_langevin(qmc, 0)
    for c in range(len(COUPLINGS)):
        o = oracle_results(("lang", c))
        tg, to = g.trace(c), o["trace"]
        assert len(tg) == len(to) == NSW * 40
        assert np.array_equal(tg[:, 6], to[:, 6]), "accept decisions differ"
        assert 0 < to[:, 6].sum() < len(to)
        assert np.array_equal(tg[:, :2], to[:, :2])
        assert np.abs(tg[:, 2] - to[:, 2]).max() < 1e-10
        assert np.abs(tg[:, 7] - to[:, 7]).max() < 1e-12
        for k in range(NSW):
            assert _rel(greens[k][c], o["green"][k]) < 1e-9, f"G differs after sweep {k}"
        assert np.abs(g.fields(c) - o["phi"]).max() < 1e-9
        obs_g = g.series()[c]
        for col in (0, 1, 3, 6, 11, 12):
            ref = o["obs"][:, col]
            assert np.abs(obs_g[:, col] - ref).max() < 1e-9 * max(1, np.abs(ref).max())
        # every restabilisation of the GPU chain found G fresh to 1e-9
        assert obs_g[:, 15].max() < 1e-9


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_tracks_the_oracle_at_benchmark_size(qmc, oracle_results, record_property,
                                                             precision):
    g, greens = _gpu_langevin(qmc, precision)
    for c in range(len(COUPLINGS)):
        o = oracle_results(("lang", c))
        tg, to = g.trace(c), o["trace"]
        mis = np.nonzero(tg[:, 6] != to[:, 6])[0]
        first = int(mis[0]) if len(mis) else len(tg)
        record_property(f"first_divergence_u{COUPLINGS[c]}", first)
        # the FP32 drift moves log A by ~1e-7: a decision can only flip when
        # log u lies that close to log A
        assert first >= 200, f"decisions diverge at update {first}"
        assert np.abs(tg[:first, 2] - to[:first, 2]).max() < 1e-5
        assert np.abs(tg[:first, 3]).max() < 1e-8
        gerr = [_rel(greens[k][c], o["green"][k]) for k in range(first // 40)]
        record_property(f"g_err_vs_oracle_u{COUPLINGS[c]}", max(gerr) if gerr else None)
        assert all(e < 1e-6 for e in gerr), gerr
        assert g.series()[c][:, 15].max() < 1e-8


@pytest.mark.parametrize("precision", [1, 2])
def test_learned_schedule_tracks_the_oracle_at_benchmark_size(qmc, oracle_results,
                                                              record_property, precision):
    g = qmc.Chain(qmc.QMC_TORUS, NPHI, BETA, DTAU, 1.25, 0.0, 5, n_stab=NSTAB, eps0=EPS0,
                  precision=precision, trace_capacity=len(SCHEDULE) * 40)
    nf = 4 * g.n_q
    net = qmc.Net(nf, NET_H, 16, 3)
    net.set_params(_theta(nf).astype(np.float32))
    greens, phis = [], []
    for kind in SCHEDULE:
        if kind == "P":
            g.sweep(1)
        else:
            g.sweep_learned(net, 1, 0.0)
        g.sync()
        greens.append(g.green(0))
        phis.append(g.fields(0))
    o = oracle_results(("sched", 0))
    tg, to = g.trace(0), o["trace"]
    assert len(tg) == len(to) == len(SCHEDULE) * 40
    mis = np.nonzero(tg[:, 6] != to[:, 6])[0]
    first = int(mis[0]) if len(mis) else len(tg)
    record_property("first_divergence", first)
    assert first >= 200, f"decisions diverge at update {first}"
    learned = np.array([SCHEDULE[int(s)] == "N" for s in to[:first, 0]])
    assert learned.any() and 0 < to[:first][learned, 6].sum() < learned.sum()
    # mu and sigma from bfloat16 weights with FP32 accumulation: proposals
    # agree to ~1e-6 relative
    assert np.abs(tg[:first, 2] - to[:first, 2]).max() < 1e-5
    nsw_same = first // 40
    for k in range(nsw_same):
        assert np.abs(phis[k] - o["phi"][k]).max() < 1e-4
        assert _rel(greens[k], o["green"][k]) < 1e-6
    obs_g = g.series()[0]
    assert np.array_equal(obs_g[:nsw_same, 17], o["obs"][:nsw_same, 17])


PRIOR_RUN = """
import sys
import numpy as np
sys.path.insert(0, ".")
from paper_2605_03700_gb300 import build
build.build()
import paper_2605_03700_gb300 as P
prec, nsw, path = int(sys.argv[1]), int(sys.argv[2]), sys.argv[3]
g = P.Chain(P.QMC_TORUS, 36, 4.0, 0.1, 1.25, 0.0, 5, n_stab=10, eps0=0.45, precision=prec,
            trace_capacity=nsw * 40)
g.sweep_prior(nsw, 0.0, graph=True)
g.sync()
np.savez(path, trace=g.trace(0), green=g.green(0), phi=g.fields(0), obs=g.series()[0])
"""


@pytest.mark.parametrize("precision,min_work", [(0, None), (2, None), (2, "1")])
def test_default_schedule_tracks_the_oracle_at_benchmark_size(oracle_results, tmp_path,
                                                             precision, min_work):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.pop("QMC_OZ_MIN_WORK", None)
    if min_work is not None:
        env["QMC_OZ_MIN_WORK"] = min_work
    path = str(tmp_path / "prior.npz")
    r = subprocess.run([sys.executable, "-c", PRIOR_RUN, str(precision), str(NSW), path], cwd=root,
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    g = np.load(path)
    o = oracle_results(("prior", 0))
    tg, to = g["trace"], o["trace"]
    assert len(tg) == len(to) == NSW * 40
    assert 0 < to[:, 6].sum() < len(to)
    if precision == 0:
        assert np.array_equal(tg[:, 6], to[:, 6]), "accept decisions differ"
        assert (np.abs(tg[:, 2] - to[:, 2]) / np.maximum(1, np.abs(to[:, 2]))).max() < 1e-10
        assert _rel(g["green"], o["green"]) < 1e-9
        assert np.abs(g["phi"] - o["phi"]).max() < 1e-9
        assert np.array_equal(g["obs"][:, 17], o["obs"][:, 17])
        return
    mis = np.nonzero(tg[:, 6] != to[:, 6])[0]
    first = int(mis[0]) if len(mis) else len(tg)
    assert first >= 200, f"decisions diverge at update {first}"
    assert (np.abs(tg[:first, 2] - to[:first, 2]) / np.maximum(1, np.abs(to[:first, 2]))).max() < 1e-6
    if first == len(tg):
        assert _rel(g["green"], o["green"]) < 1e-6
        assert np.abs(g["phi"] - o["phi"]).max() < 1e-9
