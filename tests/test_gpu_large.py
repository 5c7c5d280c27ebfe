"""Parity with the FP64 oracle at the largest matrix size the kernels take,
N = 120 (one spin block of 60 orbitals): the torus at N_phi = 60 (N_q = 553)
and the 60-orbital sphere of the benchmark's learned-proposal workload
(N_q = 3600, Methods Eq. sphere_density_operator) at its coupling u = 1.2
and at a strong coupling.  At this size the LU keeps
its matrix at row stride n, QR with pivoting keeps only the matrix and the
Householder vector in shared memory, and the right division stages its
factors in row chunks.  The oracle chains run in spawned workers while the
GPU works: identical decisions, log R within 1e-10 (relative to
max(1, |log R|)), G within 1e-9 of max|G|; in precision 2 (dense products on
the tensor cores) the chain tracks the oracle."""
import multiprocessing as mp

import numpy as np
import pytest

from oracle import model as M
from tests import oracle_runs as R
from tests.sphere_units import sphere_u

pytestmark = pytest.mark.gpu

TORUS = dict(size=60, beta=1.0, u=1.0, anis=0.1, seed=2, n_stab=5, eps0=0.3, nsw=2)
# the sphere at the workload's coupling u = 1.2 (torus-matched form factors),
# and at a strong coupling, 4 pi^2 n_orb * 0.3 (tests/sphere_units.py), where
# B is ill-conditioned
SPHERE_W = dict(size=60, beta=1.0, u=1.2, anis=0.0, seed=3, n_stab=5, eps0=0.3, nsw=1)
SPHERE = dict(size=60, beta=1.0, u=sphere_u(0.3, 60), anis=0.0, seed=3, n_stab=5, eps0=0.3,
              nsw=1)
CASES = {"torus": (M.TORUS, TORUS), "sphere": (M.SPHERE, SPHERE), "sphere_w": (M.SPHERE, SPHERE_W)}


@pytest.fixture(scope="module")
def oracle_results():
    from oracle import oracle as O
    O.build()
    pool = mp.get_context("spawn").Pool(3)
    jobs = {}
    for key, (geom, c) in CASES.items():
        jobs[key] = pool.apply_async(R.plain_chain, (geom, c["size"], c["beta"], 0.1, c["u"],
                                                     c["anis"], c["seed"], c["n_stab"],
                                                     c["eps0"], c["nsw"]))
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


def _gpu(qmc, geom, c, precision):
    nphi = c["size"] if geom == qmc.QMC_TORUS else c["size"] - 1
    L = int(round(c["beta"] / 0.1))
    # stab_tol: the sphere's wrapped G drifts from the stable one by ~1e-6
    # between restabilisations at this conditioning (the measured drift is
    # recorded in column 15 and bounded below)
    g = qmc.Chain(geom, nphi, c["beta"], 0.1, c["u"], c["anis"], c["seed"], n_stab=c["n_stab"],
                  eps0=c["eps0"], precision=precision, trace_capacity=c["nsw"] * L,
                  stab_tol=1e-3)
    assert g.N == 120
    g.sweep(c["nsw"])
    g.sync()
    return g


# (case, log R tolerance relative to max(1, |log R|), G tolerance,
# restabilisation drift bound).  On the 60-orbital sphere at the strong
# coupling G(tau) has condition number ~2e11: the oracle's stable ratio and
# its brute-force determinant ratio of the same proposal differ by
# 3e-7 .. 5e-7 there, so two FP64 evaluation orders cannot agree better; the
# torus and the sphere at the workload's coupling are well conditioned.
@pytest.mark.parametrize("geom_name,tol_logr,tol_g,tol_stab", [("torus", 1e-10, 1e-9, 1e-9),
                                                               ("sphere_w", 1e-10, 1e-9, 1e-9),
                                                               ("sphere", 1e-6, 1e-5, 1e-4)])
def test_fp64_decision_identical_at_n120(qmc, oracle_results, geom_name, tol_logr, tol_g,
                                         tol_stab):
    geom = qmc.QMC_TORUS if geom_name == "torus" else qmc.QMC_SPHERE
    c = CASES[geom_name][1]
    g = _gpu(qmc, geom, c, 0)
    o = oracle_results(geom_name)
    tg, to = g.trace(0), o["trace"]
    assert len(tg) == len(to) == c["nsw"] * o["L"]
    assert np.array_equal(tg[:, 6], to[:, 6]), "accept decisions differ"
    assert (np.abs(tg[:, 2] - to[:, 2]) / np.maximum(1, np.abs(to[:, 2]))).max() < tol_logr
    assert _rel(g.green(0), o["green"]) < tol_g
    assert np.abs(g.fields(0) - o["phi"]).max() < 1e-9
    obs = g.series()[0]
    for col in (0, 1, 11, 12):
        ref = o["obs"][:, col]
        assert np.abs(obs[:, col] - ref).max() < tol_g * max(1, np.abs(ref).max())
    assert obs[:, 15].max() < tol_stab


@pytest.mark.parametrize("geom_name", ["torus", "sphere_w"])
def test_tensor_core_precision_tracks_the_oracle_at_n120(qmc, oracle_results, geom_name):
    geom = qmc.QMC_TORUS if geom_name == "torus" else qmc.QMC_SPHERE
    g = _gpu(qmc, geom, CASES[geom_name][1], 2)
    o = oracle_results(geom_name)
    tg, to = g.trace(0), o["trace"]
    mis = np.nonzero(tg[:, 6] != to[:, 6])[0]
    first = int(mis[0]) if len(mis) else len(tg)
    assert first >= 10, f"decisions diverge at update {first}"
    assert np.abs(tg[:first, 2] - to[:first, 2]).max() < 1e-5
    if first == len(tg):
        assert _rel(g.green(0), o["green"]) < 1e-6
    assert g.series()[0][:, 15].max() < 1e-8


# --------------------------------------------------------------- N = 280 ---
# The paper's largest torus, N_phi = 140 (N = 280, N_q = 1305), in the mixed
# precisions: FP32 Jacobi with its eigenvectors in global memory and FP64
# refinement, the cluster LU, QR with pivoting on global scratch, and in
# precision 2 the tensor-core products with their accumulators split along K.
# One sweep of whole-slice moves around N(0, 1) and one Langevin sweep of
# L = 3 slices against the FP64 oracle (without the records' energy column,
# whose all-momentum Wick sum costs the oracle ~8 minutes per record here):
# the decisions and G track the oracle.
BIG = dict(size=140, beta=0.3, u=1.0, anis=0.1, seed=3, n_stab=2, eps0=0.3, schedule="0P")


@pytest.fixture(scope="module")
def oracle_big():
    from oracle import oracle as O
    O.build()
    pool = mp.get_context("spawn").Pool(1)
    c = BIG
    job = pool.apply_async(R.plain_chain, (M.TORUS, c["size"], c["beta"], 0.1, c["u"], c["anis"],
                                           c["seed"], c["n_stab"], c["eps0"], 0),
                           dict(schedule=c["schedule"], energy=False))
    pool.close()
    yield job
    pool.terminate()


@pytest.mark.parametrize("precision", [1, 2])
def test_largest_torus_tracks_the_oracle(qmc, oracle_big, precision):
    c = BIG
    L = int(round(c["beta"] / 0.1))
    g = qmc.Chain(qmc.QMC_TORUS, c["size"], c["beta"], 0.1, c["u"], c["anis"], c["seed"],
                  n_stab=c["n_stab"], eps0=c["eps0"], precision=precision,
                  trace_capacity=len(c["schedule"]) * L)
    assert g.N == 280 and g.n_q == 1305
    for k in c["schedule"]:
        if k == "P":
            g.sweep(1)
        else:
            g.sweep_prior(1, 0.0)
    g.sync()
    o = oracle_big.get(timeout=3000)
    tg, to = g.trace(0), o["trace"]
    assert len(tg) == len(to) == len(c["schedule"]) * L
    assert np.array_equal(tg[:, 6], to[:, 6]), "accept decisions differ"
    assert 0 < to[:, 6].sum()
    assert np.abs(tg[:, 2] - to[:, 2]).max() < 1e-6
    assert _rel(g.green(0), o["green"]) < 1e-6
    assert np.abs(g.fields(0) - o["phi"]).max() < 1e-6
    obs = g.series()[0]
    for col in (0, 1, 11):
        ref = o["obs"][:, col]
        assert np.abs(obs[:, col] - ref).max() < 1e-6 * max(1, np.abs(ref).max())
    assert obs[:, 15].max() < 1e-8 and np.all(np.isfinite(obs[:, :13]))
