"""Parity of the CUDA sweep (libqmc, FP64) with the FP64 CPU oracle.

Same seeds, same Philox streams, same slice order: the two must make
identical accept/reject decisions, agree on every log determinant ratio to
1e-10 and on G to 1e-9 relative (max-norm over the matrix relative to
max|G|).  Cases span several GEMM tiles and ragged tails (N = 2 N_phi not a
multiple of 16, odd N_phi for the Jacobi ordering, L not a multiple of
n_stab), batches of chains with different couplings, the full matrix size of
the N_phi = 36 workload, and its full imaginary-time length on
size-independent properties.
"""

import numpy as np
import pytest

from oracle import model as M
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL_LOGR = 1e-10
TOL_G = 1e-9


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


def _compare_chain(gpu, c, orc, nsw, trace_gpu, trace_orc):
    assert len(trace_gpu) == len(trace_orc) == nsw * orc.L
    # identical decisions and per-update quantities
    assert np.array_equal(trace_gpu[:, 6], trace_orc[:, 6]), "accept decisions differ"
    assert np.array_equal(trace_gpu[:, :2], trace_orc[:, :2])
    assert np.abs(trace_gpu[:, 2] - trace_orc[:, 2]).max() < TOL_LOGR
    dA = np.abs(trace_gpu[:, 4] - trace_orc[:, 4]) / np.maximum(1, np.abs(trace_orc[:, 4]))
    assert dA.max() < 1e-8
    assert np.abs(trace_gpu[:, 5] - trace_orc[:, 5]).max() < 1e-12
    assert np.abs(trace_gpu[:, 7] - trace_orc[:, 7]).max() < 1e-12
    assert _rel(gpu.green(c), orc.green()) < TOL_G
    assert np.abs(gpu.fields(c) - orc.phi()).max() < 1e-9


def test_config1_ten_thousand_updates_decision_identical(qmc):
    """torus N_phi = 4 (N = 8, N_q = 37), beta = 2, dtau = 0.1, u = 1,
    seed 0, stabilise every 5 slices: 500 sweeps x 20 slices = 10^4 updates."""
    nsw = 500
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5, trace_capacity=nsw * 20)
    g.sweep(nsw)
    g.sync()
    o = O.Chain(M.TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5)
    o.enable_trace(nsw * 20)
    obs_o = o.sweep(nsw)
    _compare_chain(g, 0, o, nsw, g.trace(0), o.trace())
    obs_g = g.series()[0]
    assert obs_g.shape == obs_o.shape
    for col in (0, 1, 3, 6, 11, 12):
        assert np.abs(obs_g[:, col] - obs_o[:, col]).max() < 1e-9 * max(1, np.abs(obs_o[:, col]).max())
    assert np.array_equal(obs_g[:, 17], obs_o[:, 17])
    assert np.abs(obs_g[:, 14] - obs_o[:, 14]).max() < 1e-12
    assert obs_g[:, 15].max() < 1e-9 and obs_g[:, 16].max() < 1e-9


@pytest.mark.parametrize("nphi,beta,nstab", [(3, 1.3, 5), (5, 1.0, 4), (9, 0.8, 3)])
def test_ragged_sizes_parity(qmc, nphi, beta, nstab):
    nsw = 6
    L = int(round(beta / 0.1))
    g = qmc.Chain(qmc.QMC_TORUS, nphi, beta, 0.1, 1.5, 0.1, 7, n_stab=nstab, trace_capacity=nsw * L)
    g.sweep(nsw)
    g.sync()
    o = O.Chain(M.TORUS, nphi, beta, 0.1, 1.5, 0.1, 7, n_stab=nstab)
    o.enable_trace(nsw * L)
    o.sweep(nsw)
    _compare_chain(g, 0, o, nsw, g.trace(0), o.trace())


def test_batched_chains_with_different_couplings(qmc):
    us = [0.5, 1.2, 2.0]
    als = [0.0, 0.1, -0.15]
    seeds = [3, 11, 42]
    nsw = 20
    g = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, 0.0, 0, n_chains=3, couplings=us,
                  anisotropies=als, seeds=seeds, n_stab=5, trace_capacity=nsw * 10)
    g.sweep(nsw)
    g.sync()
    for c in range(3):
        o = O.Chain(M.TORUS, 4, 1.0, 0.1, us[c], als[c], seeds[c], n_stab=5)
        o.enable_trace(nsw * 10)
        o.sweep(nsw)
        _compare_chain(g, c, o, nsw, g.trace(c), o.trace())


def test_full_matrix_size_of_the_nphi36_workload(qmc):
    """N_phi = 36 (N = 72, N_q = 333, 1332 fields per slice), the matrix
    sizes the benchmark times, with a short imaginary-time axis the oracle
    finishes in seconds: beta = 0.4, L = 4, two chains, u in {0.5, 2.0}."""
    us = [0.5, 2.0]
    g = qmc.Chain(qmc.QMC_TORUS, 36, 0.4, 0.1, 0.0, 0.0, 0, n_chains=2, couplings=us,
                  seeds=[0, 1], n_stab=10, eps0=0.2, trace_capacity=8)
    g.sweep(2)
    g.sync()
    m = M.Model(M.TORUS, 36)
    for c in range(2):
        o = O.Chain(M.TORUS, 36, 0.4, 0.1, us[c], 0.0, c, n_stab=10, eps0=0.2, model=m)
        o.enable_trace(8)
        o.sweep(2)
        _compare_chain(g, c, o, 2, g.trace(c), o.trace())


def test_full_length_nphi36_properties(qmc):
    """The benchmark's workload itself (N_phi = 36, beta = 36, L = 360, eight
    couplings in [0.5, 2.0], stabilisation every 10 slices): properties that
    hold at any size -- sign-free ratios, G fresh to 1e-8 at every
    restabilisation, the full 4 N_phi Green's function equal to G (x) I_spin,
    finite observables with S^3 = S^4 = S^5."""
    us = np.linspace(0.5, 2.0, 8)
    g = qmc.Chain(qmc.QMC_TORUS, 36, 36.0, 0.1, 0.0, 0.0, 0, n_chains=8, couplings=us,
                  seeds=np.arange(8), n_stab=10, eps0=0.2)
    g.sweep(1)
    g.sync()
    s = g.series()
    assert s.shape == (8, 1, 20)
    assert s[:, :, 15].max() < 1e-8
    assert s[:, :, 16].max() < 1e-8
    assert np.all(np.isfinite(s))
    assert np.all(s[:, :, 3] == s[:, :, 4]) and np.all(s[:, :, 4] == s[:, :, 5])
    Gf = g.green(3, block=False)
    Gb = g.green(3)
    N = Gb.shape[0]
    assert np.array_equal(Gf[:N, :N], Gb) and np.array_equal(Gf[N:, N:], Gb)
    assert np.abs(Gf[:N, N:]).max() == 0 and np.abs(Gf[N:, :N]).max() == 0


def test_tau_int_matches_oracle_estimator(qmc):
    from oracle import analysis as A
    rng = np.random.default_rng(5)
    x = np.cumsum(rng.normal(size=3000)) * 0.01 + rng.normal(size=3000)
    assert abs(qmc.qmc_tau_int(x) - A.tau_int(x)) < 1e-9


def test_ratio_update_entry_point_matches_oracle(qmc):
    """qmc_ratio_update (det M and G M^-1 for a batch) against the oracle's
    brute-force-G ratio of a random proposal on three slices."""
    import torch
    ch = O.Chain(M.TORUS, 5, 1.0, 0.1, 2.0, 0.2, seed=4)
    rng = np.random.default_rng(8)
    Gs, Ds, refs = [], [], []
    for t in (2, 5, 9):
        G = ch.green_bruteforce(t)
        B, Bi = ch.B(t)
        E, tw = ch.factors(t)
        p0 = ch.phi()[t - 1].copy()
        p1 = p0 + 0.3 * rng.normal(size=p0.shape)
        logR, Gp = ch.ratio_at(t, p1)
        ch.set_slice_phi(t, p1)
        Bp, _ = ch.B(t)
        _, twp = ch.factors(t)
        ch.set_slice_phi(t, p0)
        Gs.append(G)
        Ds.append(Bp @ Bi)
        refs.append((logR + 0.5 * (twp - tw), Gp))
    N = Gs[0].shape[0]
    Gd = torch.tensor(np.array(Gs), dtype=torch.complex128, device="cuda")
    Dd = torch.tensor(np.array(Ds), dtype=torch.complex128, device="cuda")
    Gp = torch.empty_like(Gd)
    ld = torch.empty(3, dtype=torch.complex128, device="cuda")
    qmc.qmc_ratio_update(N, 3, Gd.data_ptr(), Dd.data_ptr(), Gp.data_ptr(), ld.data_ptr())
    Gp, ld = Gp.cpu().numpy(), ld.cpu().numpy()
    for b, (lr, gref) in enumerate(refs):
        assert abs(ld[b].real - lr.real) < TOL_LOGR
        assert abs(np.exp(1j * ld[b].imag) - np.exp(1j * lr.imag)) < 1e-9
        assert _rel(Gp[b], gref) < TOL_G


# ------------------------------------------------------------ mixed mode ---
# precision = 1: FP32 Jacobi sweeps with an FP64 polish, FP32 gradient
# transforms; everything in the MH ratio FP64.  The drift differs from the
# oracle's by FP32 rounding (~1e-7 relative), so proposals agree to ~1e-8 and
# ratios to ~1e-7; decisions agree except for a |log u - log A| below that.
TOL_MIXED_LOGR = 1e-5
TOL_MIXED_G = 1e-6


def _compare_mixed(gpu, c, orc, nsw, min_identical):
    tg, to = gpu.trace(c), orc.trace()
    assert len(tg) == len(to) == nsw * orc.L
    mis = np.nonzero(tg[:, 6] != to[:, 6])[0]
    first = int(mis[0]) if len(mis) else len(tg)
    assert first >= min_identical, f"decisions diverge at update {first}"
    assert np.abs(tg[:first, 2] - to[:first, 2]).max() < TOL_MIXED_LOGR
    assert np.abs(tg[:first, 3]).max() < 1e-8          # sign-free to FP64 rounding
    if first == len(tg):
        assert _rel(gpu.green(c), orc.green()) < TOL_MIXED_G
    return first


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_config1_tracks_the_oracle(qmc, precision):
    nsw = 200
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5, precision=precision,
                  trace_capacity=nsw * 20)
    g.sweep(nsw)
    g.sync()
    o = O.Chain(M.TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5)
    o.enable_trace(nsw * 20)
    o.sweep(nsw)
    assert _compare_mixed(g, 0, o, nsw, 2000) == nsw * 20
    s = g.series()[0]
    assert s[:, 15].max() < 1e-9 and s[:, 16].max() < 1e-9


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_nphi36_propagators_and_ratios(qmc, precision):
    """The benchmark's matrix size: propagators built through the FP32+polish
    eigensolver (and, in precision 2, tensor-core products) equal the
    oracle's (FP64 Jacobi) to 1e-10, the first updates make the oracle's
    decisions and G stays within 1e-6."""
    g = qmc.Chain(qmc.QMC_TORUS, 36, 0.4, 0.1, 2.0, 0.0, 0, n_stab=10, eps0=0.2,
                  precision=precision, trace_capacity=8)
    m = M.Model(M.TORUS, 36)
    o = O.Chain(M.TORUS, 36, 0.4, 0.1, 2.0, 0.0, 0, n_stab=10, eps0=0.2, model=m)
    for t in (1, 3):
        B, Bi = g.propagator(t)
        Bo, Boi = o.B(t)
        assert np.abs(B - Bo).max() < 1e-10 and np.abs(Bi - Boi).max() < 1e-10
    assert _rel(g.green(0), o.green()) < 1e-10
    g.sweep(2)
    g.sync()
    o.enable_trace(8)
    o.sweep(2)
    _compare_mixed(g, 0, o, 2, 8)


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_full_workload_properties(qmc, precision):
    us = np.linspace(0.5, 2.0, 8)
    g = qmc.Chain(qmc.QMC_TORUS, 36, 36.0, 0.1, 0.0, 0.0, 0, n_chains=8, couplings=us,
                  seeds=np.arange(8), n_stab=10, eps0=0.45, precision=precision)
    g.sweep(2)
    g.sync()
    s = g.series()
    assert s[:, :, 15].max() < 1e-8 and s[:, :, 16].max() < 1e-8
    assert np.all(np.isfinite(s))
    assert 0.2 < s[:, :, 13].mean() < 0.95


def test_ratio_update_in_a_fresh_process(qmc):
    """The context-free entry points must work in a process that never
    created a context (the kernels' shared-memory limits are set by the
    entry point itself)."""
    import os
    import subprocess
    import sys
    code = (
        "import ctypes as C, numpy as np, torch\n"
        "from paper_2605_03700_gb300 import qmc\n"
        "N, b = 72, 2\n"
        "r = np.random.default_rng(1)\n"
        "G = torch.tensor(0.5 * np.eye(N) + 0.01 * r.normal(size=(b, N, N)), dtype=torch.complex128, device='cuda')\n"
        "D = torch.tensor(np.eye(N) + 0.01 * r.normal(size=(b, N, N)), dtype=torch.complex128, device='cuda')\n"
        "for f in (qmc.lib().qmc_ratio_update, qmc.lib().qmc_ratio_update_noalloc):\n"
        "    Gp = torch.empty_like(G); ld = torch.empty(b, dtype=torch.complex128, device='cuda')\n"
        "    c = f(N, b, C.c_void_p(G.data_ptr()), C.c_void_p(D.data_ptr()), C.c_void_p(Gp.data_ptr()),\n"
        "          C.c_void_p(ld.data_ptr()), C.c_void_p(0))\n"
        "    torch.cuda.synchronize()\n"
        "    assert c == 0 and torch.isfinite(ld).all(), c\n"
        "print('ok')\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stderr[-2000:]
