"""Trotter convergence of the oracle's discretisation toward exact
diagonalisation (Methods, Eq. trotter_decomposition_methods and Eq.
hs_transform_methods).

The symmetric seven-factor split of the four channels is second order, but
the continuous HS step puts all 2 N_q Hermitian bilinears Q_q^i of a channel
into one exponential e^{alpha sum_q phi_q Q_q}.  For non-commuting Q_q
(projected densities do not commute) its Gaussian average differs from
e^{-dtau g sum_q Q_q^2 / 2} by O(alpha^4) = O(dtau^2) per slice, so the
total error is first order in dtau.  The lemma is checked by quadrature on
random matrices; the oracle's Monte Carlo averages against ED then show the
first-order approach (halving dtau halves the bias, a second-order error
would quarter it) and extrapolate to the exact values.
"""
import math
import os
from multiprocessing import get_context

import numpy as np
import scipy.linalg as sl

from oracle import ed as E
from oracle import model as M
from oracle import oracle as O

U, AL, BETA = 8.0, 0.3, 2.0
DTAUS = (0.5, 0.25, 0.125)
SEEDS = range(8)


def test_gaussian_average_of_a_noncommuting_exponential_is_off_at_fourth_order():
    rng = np.random.default_rng(0)
    A = []
    for _ in range(2):
        a = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        A.append((a + a.conj().T) / 2)
    x, w = np.polynomial.hermite_e.hermegauss(60)
    w = w / w.sum()
    errs = []
    for al in (0.1, 0.05, 0.025):
        avg = sum(wi * wj * sl.expm(al * (xi * A[0] + xj * A[1]))
                  for xi, wi in zip(x, w) for xj, wj in zip(x, w))
        errs.append(np.abs(avg - sl.expm(al ** 2 * (A[0] @ A[0] + A[1] @ A[1]) / 2)).max())
    # error / alpha^4 tends to a non-zero constant
    c = [e / al ** 4 for e, al in zip(errs, (0.1, 0.05, 0.025))]
    assert 1.0 < c[2] < 5.0 and abs(c[1] / c[2] - 1) < 0.05
    # commuting operators: the average is exact
    D = np.diag(rng.standard_normal(4))
    avg = sum(wi * wj * sl.expm(0.1 * (xi * D + xj * 2 * D)) for xi, wi in zip(x, w) for xj, wj in zip(x, w))
    assert np.abs(avg - sl.expm(0.01 * 5 * D @ D / 2)).max() < 1e-13


def _run(args):
    dt, seed = args
    ch = O.Chain(M.TORUS, 2, BETA, dt, U, AL, seed=seed, n_stab=2, n_adapt=150)
    ch.sweep(150)
    return dt, ch.sweep(4000)[:, [12, 0]].reshape(20, -1, 2).mean(1)


def test_first_order_approach_to_exact_diagonalisation():
    """Torus N_phi = 2, u = 8, alpha = 0.3, beta = 2; E and m^2 at
    dtau = 0.5, 0.25, 0.125 (8 chains x 4000 sweeps each)."""
    ref = E.ED(M.Model(M.TORUS, 2), M.couplings(U, AL), BETA).observables()
    jobs = [(dt, s) for dt in DTAUS for s in SEEDS]
    with get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(_run, jobs)
    for k, exact in ((0, ref["E"]), (1, ref["m2"])):
        dev, err = [], []
        for dt in DTAUS:
            b = np.concatenate([r for t, r in res if t == dt])[:, k]
            dev.append(b.mean() - exact)
            err.append(b.std(ddof=1) / math.sqrt(len(b)))
        # a clear discretisation bias at the coarsest step
        assert abs(dev[0]) > 10 * err[0], (k, dev, err)
        # halving dtau: ratio ~2 (first order), not 4 (second order)
        for i in (0, 1):
            r = dev[i] / dev[i + 1]
            er = abs(r) * math.hypot(err[i] / dev[i], err[i + 1] / dev[i + 1])
            assert 1.2 < r < 3.0 and (4.0 - r) > 3 * er, (k, i, r, er)
        # linear extrapolation of the two finest steps lands on ED
        ext = 2 * dev[2] - dev[1]
        assert abs(ext) < 4 * math.hypot(2 * err[2], err[1]), (k, ext)
