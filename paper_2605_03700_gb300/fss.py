"""Finite-size-scaling analysis of measured observables (host post-processing
of the records the sweep produces; not part of the sweep).

Implements the paper's analysis along the SO(5) line (Results, "Finite-size
scaling"):

* scaling variable x = (u/u_c - 1) * sqrt(N_phi)^(3 - Delta_s) (Eq.
  finite-size-scaling-R); the correlation ratio obeys R = F(x) and the order
  parameter m^2 N_phi^Delta_v = F(x) (Eq. finite-size-scaling-m), with F a
  universal function;
* R^2-optimised grid scan: F approximated by a polynomial of third order
  around u_c, fitted by least squares for every (u_c, Delta_s) on a grid; the
  collapse quality is the coefficient of determination
  R^2 = 1 - sum (y - F(x))^2 / sum (y - mean y)^2, and the best grid point is
  the estimate;
* Delta_v from the slope of ln m^2 against ln N_phi, with the smallest sizes
  progressively excluded from the fit;
* crossing points of the curves of consecutive sizes, for R and for
  m^2 N_phi^Delta_v (Supplementary Note 3, data scaling analysis);
* the same scans in the anisotropy alpha for the VBS and AFM ratios away
  from the SO(5) line (Results, "Phase boundaries away from the
  SO(5)-symmetric line"; Supplementary Note 1);
* the SO(5) gap from the tail of the imaginary-time correlation and the
  dynamical exponent z from its size dependence (Supplementary Note 2).

Inputs are per-(u, N_phi) means of the observable records (Chain.series()),
with errors from order_parameter_errors (jackknife over bins) or mean_err;
everything is numpy on the host.
"""
from __future__ import annotations

import numpy as np


def mean_err(x, tau=0.5):
    """Mean of a Markov-chain series and its error sqrt(2 tau var / n), tau
    the integrated autocorrelation time (0.5 for independent samples)."""
    x = np.asarray(x, dtype=float)
    return float(x.mean()), float(np.sqrt(2.0 * tau * x.var(ddof=1) / len(x)))


# SO(5) components of an observable record: 1, 2 couple to U_K (valley,
# Kekule VBS order), 3, 4, 5 to U_N (spin, Neel AFM order) (Model, Eq.
# newmodel with U_1 = U_2 = U_K, U_3 = U_4 = U_5 = U_N).
CHANNELS = {"SO5": (0, 1, 2, 3, 4), "VBS": (0, 1), "AFM": (2, 3, 4)}


def order_parameters(records, nphi, channel="SO5"):
    """m^2 and the correlation ratio R of one order parameter from observable
    records (last axis the 20-double record: 1..5 S^i_{q=0}, 6..10 S^i at the
    smallest non-zero momenta):
    m^2_X = sum_{i in X} S^i_0 / (|X| N_phi^2) and R_X = 1 - S_X(dq)/S_X(0),
    S_X = sum_{i in X} S^i (Results: m^2_SO(5), the correlation ratio; the
    VBS and AFM ratios of the anisotropy scans use the subsets).  Pass the
    mean record to get R as the ratio of expectation values."""
    rec = np.asarray(records, dtype=float)
    comp = np.asarray(CHANNELS[channel])
    s0 = rec[..., 1 + comp].sum(-1)
    sd = rec[..., 6 + comp].sum(-1)
    return s0 / (len(comp) * float(nphi) ** 2), 1.0 - sd / s0


def scaling_x(u, nphi, uc, ds, relative=True):
    """x = (u/u_c - 1) sqrt(N_phi)^(3 - Delta_s) (relative, the SO(5)-line
    form), or (u - u_c) sqrt(N_phi)^(3 - Delta_s) for a tuning parameter whose
    critical value may be zero or negative (the anisotropy alpha); the two
    differ by the factor u_c, which a polynomial F absorbs, so at u_c != 0
    both give the same collapse."""
    u = np.asarray(u, dtype=float)
    nphi = np.asarray(nphi, dtype=float)
    d = u / uc - 1.0 if relative else u - uc
    return d * np.sqrt(nphi) ** (3.0 - ds)


def collapse_r2(u, nphi, y, uc, ds, order=3, relative=True):
    """Coefficient of determination of the polynomial collapse of y(u, N_phi)
    onto F(x) at the trial (u_c, Delta_s); returns (R^2, polynomial coeffs)."""
    y = np.asarray(y, dtype=float)
    x = scaling_x(u, nphi, uc, ds, relative)
    coef = np.polyfit(x, y, order)
    res = y - np.polyval(coef, x)
    tot = y - y.mean()
    return 1.0 - float(res @ res) / float(tot @ tot), coef


def grid_scan(u, nphi, y, uc_grid, ds_grid, order=3, relative=True):
    """R^2 map over the (u_c, Delta_s) grid and its maximum:
    returns (r2[len(uc_grid), len(ds_grid)], best_uc, best_ds, best_r2)."""
    r2 = np.full((len(uc_grid), len(ds_grid)), -np.inf)
    for i, uc in enumerate(uc_grid):
        for j, ds in enumerate(ds_grid):
            r2[i, j] = collapse_r2(u, nphi, y, uc, ds, order, relative)[0]
    i, j = np.unravel_index(np.argmax(r2), r2.shape)
    return r2, float(uc_grid[i]), float(ds_grid[j]), float(r2[i, j])


def order_parameter_collapse_y(m2, nphi, dv):
    """y = m^2 N_phi^Delta_v, the left-hand side of the order-parameter
    ansatz, for use with collapse_r2 / grid_scan at fixed Delta_v."""
    return np.asarray(m2, dtype=float) * np.asarray(nphi, dtype=float) ** dv


def power_law_dimension(nphi, m2, err=None, nmin_list=None):
    """Delta_v from weighted linear fits of ln m^2 against ln N_phi over the
    sizes N_phi >= N_min, for every N_min in nmin_list (default: every size
    that leaves at least three points).  Returns a list of
    (N_min, Delta_v, standard error)."""
    nphi = np.asarray(nphi, dtype=float)
    m2 = np.asarray(m2, dtype=float)
    sig = np.ones_like(m2) if err is None else np.asarray(err, dtype=float) / m2
    sizes = np.unique(nphi)
    if nmin_list is None:
        nmin_list = sizes[:-2]
    out = []
    for nmin in nmin_list:
        k = nphi >= nmin
        if k.sum() < 3:
            continue
        X = np.vstack([np.ones(k.sum()), np.log(nphi[k])]).T
        w = 1.0 / sig[k] ** 2
        A = X.T @ (X * w[:, None])
        b = X.T @ (w * np.log(m2[k]))
        beta = np.linalg.solve(A, b)
        cov = np.linalg.inv(A)
        if err is None:   # unit weights: scale by the residual variance
            r = np.log(m2[k]) - X @ beta
            cov = cov * (r @ r) / max(k.sum() - 2, 1)
        out.append((float(nmin), float(-beta[1]), float(np.sqrt(cov[1, 1]))))
    return out


def crossings(u, nphi, R):
    """u where the curves R(u) of consecutive sizes cross (R a correlation
    ratio, or m^2 N_phi^Delta_v; linear interpolation of their difference on
    the common u grid): a list of (N_phi_1, N_phi_2, u_cross); pairs that do
    not cross are skipped."""
    u = np.asarray(u, dtype=float)
    nphi = np.asarray(nphi, dtype=float)
    R = np.asarray(R, dtype=float)
    sizes = np.unique(nphi)
    out = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        ia, ib = nphi == a, nphi == b
        oa, ob = np.argsort(u[ia]), np.argsort(u[ib])
        ua, ra = u[ia][oa], R[ia][oa]
        ub, rb = u[ib][ob], R[ib][ob]
        grid = np.intersect1d(ua, ub)
        if len(grid) < 2:
            continue
        d = np.interp(grid, ub, rb) - np.interp(grid, ua, ra)
        s = np.nonzero((d[:-1] == 0) | (np.sign(d[:-1]) * np.sign(d[1:]) < 0))[0]
        if len(s) == 0:
            continue
        i = s[0]
        uc = grid[i] if d[i] == 0 else grid[i] - d[i] * (grid[i + 1] - grid[i]) / (d[i + 1] - d[i])
        out.append((float(a), float(b), float(uc)))
    return out


def r2_region(r2, uc_grid, ds_grid, threshold=0.99):
    """Ranges of u_c and Delta_s over the grid points whose collapse has
    R^2 > threshold: ((uc_min, uc_max), (ds_min, ds_max)), or None when no
    point passes."""
    i, j = np.nonzero(np.asarray(r2) > threshold)
    if len(i) == 0:
        return None
    uc, ds = np.asarray(uc_grid)[i], np.asarray(ds_grid)[j]
    return (float(uc.min()), float(uc.max())), (float(ds.min()), float(ds.max()))


def refine_scan(u, nphi, y, uc_grid, ds_grid, levels=2, shrink=5, order=3, relative=True):
    """grid_scan, then `levels` further scans on grids of the same size
    centred on the best point and `shrink` times narrower; returns
    (best_uc, best_ds, best_r2)."""
    uc_grid, ds_grid = np.asarray(uc_grid, float), np.asarray(ds_grid, float)
    _, uc, ds, r = grid_scan(u, nphi, y, uc_grid, ds_grid, order, relative)
    for _ in range(levels):
        huc = (uc_grid[-1] - uc_grid[0]) / (2 * shrink)
        hds = (ds_grid[-1] - ds_grid[0]) / (2 * shrink)
        uc_grid = np.linspace(uc - huc, uc + huc, len(uc_grid))
        ds_grid = np.linspace(ds - hds, ds + hds, len(ds_grid))
        _, uc, ds, r = grid_scan(u, nphi, y, uc_grid, ds_grid, order, relative)
    return uc, ds, r


def bootstrap_scan(u, nphi, y, err, uc_grid, ds_grid, n_boot=100, seed=0, order=3,
                   relative=True):
    """Statistical error of the grid-scan estimate: rescan n_boot synthetic
    data sets y + err * N(0, 1) (Gaussian resampling of the means within
    their errors).  Returns (mean u_c, std u_c, mean Delta_s, std Delta_s)."""
    rng = np.random.default_rng(seed)
    y, err = np.asarray(y, float), np.asarray(err, float)
    best = []
    for _ in range(n_boot):
        yb = y + err * rng.standard_normal(len(y))
        best.append(grid_scan(u, nphi, yb, uc_grid, ds_grid, order, relative)[1:3])
    best = np.array(best)
    return (float(best[:, 0].mean()), float(best[:, 0].std(ddof=1)),
            float(best[:, 1].mean()), float(best[:, 1].std(ddof=1)))


def select(u, nphi, *cols, nphi_min=None, u_range=None):
    """Restrict the data to the critical window used in the fits
    (N_phi >= nphi_min, u_range[0] <= u <= u_range[1])."""
    u, nphi = np.asarray(u, float), np.asarray(nphi, float)
    k = np.ones(len(u), dtype=bool)
    if nphi_min is not None:
        k &= nphi >= nphi_min
    if u_range is not None:
        k &= (u >= u_range[0]) & (u <= u_range[1])
    return (u[k], nphi[k]) + tuple(np.asarray(c, float)[k] for c in cols)


# ------------------------------------------------- gap and dynamics --------
# Supplementary Note 2: the imaginary-time SO(5) correlation
# m^2(tau, q=0) = (1/5) sum_i <n_0^{Gamma^i}(tau) n_0^{Gamma^i}(0)> decays as
# e^{-Delta tau} at long times; Delta ~ sqrt(N_phi)^-z gives the dynamical
# exponent z from ln Delta = z ln(1/sqrt(N_phi)) + C.

def effective_gap(tau, C):
    """-d ln C / d tau between consecutive points: (tau midpoints, Delta_eff);
    a plateau marks the range where one exponential dominates."""
    tau = np.asarray(tau, dtype=float)
    C = np.asarray(C, dtype=float)
    return 0.5 * (tau[1:] + tau[:-1]), -np.diff(np.log(C)) / np.diff(tau)


def fit_gap(tau, C, err=None, tmin=None, tmax=None, beta=None):
    """Gap from the long-time tail of a correlation function over
    tmin <= tau <= tmax: without beta, the exponential A e^{-Delta tau}
    (weighted linear fit of ln C); with beta, the periodic form
    A (e^{-Delta tau} + e^{-Delta (beta - tau)}) of a finite-temperature
    correlation (nonlinear least squares started from the exponential fit).
    Returns (Delta, standard error, A)."""
    tau = np.asarray(tau, dtype=float)
    C = np.asarray(C, dtype=float)
    sig = np.full(len(C), 1.0) if err is None else np.asarray(err, dtype=float)
    k = np.ones(len(tau), dtype=bool)
    if tmin is not None:
        k &= tau >= tmin
    if tmax is not None:
        k &= tau <= tmax
    t, c, s = tau[k], C[k], sig[k]
    if len(t) < 3 or np.any(c <= 0):
        raise ValueError("need at least three positive points in the window")
    # ln C has error err / C; without errors, equal weights in ln C
    w = np.ones(len(c)) if err is None else (c / s) ** 2
    X = np.vstack([np.ones(len(t)), -t]).T
    A = X.T @ (X * w[:, None])
    beta_ = np.linalg.solve(A, X.T @ (w * np.log(c)))
    cov = np.linalg.inv(A)
    if err is None:
        r = np.log(c) - X @ beta_
        cov = cov * (r @ r) / max(len(t) - 2, 1)
    gap, amp = float(beta_[1]), float(np.exp(beta_[0]))
    egap = float(np.sqrt(cov[1, 1]))
    if beta is None:
        return gap, egap, amp
    from scipy.optimize import curve_fit

    def f(x, a, d):
        return a * (np.exp(-d * x) + np.exp(-d * (beta - x)))
    # start from the decay of the first half of the window (before the
    # periodic image turns the curve up)
    h = t <= 0.5 * beta
    d0 = -np.polyfit(t[h], np.log(c[h]), 1)[0] if h.sum() >= 2 else 0.0
    d0 = d0 if d0 > 0 else 1.0 / beta
    a0 = float(c[0] / (np.exp(-d0 * t[0]) + np.exp(-d0 * (beta - t[0]))))
    p, pc = curve_fit(f, t, c, p0=[a0, d0], sigma=s, absolute_sigma=err is not None,
                      bounds=([0.0, 0.0], [np.inf, np.inf]))
    return float(p[1]), float(np.sqrt(pc[1, 1])), float(p[0])


def dynamical_exponent(nphi, gap, err=None):
    """z and C of ln Delta = z ln(1/sqrt(N_phi)) + C (weighted by the gaps'
    errors when given): returns (z, standard error, C)."""
    nphi = np.asarray(nphi, dtype=float)
    gap = np.asarray(gap, dtype=float)
    x = np.log(1.0 / np.sqrt(nphi))
    sig = np.ones(len(gap)) if err is None else np.asarray(err, dtype=float) / gap
    w = 1.0 / sig ** 2
    X = np.vstack([np.ones(len(x)), x]).T
    A = X.T @ (X * w[:, None])
    b = np.linalg.solve(A, X.T @ (w * np.log(gap)))
    cov = np.linalg.inv(A)
    if err is None:
        r = np.log(gap) - X @ b
        cov = cov * (r @ r) / max(len(x) - 2, 1)
    return float(b[1]), float(np.sqrt(cov[1, 1])), float(b[0])


# ---------------------------------------------------- errors of ratios -----
def jackknife(records, fn, nbins=20):
    """Jackknife mean and error of fn(mean record) over a Markov-chain series
    of records (first axis: sweeps), with the series cut into nbins
    consecutive bins (longer than the autocorrelation time): fn sees the
    mean of all bins but one.  Returns (estimate, error), each shaped like
    fn's value; the estimate is bias-corrected to O(1/nbins^2)."""
    rec = np.asarray(records, dtype=float)
    nb = int(nbins)
    if nb < 2 or len(rec) < nb:
        raise ValueError("need at least two bins with one record each")
    m = len(rec) // nb
    bins = rec[: m * nb].reshape((nb, m) + rec.shape[1:]).mean(axis=1)
    total = bins.sum(axis=0)
    full = np.asarray(fn(total / nb), dtype=float)
    loo = np.array([fn((total - bins[k]) / (nb - 1)) for k in range(nb)], dtype=float)
    mean_loo = loo.mean(axis=0)
    err = np.sqrt((nb - 1) / nb * ((loo - mean_loo) ** 2).sum(axis=0))
    return nb * full - (nb - 1) * mean_loo, err


def order_parameter_errors(records, nphi, channel="SO5", nbins=20):
    """(m^2, error, R, error) of one channel from a series of observable
    records, R taken as the ratio of the means (jackknife errors)."""
    (m2, R), (em2, eR) = jackknife(records, lambda r: order_parameters(r, nphi, channel), nbins)
    return float(m2), float(em2), float(R), float(eR)
