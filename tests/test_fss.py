"""Finite-size-scaling tools (paper_2605_03700_gb300.fss) on synthetic data
drawn from known scaling forms: the grid scan, its refinement and bootstrap,
the Delta_v fits and the crossing points must give back the exponents and the
critical coupling the data were generated with.

The generators write the scaling variable as N_phi^((3 - Delta_s)/2) times
(u - u_c)/u_c, independently of the module's sqrt form, so a wrong power of
N_phi (e.g. N_phi^(3 - Delta_s)) or a sign slip in u/u_c - 1 moves the
recovered Delta_s or u_c far outside the tolerances.
"""
import numpy as np
import pytest

from paper_2605_03700_gb300 import fss

UC, DS, DV = 0.163, 2.46, 0.53
SIZES = [15, 20, 27, 36, 45, 59]
US = np.linspace(0.075, 0.30, 10)


def _grid():
    u = np.repeat(US, len(SIZES))
    n = np.tile(np.asarray(SIZES, float), len(US))
    return u, n


def _x(u, n, uc=UC, ds=DS):
    return (u - uc) / uc * n ** ((3.0 - ds) / 2.0)


def _cubic(x):
    return 0.55 - 0.21 * x + 0.018 * x ** 2 + 0.004 * x ** 3


def _ratio(x):
    """a correlation-ratio-like F: 1 deep in the ordered phase (x << 0), 0
    in the disordered one"""
    return 1.0 / (1.0 + np.exp(1.3 * x))


def test_exact_cubic_collapses_perfectly_at_the_true_point():
    u, n = _grid()
    y = _cubic(_x(u, n))
    r2, coef = fss.collapse_r2(u, n, y, UC, DS)
    assert abs(1.0 - r2) < 1e-12
    assert np.allclose(coef, [0.004, 0.018, -0.21, 0.55], atol=1e-10)
    ucg = np.round(np.arange(0.140, 0.190, 0.001), 6)
    dsg = np.round(np.arange(2.20, 2.70, 0.01), 6)
    m, uc, ds, best = fss.grid_scan(u, n, y, ucg, dsg)
    assert m.shape == (len(ucg), len(dsg))
    assert abs(uc - UC) < 1e-9 and abs(ds - DS) < 1e-9 and abs(best - 1) < 1e-12
    # away from the truth the collapse is visibly worse
    assert fss.collapse_r2(u, n, y, 0.175, DS)[0] < 1 - 1e-4
    assert fss.collapse_r2(u, n, y, UC, 2.2)[0] < 1 - 1e-4


def test_r2_is_the_coefficient_of_determination():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(1)
    u, n = _grid()
    y = _ratio(_x(u, n)) + 0.02 * rng.standard_normal(len(u))
    r2, coef = fss.collapse_r2(u, n, y, 0.17, 2.3)
    x = (u - 0.17) / 0.17 * n ** 0.35
    assert abs(r2 - sk.r2_score(y, np.polyval(coef, x))) < 1e-12
    # the cubic is the least-squares one: perturbing a coefficient worsens R^2
    for k in range(4):
        c = coef.copy()
        c[k] += 1e-3
        assert sk.r2_score(y, np.polyval(c, x)) < r2


def test_noisy_ratio_recovers_uc_and_delta_s():
    """F a logistic curve (not a polynomial), 0.5% noise, the paper's window
    N_phi >= 15, u in [0.075, 0.30]; the fit keeps the points near u_c where
    the cubic is accurate."""
    rng = np.random.default_rng(2)
    u, n = _grid()
    err = np.full(len(u), 0.005)
    y = _ratio(_x(u, n)) + err * rng.standard_normal(len(u))
    us, ns, ys, es = fss.select(u, n, y, err, nphi_min=15, u_range=(0.12, 0.22))
    ucg, dsg = np.linspace(0.12, 0.22, 41), np.linspace(1.8, 3.0, 41)
    uc, ds, best = fss.refine_scan(us, ns, ys, ucg, dsg)
    assert abs(uc - UC) < 0.006 and abs(ds - DS) < 0.12, (uc, ds)
    assert best > 0.99
    m, _, _, _ = fss.grid_scan(us, ns, ys, ucg, dsg)
    reg = fss.r2_region(m, ucg, dsg, 0.99)
    assert reg[0][0] <= UC <= reg[0][1] and reg[1][0] <= DS <= reg[1][1]
    assert fss.r2_region(m, ucg, dsg, 1.01) is None
    muc, suc, mds, sds = fss.bootstrap_scan(us, ns, ys, es, np.linspace(0.14, 0.19, 26),
                                            np.linspace(2.1, 2.8, 36), n_boot=30, seed=3)
    assert 0 < suc < 0.01 and 0 < sds < 0.2
    assert abs(muc - UC) < 4 * suc + 0.002 and abs(mds - DS) < 4 * sds + 0.02


def test_order_parameter_ansatz():
    """m^2 = N_phi^-Delta_v F(x): at fixed Delta_v the collapse of
    m^2 N_phi^Delta_v recovers u_c and Delta_s; the fits of ln m^2 against
    ln N_phi give Delta_v at u_c whatever the smallest size kept."""
    u, n = _grid()
    F = lambda x: 0.08 * np.exp(-0.6 * x)
    m2 = n ** (-DV) * F(_x(u, n))
    y = fss.order_parameter_collapse_y(m2, n, DV)
    assert np.allclose(y, F(_x(u, n)), rtol=1e-13)
    us, ns, ys = fss.select(u, n, y, u_range=(0.12, 0.22))
    uc, ds, best = fss.refine_scan(us, ns, ys, np.linspace(0.12, 0.22, 41),
                                   np.linspace(1.8, 3.0, 41))
    assert abs(uc - UC) < 0.003 and abs(ds - DS) < 0.06, (uc, ds)
    # at u = u_c exactly
    nn = np.asarray(SIZES, float)
    fits = fss.power_law_dimension(nn, 0.08 * nn ** (-DV))
    assert [f[0] for f in fits] == SIZES[:-2]
    assert all(abs(f[1] - DV) < 1e-12 and f[2] < 1e-10 for f in fits)
    # deep in the ordered phase m^2 -> const: Delta_v falls as small sizes go
    m2o = 0.05 + 0.4 / nn
    dvs = [f[1] for f in fss.power_law_dimension(nn, m2o)]
    assert all(a > b for a, b in zip(dvs, dvs[1:])) and dvs[-1] < 0.5
    # weighted fit with errors: the standard error follows the errors
    rng = np.random.default_rng(4)
    e = 0.01 * 0.08 * nn ** (-DV)
    m2n = 0.08 * nn ** (-DV) + e * rng.standard_normal(len(nn))
    (nmin, dv, sdv), = fss.power_law_dimension(nn, m2n, e, nmin_list=[15])
    assert 0.001 < sdv < 0.05 and abs(dv - DV) < 4 * sdv


def test_crossings_bracket_uc():
    u, n = _grid()
    R = _ratio(_x(u, n))
    cr = fss.crossings(u, n, R)
    assert [(a, b) for a, b, _ in cr] == list(zip(map(float, SIZES[:-1]), map(float, SIZES[1:])))
    h = US[1] - US[0]
    assert all(abs(c - UC) < 0.25 * h for _, _, c in cr), cr
    # u_c on the grid: the curves meet exactly there
    ug = np.repeat(np.array([0.12, UC, 0.2]), 2)
    ng = np.tile([20.0, 27.0], 3)
    (_, _, c), = fss.crossings(ug, ng, _ratio(_x(ug, ng)))
    assert c == UC
    # shuffled input order does not matter
    p = np.random.default_rng(5).permutation(len(u))
    assert fss.crossings(u[p], n[p], R[p]) == cr
    # curves that never cross
    assert fss.crossings(ug, ng, ng / 100.0) == []


def test_mean_err():
    x = np.random.default_rng(6).standard_normal(10000)
    m, e = fss.mean_err(x)
    assert abs(e - 0.01) < 0.001 and abs(m) < 4 * e
    assert abs(fss.mean_err(x, tau=2.0)[1] - 2 * e) < 1e-12
