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
from tests.sphere_units import sphere_u

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


def test_absolute_form_for_an_anisotropy_scan():
    """Away from the SO(5) line the tuning parameter is alpha with alpha_c < 0:
    the (alpha - alpha_c) form recovers it, and at a non-zero critical value
    it gives exactly the relative form's R^2 (the factor is absorbed by F)."""
    al = np.repeat(np.linspace(-0.5, -0.1, 9), len(SIZES))
    n = np.tile(np.asarray(SIZES, float), 9)
    ac, ds = -0.29, 1.43
    y = _cubic((al - ac) * n ** ((3 - ds) / 2) * 3.0)
    m, a, d, best = fss.grid_scan(al, n, y, np.round(np.arange(-0.40, -0.20, 0.01), 6),
                                  np.round(np.arange(1.2, 1.7, 0.01), 6), relative=False)
    assert abs(a - ac) < 1e-9 and abs(d - ds) < 1e-9 and abs(best - 1) < 1e-12
    for trial in ((-0.25, 1.5), (-0.33, 1.3)):
        ra = fss.collapse_r2(al, n, y, *trial, relative=False)[0]
        rr = fss.collapse_r2(al, n, y, *trial, relative=True)[0]
        assert abs(ra - rr) < 1e-12


def _records(s0, sd):
    rec = np.zeros(s0.shape[:-1] + (20,))
    rec[..., 1:6], rec[..., 6:11] = s0, sd
    return rec


def test_order_parameters_from_records():
    rng = np.random.default_rng(7)
    s0 = rng.uniform(1, 3, (4, 5))
    sd = rng.uniform(0, 1, (4, 5))
    rec = _records(s0, sd)
    for ch, comp in (("SO5", [0, 1, 2, 3, 4]), ("VBS", [0, 1]), ("AFM", [2, 3, 4])):
        m2, R = fss.order_parameters(rec, 6, ch)
        for r in range(4):
            a = sum(s0[r, i] for i in comp)
            b = sum(sd[r, i] for i in comp)
            assert abs(m2[r] - a / (len(comp) * 36)) < 1e-15
            assert abs(R[r] - (1 - b / a)) < 1e-15
    # the SO(5) channel is the weighted mean of the VBS and AFM ones
    m5 = fss.order_parameters(rec, 6)[0]
    mv, ma = fss.order_parameters(rec, 6, "VBS")[0], fss.order_parameters(rec, 6, "AFM")[0]
    assert np.allclose(m5, (2 * mv + 3 * ma) / 5, rtol=1e-14)
    with pytest.raises(KeyError):
        fss.order_parameters(rec, 6, "XY")


def test_channels_against_the_oracle_chain_and_exact_diagonalisation():
    """Torus N_phi = 2, u = 4, alpha = 0.3, beta = 2: the SO(5) channel
    reproduces the sweep's own m^2 and R columns, and the VBS and AFM m^2 and
    R (ratio of means) agree with exact diagonalisation within 4 sigma.
    Sphere N_phi = 2, u = 79, alpha = -63 (strong coupling,
    tests/sphere_units.py; U_K > U_N): VBS order exceeds AFM order in both m^2
    and R, as exact diagonalisation says (S^1_0 = 0.0327 vs S^3_0 = 0.0285);
    a swapped channel assignment fails here.  (At N_phi = 2 the
    torus channels differ by < 1%, too little to tell them apart.)"""
    from oracle import ed as E
    from oracle import model as M
    from oracle import oracle as O
    m = M.Model(M.TORUS, 2)
    ref = E.ED(m, M.couplings(4.0, 0.3), 2.0).observables()
    ch = O.Chain(M.TORUS, 2, 2.0, 0.05, 4.0, 0.3, seed=11, n_stab=5, n_adapt=150, model=m)
    ch.sweep(150)
    obs = ch.sweep(2500)
    m2, R = fss.order_parameters(obs, 2)
    assert np.allclose(m2, obs[:, 0], rtol=1e-13) and np.allclose(R, obs[:, 11], rtol=1e-12)
    b = obs.reshape(25, -1, 20).mean(1)          # 25 bins of 100 sweeps
    for chn, comp in (("VBS", [0, 1]), ("AFM", [2, 3, 4])):
        s0, sd = ref["S0"][comp].sum(), ref["Sdq"][comp].sum()
        for k, (val, exact) in enumerate(((fss.order_parameters(b, 2, chn)[0], s0 / (len(comp) * 4)),
                                          (fss.order_parameters(b, 2, chn)[1], 1 - sd / s0))):
            mu, err = val.mean(), val.std(ddof=1) / 5
            assert abs(mu - exact) < 4 * err, (chn, k, mu, exact, err)

    m = M.Model(M.SPHERE, 2)
    us, als = sphere_u(1.0, 2), sphere_u(-0.8, 2)
    ref = E.ED(m, M.couplings(us, als), 2.0).observables()
    assert ref["S0"][0] > 1.1 * ref["S0"][2]
    assert ref["Sdq"][0] / ref["S0"][0] < ref["Sdq"][2] / ref["S0"][2]
    ch = O.Chain(M.SPHERE, 2, 2.0, 0.1, us, als, seed=2, n_stab=5, n_adapt=150, model=m)
    ch.sweep(150)
    b = ch.sweep(2000).reshape(20, -1, 20).mean(1)
    mv, Rv = fss.order_parameters(b, 2, "VBS")
    ma, Ra = fss.order_parameters(b, 2, "AFM")
    for d in (mv - ma, Rv - Ra):
        assert d.mean() > 3 * d.std(ddof=1) / np.sqrt(20)


def test_gap_fits_on_synthetic_correlations():
    tau = np.arange(0, 10.01, 0.25)
    C = 2.0 * np.exp(-0.7 * tau) + 0.5 * np.exp(-3.0 * tau)
    mid, de = fss.effective_gap(tau, C)
    assert de[0] > 1.0 and abs(de[-1] - 0.7) < 1e-9          # plateau at the gap
    d, e, a = fss.fit_gap(tau, C, tmin=5)
    assert abs(d - 0.7) < 1e-6 and abs(a - 2.0) < 1e-5
    # finite temperature: the periodic form
    beta = 12.0
    Cb = 2.0 * (np.exp(-0.7 * tau) + np.exp(-0.7 * (beta - tau)))
    d, e, a = fss.fit_gap(tau, Cb, tmin=2, tmax=10, beta=beta)
    assert abs(d - 0.7) < 1e-8 and abs(a - 2.0) < 1e-7
    assert abs(fss.fit_gap(tau, Cb, tmin=2, tmax=10)[0] - 0.7) > 0.05   # the plain exponential is biased
    # noisy data: the error covers the truth
    rng = np.random.default_rng(8)
    err = 0.01 * C
    Cn = C + err * rng.standard_normal(len(C))
    d, e, _ = fss.fit_gap(tau, Cn, err, tmin=4)
    assert 0 < e < 0.05 and abs(d - 0.7) < 4 * e
    with pytest.raises(ValueError):
        fss.fit_gap(tau, -C, tmin=4)


def test_dynamical_exponent():
    n = np.array([8.0, 12, 16, 24, 32])
    z, ez, c = fss.dynamical_exponent(n, 3.0 * n ** -0.5)
    assert abs(z - 1.0) < 1e-12 and abs(c - np.log(3.0)) < 1e-12 and ez < 1e-10
    z, _, _ = fss.dynamical_exponent(n, 3.0 * n ** -1.0)
    assert abs(z - 2.0) < 1e-12
    rng = np.random.default_rng(9)
    g = 3.0 * n ** -0.5 * (1 + 0.02 * rng.standard_normal(len(n)))
    z, ez, _ = fss.dynamical_exponent(n, g, 0.02 * g)
    assert 0.02 < ez < 0.5 and abs(z - 1.0) < 4 * ez


def test_gap_fit_against_the_exact_spectrum():
    """Torus N_phi = 2, u = 15 (deep in the disordered phase, the coupling of
    the paper's dynamics measurement), beta = 40: the decay rate fitted to
    the exact S^i_0(tau) equals the lowest excitation energy that n^{Gamma^i}_0
    reaches from the ground state (ED spectrum)."""
    from oracle import ed as E
    from oracle import model as M
    m = M.Model(M.TORUS, 2)
    ed = E.ED(m, M.couplings(15.0, 0.0), 40.0)
    q0 = m.q0()
    taus = np.arange(0.0, 10.5, 1.0)      # S(tau) >= 1e-6 S(0): ED is exact there
    for gi in (0, 2):
        S = np.array([ed.structure_factor_tau(gi, q0, t) for t in taus])
        d, e, _ = fss.fit_gap(taus, S, tmin=3, beta=40.0)
        assert abs(d - ed.gap(gi, q0)) < 1e-8, (gi, d, ed.gap(gi, q0))
        assert 0.9 < d < 1.2


def test_jackknife_errors():
    """Independent samples: the jackknife error of a mean equals the
    standard error; for a ratio of means it matches the delta-method error,
    and the estimate of a nonlinear function is bias-corrected."""
    rng = np.random.default_rng(10)
    n = 20000
    x = rng.normal(3.0, 1.0, n)
    y = rng.normal(2.0, 0.5, n)
    rec = np.stack([x, y], axis=1)
    est, err = fss.jackknife(rec, lambda r: r[0], nbins=50)
    assert abs(est - x.mean()) < 1e-12 and abs(err / (x.std() / np.sqrt(n)) - 1) < 0.3
    est, err = fss.jackknife(rec, lambda r: r[1] / r[0], nbins=50)
    delta = (2.0 / 3.0) * np.sqrt((0.5 / 2.0) ** 2 + (1.0 / 3.0) ** 2) / np.sqrt(n)
    assert abs(est - 2.0 / 3.0) < 4 * delta and abs(err / delta - 1) < 0.3
    # bias correction: E[1/mean] over small samples
    small = rng.normal(1.0, 0.5, (400, 10))
    naive = np.mean([1.0 / s.mean() for s in small])
    jk = np.mean([fss.jackknife(s[:, None], lambda r: 1.0 / r[0], nbins=10)[0] for s in small])
    assert abs(jk - 1.0) < abs(naive - 1.0)
    with pytest.raises(ValueError):
        fss.jackknife(rec[:1], lambda r: r[0], nbins=2)


def test_order_parameter_errors_on_records():
    rng = np.random.default_rng(11)
    s0 = rng.uniform(1, 3, (2000, 5))
    sd = rng.uniform(0, 1, (2000, 5))
    rec = np.zeros((2000, 20))
    rec[:, 1:6], rec[:, 6:11] = s0, sd
    m2, em2, R, eR = fss.order_parameter_errors(rec, 6)
    assert abs(m2 - s0.sum(1).mean() / (5 * 36)) < 1e-12
    assert 0 < em2 < 0.01 and 0 < eR < 0.01
    # the ratio of means, up to the O(1/n) bias correction
    assert abs(R - (1 - sd.sum(1).mean() / s0.sum(1).mean())) < 0.05 * eR
