"""Pins of the oracle's slice and drift variants (the single-exponential
slice, independent half-factor fields, the first-order drift) against
things other than the oracle: Fock-space traces built from the model tables,
finite differences, and exact diagonalisation.

The default discretisation (seven factors with shared fields, exact drift)
is pinned in test_oracle_pins.py and test_oracle_stat.py.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ed as E
from oracle import model as M
from oracle import oracle as O
from tests.test_oracle_pins import _bilinear, _jw
from tests.sphere_units import sphere_u

OV = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
ORDER = [(0, .5), (1, .5), (2, .5), (3, 1.0), (2, .5), (1, .5), (0, .5)]


def _exponents(m, phi_t, kind, dtau, g):
    """[(X, is_channel_0)] of one slice, from the model tables"""
    alpha = M.hs_alpha(g, dtau)

    def H(i, ph):
        z = M.z_from_phi(m, ph)
        return np.kron(OV[i], sum(z[q] * m.dense_F(q) for q in range(m.nq)))
    if kind == O.SLICE_SINGLE:
        W = [alpha[i] * H(i, phi_t[i]) for i in range(4)]
        return [(sum(W), None, W[0])]
    out = []
    for j, (i, c) in enumerate(ORDER):
        a = np.sqrt(complex(-c * dtau * g[i])) if kind == O.SLICE_INDEP else c * alpha[i]
        X = a * H(i, phi_t[j] if kind == O.SLICE_INDEP else phi_t[i])
        out.append((X, i, X if i == 0 else None))
    return out


def _fock_log_bracket(ch, m, kind, dtau, g):
    cs = _jw(m.N)
    phi = ch.phi()
    U = np.eye(2 ** m.N, dtype=complex)
    bg = 0
    for t in range(ch.L):
        Bt = np.eye(2 ** m.N, dtype=complex)
        for X, _, X0 in _exponents(m, phi[t], kind, dtau, g):
            Bt = Bt @ sla.expm(_bilinear(cs, X))
            if X0 is not None:
                bg += -0.5 * np.trace(X0)
        U = Bt @ U
    return np.log(np.trace(U)) + bg


@pytest.mark.parametrize("kind", [O.SLICE_SINGLE, O.SLICE_INDEP])
@pytest.mark.parametrize("u,al", [(1.0, 0.0), (3.0, 0.2)])
def test_determinant_equals_fock_trace_and_is_real(kind, u, al):
    m = M.Model(M.TORUS, 2)
    ch = O.Chain(M.TORUS, 2, 0.3, 0.1, u, al, seed=5, model=m, slice_kind=kind)
    assert ch.phi().shape == (3, 7 if kind == O.SLICE_INDEP else 4, m.nq)
    assert len(ch.factors(1)[0]) == (1 if kind == O.SLICE_SINGLE else 7)
    lb = ch.log_bracket()
    ref = _fock_log_bracket(ch, m, kind, 0.1, M.couplings(u, al))
    assert abs(lb.real - ref.real) < 1e-10
    assert abs(math.sin(lb.imag)) < 1e-10
    assert abs(math.sin(ref.imag)) < 1e-10


@pytest.mark.parametrize("kind", [O.SLICE_SINGLE, O.SLICE_INDEP])
@pytest.mark.parametrize("geom,size,u,al", [(M.TORUS, 4, 5.0, 0.3), (M.SPHERE, 3, sphere_u(1.0, 3), sphere_u(0.1, 3))])
def test_variants_are_sign_free_on_random_fields(kind, geom, size, u, al):
    for seed in range(3):
        ch = O.Chain(geom, size, 1.0, 0.1, u, al, seed=seed, slice_kind=kind)
        assert abs(math.sin(ch.log_bracket().imag)) < 1e-9


def _action(ch):
    return 0.5 * np.sum(ch.phi() ** 2) - 2 * ch.log_bracket().real


@pytest.mark.parametrize("kind", [O.SLICE_SINGLE, O.SLICE_INDEP])
@pytest.mark.parametrize("geom,size,u,al,t", [(M.TORUS, 2, 2.0, 0.3, 2), (M.SPHERE, 2, sphere_u(1.0, 2), sphere_u(0.2, 2), 1)])
def test_exact_drift_matches_finite_differences(kind, geom, size, u, al, t):
    ch = O.Chain(geom, size, 0.5, 0.1, u, al, seed=11, slice_kind=kind)
    g = ch.gradient(t)
    p0 = ch.phi()[t - 1].copy()
    h = 1e-5
    fd = np.zeros_like(g)
    for k in range(p0.shape[0]):
        for r in range(ch.nq):
            p = p0.copy(); p[k, r] += h; ch.set_slice_phi(t, p); sp = _action(ch)
            p = p0.copy(); p[k, r] -= h; ch.set_slice_phi(t, p); sm = _action(ch)
            fd[k, r] = (sp - sm) / (2 * h)
    ch.set_slice_phi(t, p0)
    assert np.abs(fd - g).max() < 1e-6 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("kind", [O.SLICE_SYM, O.SLICE_SINGLE, O.SLICE_INDEP])
def test_first_order_drift(kind):
    """The first-order drift is phi - 2 dF/dphi with the linear functional
    F = Re[sum_j Tr((1-G) X_j) - 1/2 sum_{channel-0 j} Tr X_j] at fixed G
    (X_j from the model tables), and it approaches the exact drift as
    dtau -> 0: the difference of the fermion forces, relative to the force,
    falls like sqrt(dtau)."""
    m = M.Model(M.TORUS, 2)
    u, al, t = 2.0, 0.3, 2
    rel = []
    for dtau in (0.1, 0.025):
        ex = O.Chain(M.TORUS, 2, 4 * dtau, dtau, u, al, seed=3, model=m, slice_kind=kind)
        fo = O.Chain(M.TORUS, 2, 4 * dtau, dtau, u, al, seed=3, model=m, slice_kind=kind,
                     drift_kind=O.DRIFT_FIRST)
        phi = fo.phi()[t - 1]
        G = fo.green_bruteforce(t)
        A = np.eye(m.N) - G

        def F(ph):
            s = 0.0
            for X, _, X0 in _exponents(m, ph, kind, dtau, M.couplings(u, al)):
                s += np.trace(A @ X)
                if X0 is not None:
                    s -= 0.5 * np.trace(X0)
            return s.real
        ref = np.zeros_like(phi)
        h = 1e-3                       # F is linear in phi: differences are exact
        for k in range(phi.shape[0]):
            for r in range(m.nq):
                p = phi.copy(); p[k, r] += h; fp = F(p)
                p = phi.copy(); p[k, r] -= h; fm = F(p)
                ref[k, r] = phi[k, r] - 2 * (fp - fm) / (2 * h)
        gf = fo.gradient(t)
        assert np.abs(gf - ref).max() < 1e-9 * max(1.0, np.abs(gf).max())
        ge = ex.gradient(t)
        rel.append(np.abs(gf - ge).max() / np.abs(ge - phi).max())
    assert rel[0] > 1e-3
    assert 1.4 < rel[0] / rel[1] < 2.8, rel


def _mean_err(x, nb=25):
    b = np.asarray(x)[: len(x) // nb * nb].reshape(nb, -1).mean(1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


@pytest.mark.parametrize("kind,drift", [(O.SLICE_SYM, O.DRIFT_FIRST), (O.SLICE_SINGLE, O.DRIFT_EXACT),
                                        (O.SLICE_INDEP, O.DRIFT_EXACT)])
def test_variant_chains_match_exact_diagonalisation(kind, drift):
    """Torus N_phi = 2, u = 4, alpha = 0.3, beta = 2, dtau = 0.05: E, m^2,
    S^1_0 and S^3_0 within 4 sigma of ED; the weight stays sign-free."""
    m = M.Model(M.TORUS, 2)
    ref = E.ED(m, M.couplings(4.0, 0.3), 2.0).observables()
    ch = O.Chain(M.TORUS, 2, 2.0, 0.05, 4.0, 0.3, seed=1, n_stab=5, n_adapt=150, model=m,
                 slice_kind=kind, drift_kind=drift)
    ch.sweep(150)
    obs = ch.sweep(2500)
    for col, r in ((12, ref["E"]), (0, ref["m2"]), (1, ref["S0"][0]), (3, ref["S0"][2])):
        mu, err = _mean_err(obs[:, col])
        assert abs(mu - r) < 4 * err, (col, mu, r, err)
    assert obs[:, 16].max() < 1e-8
    assert 0.3 < obs[:, 13].mean() < 0.8


def test_set_variant_rejects_bad_kinds():
    with pytest.raises(ValueError):
        O.Chain(M.TORUS, 2, 0.3, 0.1, 1.0, 0.0, seed=1, slice_kind=3)
    with pytest.raises(ValueError):
        O.Chain(M.TORUS, 2, 0.3, 0.1, 1.0, 0.0, seed=1, drift_kind=2)
