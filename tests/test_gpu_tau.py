"""GPU time-displaced structure factors (qmc_measure_tau) against the FP64
oracle: the stable-form Green's functions at the stabilisation points and
their propagation between them give the oracle's S^i_0(tau) (plain
propagation at small beta, the oracle's stable form at beta = 10), on ragged
sizes and per chain of a batch; S(0) is the equal-time record and
S(beta) = S(0)."""
import numpy as np
import pytest

from oracle import model as M
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("nphi,beta,nstab,nsw", [(4, 2.0, 5, 3), (5, 1.3, 4, 2)])
def test_measure_tau_matches_the_oracle(qmc, nphi, beta, nstab, nsw):
    g = qmc.Chain(qmc.QMC_TORUS, nphi, beta, 0.1, 1.5, 0.1, 3, n_stab=nstab)
    o = O.Chain(M.TORUS, nphi, beta, 0.1, 1.5, 0.1, 3, n_stab=nstab)
    g.sweep(nsw)
    g.sync()
    o.sweep(nsw)
    taus = list(range(o.L + 1))
    Sg = g.measure_tau(taus)
    So = o.measure_tau(taus)
    assert Sg.shape == (1, len(taus), 5)
    assert _rel(Sg[0], So) < 1e-9
    eq = g.measure()[0, 1:6]
    assert np.abs(Sg[0, 0] - eq).max() < 1e-10 * np.abs(eq).max()
    assert np.abs(Sg[0, -1] - Sg[0, 0]).max() < 1e-9 * np.abs(eq).max()
    # a subset in any spacing gives the same values
    sub = [0, 3, nstab, o.L]
    assert np.abs(g.measure_tau(sub)[0] - Sg[0, sub]).max() < 1e-13 * np.abs(eq).max()


def test_measure_tau_per_chain_of_a_batch(qmc):
    us, als, seeds = [0.5, 1.2, 2.0], [0.0, 0.1, -0.15], [3, 11, 42]
    g = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, 0.0, 0, n_chains=3, couplings=us,
                  anisotropies=als, seeds=seeds, n_stab=5)
    g.sweep(2)
    g.sync()
    taus = [0, 2, 5, 9, 10]
    Sg = g.measure_tau(taus)
    for c in range(3):
        o = O.Chain(M.TORUS, 4, 1.0, 0.1, us[c], als[c], seeds[c], n_stab=5)
        o.sweep(2)
        assert _rel(Sg[c], o.measure_tau(taus)) < 1e-9, c


def test_measure_tau_at_large_beta(qmc):
    """beta = 10 (L = 100): the oracle's stable form; S decays and returns."""
    g = qmc.Chain(qmc.QMC_TORUS, 4, 10.0, 0.1, 2.0, 0.2, 5, n_stab=10)
    o = O.Chain(M.TORUS, 4, 10.0, 0.1, 2.0, 0.2, 5, n_stab=10)
    taus = [0, 1, 9, 10, 11, 37, 50, 99, 100]
    Sg = g.measure_tau(taus)[0]
    So = o.measure_tau(taus, stable=True)
    assert _rel(Sg, So) < 1e-8
    assert np.abs(Sg[-1] - Sg[0]).max() < 1e-8 * np.abs(Sg[0]).max()
    assert np.all(Sg[6, 2:] < Sg[0, 2:])


def test_measure_tau_rejects_bad_offsets(qmc):
    g = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 1.0, 0.0, 0, n_stab=5)
    for bad in ([3, 2], [-1], [11]):
        with pytest.raises(qmc.QMCError):
            g.measure_tau(bad)


def test_measure_tau_on_the_sphere(qmc):
    """Sphere, 3 orbitals (l = 0 is the ordering momentum), beta = 1, at
    the paper's sphere coupling scale u = 0.3."""
    g = qmc.Chain(qmc.QMC_SPHERE, 2, 1.0, 0.1, 0.3, 0.1, 5, n_stab=5)
    m = M.Model(M.SPHERE, 3)
    o = O.Chain(M.SPHERE, 3, 1.0, 0.1, 0.3, 0.1, 5, n_stab=5, model=m)
    g.sweep(2)
    g.sync()
    o.sweep(2)
    taus = list(range(o.L + 1))
    assert _rel(g.measure_tau(taus)[0], o.measure_tau(taus)) < 1e-8
