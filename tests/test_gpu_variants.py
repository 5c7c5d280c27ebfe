"""GPU first-order drift (qmc_opts.drift = QMC_DRIFT_FIRST) against the
oracle's DRIFT_FIRST chains: the same decisions, log ratios and G as the
FP64 oracle, per chain in a batch with different couplings (the drift uses
each chain's alpha_i), and in mixed precision within the mixed-mode
tolerances."""
import numpy as np
import pytest

from oracle import model as M
from oracle import oracle as O
from tests.test_gpu_parity import _compare_chain, _compare_mixed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _oracle(nphi, beta, u, al, seed, nstab, nsw):
    o = O.Chain(M.TORUS, nphi, beta, 0.1, u, al, seed, n_stab=nstab, drift_kind=O.DRIFT_FIRST)
    o.enable_trace(nsw * o.L)
    o.sweep(nsw)
    return o


@pytest.mark.parametrize("nphi,beta,nstab", [(4, 2.0, 5), (5, 1.0, 4)])
def test_first_order_drift_makes_the_oracle_decisions(qmc, nphi, beta, nstab):
    nsw = 40
    L = int(round(beta / 0.1))
    g = qmc.Chain(qmc.QMC_TORUS, nphi, beta, 0.1, 1.5, 0.1, 3, n_stab=nstab,
                  drift=qmc.QMC_DRIFT_FIRST, trace_capacity=nsw * L)
    g.sweep(nsw)
    g.sync()
    o = _oracle(nphi, beta, 1.5, 0.1, 3, nstab, nsw)
    _compare_chain(g, 0, o, nsw, g.trace(0), o.trace())
    # the exact drift's chain takes other decisions from the same seed
    e = qmc.Chain(qmc.QMC_TORUS, nphi, beta, 0.1, 1.5, 0.1, 3, n_stab=nstab,
                  trace_capacity=nsw * L)
    e.sweep(nsw)
    e.sync()
    assert np.abs(e.trace(0)[:, 4] - g.trace(0)[:, 4]).max() > 1e-6


def test_first_order_drift_in_a_batch(qmc):
    us, als, seeds = [0.5, 1.2, 2.0], [0.0, 0.1, -0.15], [3, 11, 42]
    nsw = 20
    g = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, 0.0, 0, n_chains=3, couplings=us,
                  anisotropies=als, seeds=seeds, n_stab=5, drift=qmc.QMC_DRIFT_FIRST,
                  trace_capacity=nsw * 10)
    g.sweep(nsw)
    g.sync()
    for c in range(3):
        o = _oracle(4, 1.0, us[c], als[c], seeds[c], 5, nsw)
        _compare_chain(g, c, o, nsw, g.trace(c), o.trace())


def test_first_order_drift_mixed_precision(qmc):
    nsw = 100
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5, precision=1,
                  drift=qmc.QMC_DRIFT_FIRST, trace_capacity=nsw * 20)
    g.sweep(nsw)
    g.sync()
    o = _oracle(4, 2.0, 1.0, 0.0, 0, 5, nsw)
    assert _compare_mixed(g, 0, o, nsw, 1000) >= 1000
