"""Independent half-factor fields on the GPU (qmc_opts.slice_kind =
QMC_SLICE_INDEP) against the oracle's SLICE_INDEP chains.

Each of the seven Trotter factors of a slice (Methods, Eq.
trotter_decomposition_methods) is decoupled with its own field set, exponent
coefficient sqrt(-c_j dtau g_i): 7 N_q fields per slice, seven
eigendecompositions, B = V0 D0 T01 D1 ... T56 D6 V6^H without the
palindrome, the exact drift through the seven eigenbases, and the channel-0
background from both channel-0 sets.  Same seeds and Philox counters as the
oracle: identical decisions, log ratios within 1e-10, G within 1e-9 in FP64;
the mixed precisions within their tolerances; the prior whole-slice move and
the first-order drift over the seven sets.
"""
import numpy as np
import pytest

from oracle import learned as LN
from oracle import model as M
from oracle import oracle as O
from tests.test_gpu_parity import _compare_chain, _compare_mixed, _rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _oracle(nphi, beta, u, al, seed, nstab, drift=O.DRIFT_EXACT):
    return O.Chain(M.TORUS, nphi, beta, 0.1, u, al, seed, n_stab=nstab,
                   slice_kind=O.SLICE_INDEP, drift_kind=drift)


@pytest.mark.parametrize("nphi,beta,nstab", [(4, 2.0, 5), (5, 1.0, 4)])
def test_indep_fields_decision_identical(qmc, nphi, beta, nstab):
    nsw = 40
    L = int(round(beta / 0.1))
    g = qmc.Chain(qmc.QMC_TORUS, nphi, beta, 0.1, 1.5, 0.1, 3, n_stab=nstab,
                  slice_kind=qmc.QMC_SLICE_INDEP, trace_capacity=nsw * L)
    o = _oracle(nphi, beta, 1.5, 0.1, 3, nstab)
    assert g.fields(0).shape == (L, 7, g.n_q)
    assert np.abs(g.fields(0) - o.phi()).max() < 1e-13
    for t in (1, L):
        B, Bi = g.propagator(t)
        Bo, Boi = o.B(t)
        assert _rel(B, Bo) < 1e-12 and _rel(Bi, Boi) < 1e-12
    assert _rel(g.green(0), o.green()) < 1e-10
    g.sweep(nsw)
    g.sync()
    o.enable_trace(nsw * L)
    obs_o = o.sweep(nsw)
    _compare_chain(g, 0, o, nsw, g.trace(0), o.trace())
    obs_g = g.series()[0]
    for col in (0, 11, 12):
        assert np.abs(obs_g[:, col] - obs_o[:, col]).max() < 1e-9 * max(1, np.abs(obs_o[:, col]).max())


def test_indep_fields_in_a_batch(qmc):
    us, als, seeds = [0.5, 1.2, 2.0], [0.0, 0.1, -0.15], [3, 11, 42]
    nsw = 20
    g = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, 0.0, 0, n_chains=3, couplings=us,
                  anisotropies=als, seeds=seeds, n_stab=5, slice_kind=qmc.QMC_SLICE_INDEP,
                  trace_capacity=nsw * 10)
    g.sweep(nsw)
    g.sync()
    for c in range(3):
        o = _oracle(4, 1.0, us[c], als[c], seeds[c], 5)
        o.enable_trace(nsw * o.L)
        o.sweep(nsw)
        _compare_chain(g, c, o, nsw, g.trace(c), o.trace())


@pytest.mark.parametrize("precision", [1, 2])
def test_indep_fields_mixed_precision(qmc, precision):
    nsw = 100
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5, precision=precision,
                  slice_kind=qmc.QMC_SLICE_INDEP, trace_capacity=nsw * 20)
    g.sweep(nsw)
    g.sync()
    o = _oracle(4, 2.0, 1.0, 0.0, 0, 5)
    o.enable_trace(nsw * 20)
    o.sweep(nsw)
    assert _compare_mixed(g, 0, o, nsw, 1000) >= 1000
    s = g.series()[0]
    assert s[:, 15].max() < 1e-9 and s[:, 16].max() < 1e-9


def test_indep_fields_first_order_drift(qmc):
    nsw = 30
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.5, 0.1, 3, n_stab=5,
                  slice_kind=qmc.QMC_SLICE_INDEP, drift=qmc.QMC_DRIFT_FIRST,
                  trace_capacity=nsw * 20)
    g.sweep(nsw)
    g.sync()
    o = _oracle(4, 2.0, 1.5, 0.1, 3, 5, O.DRIFT_FIRST)
    o.enable_trace(nsw * 20)
    o.sweep(nsw)
    _compare_chain(g, 0, o, nsw, g.trace(0), o.trace())


@pytest.mark.parametrize("graph", [False, True])
def test_indep_fields_prior_moves(qmc, graph):
    """The prior whole-slice move over all 7 N_q fields (computed ahead by
    the prior stage) against the oracle's learned move with a zero network."""
    L = 22
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.2, 0.1, 3.0, 0.05, 0, n_stab=5,
                  slice_kind=qmc.QMC_SLICE_INDEP, trace_capacity=6 * L)
    o = _oracle(4, 2.2, 3.0, 0.05, 0, 5)
    o.enable_trace(6 * L)
    th = np.zeros(LN.n_params(7 * o.nq, 8))
    g.sweep(2)
    g.sweep_prior(2, 0.0, graph=graph)
    g.sweep_prior(2, 0.5, graph=graph)
    g.sync()
    o.sweep(2)
    o.sweep_learned(2, th, 8, 0.0)
    o.sweep_learned(2, th, 8, 0.5)
    tg, to = g.trace(0), o.trace()
    assert np.array_equal(tg[:, 6], to[:, 6]), "accept decisions differ"
    assert tg[2 * L:, 6].sum() > 0
    assert np.abs(tg[:, 2] - to[:, 2]).max() < 1e-10
    assert np.abs(g.fields(0) - o.phi()).max() < 1e-9
    assert _rel(g.green(0), o.green()) < 1e-9


def test_slice_kind_argument_checks(qmc):
    with pytest.raises(qmc.QMCError):
        qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 1.0, slice_kind=1)   # single exponential: oracle only
