"""Edge cases of the GPU sweep against the oracle: a single imaginary-time
slice (L = 1), restabilisation after every slice (n_stab = 1) and only at
beta (n_stab > L), a large torus (N_phi = 56, N = 112; the largest size,
N = 120, is in test_gpu_large.py), and zero sweeps."""
import numpy as np
import pytest

from oracle import model as M
from oracle import oracle as O
from tests.test_gpu_parity import _compare_chain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _run(qmc, nphi, beta, u, al, seed, nstab, nsw):
    L = int(round(beta / 0.1))
    g = qmc.Chain(qmc.QMC_TORUS, nphi, beta, 0.1, u, al, seed, n_stab=nstab,
                  trace_capacity=nsw * L)
    g.sweep(nsw)
    g.sync()
    o = O.Chain(M.TORUS, nphi, beta, 0.1, u, al, seed, n_stab=nstab)
    o.enable_trace(nsw * L)
    o.sweep(nsw)
    _compare_chain(g, 0, o, nsw, g.trace(0), o.trace())
    return g, o


def test_single_slice(qmc):
    g, o = _run(qmc, 4, 0.1, 1.0, 0.0, 0, 5, 20)
    assert g.L == 1


@pytest.mark.parametrize("nstab", [1, 7])
def test_restabilisation_every_slice_and_only_at_beta(qmc, nstab):
    g, o = _run(qmc, 3, 0.5, 1.5, 0.1, 4, nstab, 10)
    assert g.series()[0][:, 15].max() < 1e-9


def test_large_torus(qmc):
    """N_phi = 56 (N = 112, N_q = 517): two slices, one sweep (the largest
    size whose QR keeps all its vectors in shared memory)."""
    g, o = _run(qmc, 56, 0.2, 1.0, 0.1, 2, 5, 1)
    assert g.n_q == 517 and g.N == 112


def test_zero_sweeps_change_nothing(qmc):
    g = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 1.0, 0.0, 0, n_stab=5)
    f0, G0 = g.fields(0), g.green(0)
    g.sweep(0)
    g.sync()
    assert np.array_equal(g.fields(0), f0) and np.array_equal(g.green(0), G0)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_poisoned_scratch_changes_nothing(qmc, monkeypatch, precision):
    """QMC_POISON_SCRATCH fills every scratch buffer with NaN bytes at
    creation: a buffer read before it is written would turn the chain into
    NaNs.  The Langevin and learned sweeps must still make the oracle's
    decisions (FP64) or track it (mixed)."""
    from oracle import learned as LN
    from tests.test_gpu_parity import _compare_mixed
    monkeypatch.setenv("QMC_POISON_SCRATCH", "1")
    nsw, L = 6, 10
    g = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 1.5, 0.1, 3, n_stab=5, precision=precision,
                  trace_capacity=2 * nsw * L)
    o = O.Chain(M.TORUS, 4, 1.0, 0.1, 1.5, 0.1, 3, n_stab=5)
    o.enable_trace(2 * nsw * L)
    nf = 4 * o.nq
    net = qmc.Net(nf, 16, 16, 5)
    th = np.zeros(LN.n_params(nf, 16))
    g.sweep(nsw)
    g.sweep_learned(net, nsw, 0.0)
    g.sync()
    o.sweep(nsw)
    o.sweep_learned(nsw, th, 16, 0.0)
    if precision == 0:
        _compare_chain(g, 0, o, 2 * nsw, g.trace(0), o.trace())
    else:
        assert _compare_mixed(g, 0, o, 2 * nsw, 2 * nsw * L // 2) > 0
    assert np.all(np.isfinite(g.series()[0][:, :13]))
