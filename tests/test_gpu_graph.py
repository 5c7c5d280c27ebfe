"""Graph-captured sweeps and heterogeneous groups (batched chains of
different sizes in one CUDA graph per sweep).

A captured sweep launches the same kernels on the same data as the plain
sweep, with the sweep number and the series slot read from device memory,
so every result must be bit-identical to the plain path: Philox draws,
decisions, fields, G and the measurement records.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def _state(ch):
    ch.sync()
    out = [ch.series(), np.stack([ch.fields(c) for c in range(ch.n_chains)]),
           np.stack([ch.green(c) for c in range(ch.n_chains)]), ch.eps()]
    if ch.trace_capacity:
        out.append(np.stack([ch.trace(c) for c in range(ch.n_chains)]))
    return out


def _same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert x.shape == y.shape and np.array_equal(x, y)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_graph_sweeps_bit_identical(qmc, precision):
    kw = dict(n_chains=3, couplings=[0.5, 1.0, 1.5], seeds=[4, 5, 6], n_stab=4,
              trace_capacity=200, precision=precision)
    a = qmc.Chain(qmc.QMC_TORUS, 6, 1.0, 0.1, 0.0, **kw)
    b = qmc.Chain(qmc.QMC_TORUS, 6, 1.0, 0.1, 0.0, **kw)
    a.sweep(7)
    b.sweep(3, graph=True)
    b.sweep(1)              # plain and graph sweeps interleave
    b.sweep(3, graph=True)
    _same(_state(a), _state(b))
    assert a.series().shape[1] == 7


def test_learned_graph_sweeps_bit_identical(qmc):
    """Learned sweeps replayed from a graph make the plain learned sweeps'
    draws and decisions; the graph reads the network's weights in place, so
    new weights take effect without a new capture, and another rho gets its
    own capture."""
    from tests.learned_inputs import random_params
    kw = dict(n_chains=2, couplings=[0.8, 1.6], seeds=[9, 10], n_stab=5, trace_capacity=200,
              precision=1)
    a = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, **kw)
    b = qmc.Chain(qmc.QMC_TORUS, 4, 1.0, 0.1, 0.0, **kw)
    nf = 4 * a.n_q
    nets = []
    for _ in range(2):
        n = qmc.Net(nf, 32, 16, 2)
        n.set_params(random_params(nf, 32, 6, out_scale=0.1).astype(np.float32))
        nets.append(n)
    a.sweep_learned(nets[0], 2, 0.0)
    b.sweep_learned(nets[1], 2, 0.0, graph=True)
    th = random_params(nf, 32, 7, out_scale=0.1).astype(np.float32)
    for n in nets:
        n.set_params(th)
    a.sweep_learned(nets[0], 2, 0.0)
    b.sweep_learned(nets[1], 2, 0.0, graph=True)
    a.sweep(1)
    b.sweep(1, graph=True)
    a.sweep_learned(nets[0], 2, 0.5)
    b.sweep_learned(nets[1], 2, 0.5, graph=True)
    _same(_state(a), _state(b))


def test_group_of_mixed_sizes_bit_identical(qmc):
    """Torus N_phi = 8 and 12, a 5-orbital sphere, FP64 and mixed precision
    and different couplings in one graph: each member evolves exactly as it
    would alone."""
    def make():
        return [qmc.Chain(qmc.QMC_TORUS, 8, 0.8, 0.1, 0.0, n_chains=2, couplings=[0.7, 1.3],
                          seeds=[1, 2], n_stab=4),
                qmc.Chain(qmc.QMC_TORUS, 12, 0.6, 0.1, 1.0, 0.1, 9, n_stab=3, precision=1),
                qmc.Chain(qmc.QMC_SPHERE, 4, 0.5, 0.1, 0.3, 0.0, 11, n_stab=5)]
    solo = make()
    for c in solo:
        c.sweep(5)
    grouped = make()
    g = qmc.Group(grouped)
    g.sweep(2)
    grouped[1].sweep(1)      # a member may still be swept on its own
    g.sweep(1)
    grouped[0].sweep(1)
    grouped[2].sweep(1)
    g.sweep(1)
    grouped[1].sweep(1)
    g.sync()
    assert [c.series().shape[1] for c in grouped] == [5, 6, 5]
    for c in grouped:
        c.sync()
    # members swept one extra time alone: bring the solo runs level
    solo[1].sweep(1)
    for s_, c in zip(solo, grouped):
        _same(_state(s_), _state(c))
    g.close()


def test_batched_sizes_16_to_48(qmc):
    """The batched-chains shape: torus N_phi in {16, 24, 36, 48}, couplings in
    [0.5, 2], anisotropy in [-0.2, 0.2], mixed precision, one group; short
    beta so the test stays small.  Every member stays sign-free and stable."""
    rng = np.random.default_rng(0)
    chains = []
    for k, nphi in enumerate((16, 24, 36, 48)):
        u = rng.uniform(0.5, 2.0, 2)
        a = rng.uniform(-0.2, 0.2, 2)
        chains.append(qmc.Chain(qmc.QMC_TORUS, nphi, 0.4, 0.1, 0.0, n_chains=2, couplings=u,
                                anisotropies=a, seeds=[10 * k, 10 * k + 1], n_stab=2,
                                precision=1))
    g = qmc.Group(chains)
    g.sweep(2)
    g.sync()
    for c in chains:
        s = c.series()
        assert s.shape[1] == 2
        assert s[:, :, 15].max() < 1e-8 and s[:, :, 16].max() < 1e-8
        assert np.all(np.isfinite(s))
    g.close()


def test_group_argument_checks(qmc):
    a = qmc.Chain(qmc.QMC_TORUS, 4, 0.2, 0.1, 1.0)
    with pytest.raises(qmc.QMCError):
        qmc.Group([a, a])
