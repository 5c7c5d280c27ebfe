"""GPU learned slice proposal (qmc_net_*, qmc_sweep_learned) against the
FP64 oracle (oracle/learned.py, orc_sweep_learned).

The network weights are seeded inputs rounded to bfloat16-representable
values, so the GPU's bfloat16 products and the oracle's FP64 products use
identical numbers; the remaining differences are FP32 accumulation (about
1e-6 relative).  The learned sweep must make the oracle's decisions, and a
chain that interleaves learned moves must reproduce the Langevin chain's
observables while decorrelating faster.
"""
import numpy as np
import pytest

from oracle import learned as LN
from oracle import model as M
from oracle import oracle as O
from tests.learned_inputs import random_batch, random_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qmc():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_03700_gb300 import build
    build.build()
    import paper_2605_03700_gb300 as P
    return P


def test_loss_and_gradient_match_the_oracle(qmc):
    nf, H, B = 148, 32, 20
    th = random_params(nf, H, 1, out_scale=0.5, logsig_bias=0.1)
    X, Y = random_batch(nf, B, 2)
    X, Y = X.astype(np.float32), Y.astype(np.float32)
    net = qmc.Net(nf, H, 16, 3)
    assert net.num_params == LN.n_params(nf, H)
    net.set_params(th.astype(np.float32))
    assert np.array_equal(net.get_params().astype(float), th)
    lg, gg = net.loss_grad(X, Y)
    lo, go = LN.loss_and_grad(th, X.astype(float), Y.astype(float), nf, H)
    assert abs(lg - lo) < 1e-6 * abs(lo)
    assert np.abs(gg - go).max() < 1e-5 * np.abs(go).max()
    out = net.forward(X)
    mu, s, _ = LN.forward(th, X.astype(float), nf, H)
    ref = np.concatenate([mu, s], axis=1)
    assert np.abs(out - ref).max() < 1e-5 * max(1.0, np.abs(ref).max())


def test_learned_sweep_makes_the_oracle_decisions(qmc):
    """Torus N_phi = 4, beta = 2, u = 1: two Langevin sweeps, then five
    learned sweeps at rho = 0.5 with the same seeded network."""
    L = 20
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5, trace_capacity=7 * L)
    o = O.Chain(M.TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5)
    o.enable_trace(7 * L)
    nf = 4 * o.nq
    th = random_params(nf, 16, 4, out_scale=0.1)
    net = qmc.Net(nf, 16, 16, 5)
    net.set_params(th.astype(np.float32))
    g.sweep(2)
    g.sweep_learned(net, 5, 0.5)
    g.sync()
    obs_o = np.concatenate([o.sweep(2), o.sweep_learned(5, th, 16, 0.5)])
    tg, to = g.trace(0), o.trace()
    assert len(tg) == len(to) == 7 * L
    assert np.array_equal(tg[:, 6], to[:, 6]), "accept decisions differ"
    learned = to[2 * L:]
    assert 0 < learned[:, 6].sum() < len(learned)
    assert np.all(tg[2 * L:, 7] == 0.5)
    # mu, sigma from FP32 accumulation: proposals differ at ~1e-7
    assert np.abs(tg[:, 2] - to[:, 2]).max() < 1e-7
    assert np.abs(g.fields(0) - o.phi()).max() < 1e-5
    obs_g = g.series()[0]
    assert np.array_equal(obs_g[:, 17], obs_o[:, 17])
    # learned sweeps leave the Langevin step unchanged
    assert np.all(obs_g[2:, 14] == obs_g[2, 14])


@pytest.mark.parametrize("graph", [False, True])
def test_prior_sweep_makes_the_oracle_decisions(qmc, graph):
    """Whole-slice moves around N(0, 1) without a network (qmc_sweep_prior)
    are the learned move of a network whose output is zero: the oracle's
    learned sweep with zero parameters makes the same decisions."""
    L = 20
    g = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5, trace_capacity=7 * L)
    o = O.Chain(M.TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_stab=5)
    o.enable_trace(7 * L)
    nf = 4 * o.nq
    th = np.zeros(LN.n_params(nf, 8))
    g.sweep(2)
    g.sweep_prior(3, 0.0, graph=graph)
    g.sweep_prior(2, 0.5, graph=graph)
    g.sync()
    obs_o = np.concatenate([o.sweep(2), o.sweep_learned(3, th, 8, 0.0),
                            o.sweep_learned(2, th, 8, 0.5)])
    tg, to = g.trace(0), o.trace()
    assert len(tg) == len(to) == 7 * L
    assert np.array_equal(tg[:, 6], to[:, 6]), "accept decisions differ"
    assert np.abs(tg[:, 2] - to[:, 2]).max() < 1e-10
    assert np.all(tg[2 * L:5 * L, 7] == 0.0) and np.all(tg[5 * L:, 7] == 0.5)
    assert np.abs(g.fields(0) - o.phi()).max() < 1e-9
    assert np.array_equal(g.series()[0][:, 17], obs_o[:, 17])


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_prior_stage_equals_per_slice_proposals(qmc, precision):
    """Prior sweeps compute every slice's proposal ahead, in chunks of slices
    batched over (chain, slice) on a second stream; the learned sweep of a
    network whose output is zero makes the same move one slice at a time.
    Both run the same kernels on each matrix, so two copies of one batch
    (three chains with different couplings, L = 22: chunks 6, 6, 6, 4) stay
    bit-identical through eager and graph-replayed sweeps."""
    kw = dict(n_chains=3, couplings=[0.5, 1.0, 1.6], anisotropies=[0.0, 0.1, -0.1],
              seeds=[4, 5, 6], n_stab=5, precision=precision, trace_capacity=6 * 22)
    a = qmc.Chain(qmc.QMC_TORUS, 5, 2.2, 0.1, 1.0, 0.0, 0, **kw)
    b = qmc.Chain(qmc.QMC_TORUS, 5, 2.2, 0.1, 1.0, 0.0, 0, **kw)
    net = qmc.Net(4 * a.n_q, 16, 16, 2)
    for ch in (a, b):
        ch.sweep(1)
    a.sweep_prior(2, 0.3)
    a.sweep_prior(3, 0.0, graph=True)
    b.sweep_learned(net, 2, 0.3)
    b.sweep_learned(net, 3, 0.0, graph=True)
    for ch in (a, b):
        ch.sync()
    for c in range(3):
        ta, tb = a.trace(c), b.trace(c)
        assert len(ta) == 6 * 22
        assert np.array_equal(ta, tb)
        assert np.array_equal(a.fields(c), b.fields(c))
        assert np.array_equal(a.green(c), b.green(c))
        assert 0 < ta[22:, 6].sum() < 5 * 22
    assert np.array_equal(a.series(), b.series())


def test_training_and_weight_decay(qmc):
    """Training lowers the loss on the collected data; with a large decoupled
    weight decay the weight matrices shrink toward zero."""
    ch = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_chains=4, seeds=[1, 2, 3, 4],
                   n_stab=5)
    net = qmc.Net(4 * ch.n_q, 32, 64, 9)
    with pytest.raises(qmc.QMCError):
        net.train(1)
    ch.sweep(5)
    for _ in range(8):
        ch.sweep(1)
        net.collect(ch)
    assert net.dataset_size == 32
    loss = net.train(400, 128, 3e-3)
    assert loss[-50:].mean() < loss[:20].mean() - 1.0
    w0 = net.get_params()
    # lr * weight_decay = 0.02 per step: the decay factor over 200 steps is
    # ~0.02, far below the drift Adam's own steps (~lr each) can undo
    net.train(200, 128, 1e-3, weight_decay=20.0)
    w1 = net.get_params()
    p0, p1 = LN.unpack(w0.astype(float), net.nf, 32), LN.unpack(w1.astype(float), net.nf, 32)
    assert np.abs(p1["W2"]).mean() < 0.4 * np.abs(p0["W2"]).mean()


def test_learned_chain_exact_and_decorrelates_faster(qmc):
    """Torus N_phi = 4, beta = 2, u = 1, 8 chains each.  Plain Langevin chains
    and chains alternating Langevin and learned sweeps (the untrained network,
    i.e. whole-slice moves from the Gaussian prior, rho = 0) agree on E and
    m^2 within errors, and the learned chains' integrated autocorrelation
    time is smaller."""
    nsw = 400
    res = {}
    for name, seed0 in (("plain", 100), ("learned", 200)):
        ch = qmc.Chain(qmc.QMC_TORUS, 4, 2.0, 0.1, 1.0, 0.0, 0, n_chains=8,
                       seeds=np.arange(8) + seed0, n_stab=5, series_capacity=2 * nsw + 64)
        net = qmc.Net(4 * ch.n_q, 64, 16, 1)
        ch.sweep(30)
        for _ in range(nsw // 2):
            if name == "plain":
                ch.sweep(2)
            else:
                ch.sweep(1)
                ch.sweep_learned(net, 1, 0.0)
        ch.sync()
        s = ch.series()[:, 30:, :]
        taus = [max(qmc.qmc_tau_int(s[c, :, 0]), qmc.qmc_tau_int(s[c, :, 12])) for c in range(8)]
        res[name] = (s[:, :, 12].mean(1), s[:, :, 0].mean(1), np.mean(taus))
    for k in (0, 1):
        a, b = res["plain"][k], res["learned"][k]
        err = np.sqrt(a.var() / len(a) + b.var() / len(b))
        assert abs(a.mean() - b.mean()) < 5 * err + 1e-12, (a.mean(), b.mean(), err)
    assert res["learned"][2] < res["plain"][2], (res["learned"][2], res["plain"][2])
