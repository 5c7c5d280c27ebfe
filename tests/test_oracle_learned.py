"""Pins of the oracle's learned slice move (oracle/learned.py and the C
oracle's orc_sweep_learned) against the mathematics: finite differences,
closed forms, the optimiser's first step, the exactly solvable
non-interacting limit, stationarity of N(0,1) there for any network, and
agreement of the learned chain's observables with the Langevin chain."""
import numpy as np

from oracle import learned as LN
from oracle import model as M
from oracle import oracle as O
from tests.learned_inputs import random_batch, random_params


def test_gradient_matches_central_differences():
    nf, H, B = 3, 4, 5
    th = random_params(nf, H, 1, out_scale=0.7, logsig_bias=0.2)
    X, Y = random_batch(nf, B, 2)
    _, g = LN.loss_and_grad(th, X, Y, nf, H)
    h = 1e-6
    fd = np.zeros_like(th)
    for k in range(len(th)):
        e = np.zeros_like(th)
        e[k] = h
        fd[k] = (LN.loss_and_grad(th + e, X, Y, nf, H)[0] -
                 LN.loss_and_grad(th - e, X, Y, nf, H)[0]) / (2 * h)
    assert np.abs(g - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def test_output_bias_closed_form():
    """W3 = 0: mu = m and s = s0 for every input, so the loss is
    mean_b sum_f [ (y - m)^2 exp(-2 s0)/2 + s0 ] with the gradient below."""
    nf, H, B = 4, 6, 7
    th = random_params(nf, H, 3).copy()
    p = LN.unpack(th, nf, H)
    p["W3"][:] = 0.0
    m, s0 = 0.3, -0.4
    p["b3"][:nf] = m
    p["b3"][nf:] = s0
    th = LN.pack(p, nf, H)
    X, Y = random_batch(nf, B, 4)
    L, g = LN.loss_and_grad(th, X, Y, nf, H)
    w = np.exp(-2 * s0)
    assert abs(L - np.sum(0.5 * (Y - m) ** 2 * w + s0) / B) < 1e-12
    gb = LN.unpack(g, nf, H)["b3"]
    assert np.allclose(gb[:nf], -np.sum((Y - m) * w, axis=0) / B, atol=1e-12)
    assert np.allclose(gb[nf:], np.sum(1 - (Y - m) ** 2 * w, axis=0) / B, atol=1e-12)
    # nothing flows into the hidden layers through a zero output layer
    assert np.abs(LN.unpack(g, nf, H)["W1"]).max() == 0.0


def test_adam_first_step_is_a_sign_step():
    r = np.random.default_rng(5)
    th, g = r.standard_normal(50), r.standard_normal(50)
    new, m, v = LN.adam_step(th, g, np.zeros(50), np.zeros(50), 1, 0.01)
    assert np.allclose(new - th, -0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)


def test_decoupled_weight_decay_step():
    """Zero gradient: the moments stay 0 and only the decay acts, on the
    weight matrices and not on the biases."""
    nf, H = 2, 3
    th = random_params(nf, H, 12, out_scale=1.0, mu_bias=0.5)
    n = len(th)
    new, _, _ = LN.adam_step(th, np.zeros(n), np.zeros(n), np.zeros(n), 1, 0.1, wd=0.5,
                             mask=LN.weight_mask(nf, H))
    p, q = LN.unpack(th, nf, H), LN.unpack(new, nf, H)
    for name in ("W1", "W2", "W3"):
        assert np.allclose(q[name], p[name] * (1 - 0.05), atol=1e-15)
    for name in ("b1", "b2", "b3"):
        assert np.array_equal(q[name], p[name])


def test_c_forward_equals_numpy():
    nf, H = 7, 16
    th = random_params(nf, H, 6, out_scale=0.5)
    X, _ = random_batch(nf, 9, 7)
    mu, s, _ = LN.forward(th, X, nf, H)
    out = O.mlp_forward(th, X, nf, H)
    assert np.abs(out - np.concatenate([mu, s], axis=1)).max() < 1e-13


def test_pcn_special_cases():
    r = np.random.default_rng(8)
    mu, s, phi, xi = (r.standard_normal(6) for _ in range(4))
    php, lq = LN.pcn_move(mu, s, phi, 1.0, xi)
    assert np.allclose(php, phi, rtol=0, atol=1e-15) and abs(lq) < 1e-14
    php, lq = LN.pcn_move(np.zeros(6), np.zeros(6), phi, 0.0, xi)
    assert np.allclose(php, xi) and abs(lq - (-0.5 * xi @ xi + 0.5 * phi @ phi)) < 1e-13


def _free_chain(nphi=2, beta=0.4, seed=0):
    return O.Chain(M.TORUS, nphi, beta, 0.1, 0.0, 0.0, seed, n_stab=2, g=np.zeros(4))


def test_free_limit_exact_proposal_always_accepted():
    """g = 0: B = 1, the weight is the Gaussian N(0, 1) itself.  A network
    with zero output (mu = 0, sigma = 1) and rho = 0 proposes exactly the
    target, so log A = 0 and every move is accepted."""
    o = _free_chain()
    nf, H = 4 * o.nq, 8
    th = random_params(nf, H, 9, out_scale=0.0)
    o.enable_trace(5 * o.L)
    obs = o.sweep_learned(5, th, H, 0.0)
    tr = o.trace()
    assert np.abs(tr[:, 4]).max() < 1e-12 and tr[:, 6].all()
    assert np.all(obs[:, 13] == 1.0)


def test_free_limit_stationary_for_any_network():
    """g = 0 with a network far from the target (mu = 0.6, sigma = 0.6): the
    MH correction must still leave N(0, 1) invariant (a wrong sign of the
    proposal-density term would pull the fields towards mu)."""
    o = _free_chain(nphi=2, beta=0.4, seed=3)
    nf, H = 4 * o.nq, 8
    th = random_params(nf, H, 10, out_scale=0.3, mu_bias=0.6, logsig_bias=np.log(0.6))
    o.sweep_learned(20, th, H, 0.3)
    means, sq = [], []
    for _ in range(60):
        o.sweep_learned(5, th, H, 0.3)
        p = o.phi()
        means.append(p.mean())
        sq.append((p * p).mean())
    n_fields = o.phi().size
    m, v = np.mean(means), np.mean(sq)
    em = np.std(means) / np.sqrt(len(means)) + 1.0 / np.sqrt(n_fields * len(means))
    assert abs(m) < 5 * em, (m, em)
    assert abs(v - 1.0) < 5 * (np.std(sq) / np.sqrt(len(sq)) + 0.02), v


def test_learned_chain_matches_langevin_chain():
    """Interacting torus N_phi = 2: observables of learned-move chains (an
    untrained network) agree with the Langevin chains within errors."""
    nf = None
    Eg, El, Mg, Ml = [], [], [], []
    for seed in range(4):
        a = O.Chain(M.TORUS, 2, 1.0, 0.1, 1.0, 0.0, 100 + seed, n_stab=5)
        b = O.Chain(M.TORUS, 2, 1.0, 0.1, 1.0, 0.0, 200 + seed, n_stab=5)
        nf = 4 * a.nq
        th = random_params(nf, 8, 11 + seed, out_scale=0.1)
        a.sweep(50)
        b.sweep(50)
        oa = a.sweep(300)
        ob = np.concatenate([np.concatenate([b.sweep(1), b.sweep_learned(1, th, 8, 0.5)])
                             for _ in range(150)])
        Eg.append(oa[:, 12].mean()); Mg.append(oa[:, 0].mean())
        El.append(ob[:, 12].mean()); Ml.append(ob[:, 0].mean())
    for x, y in ((Eg, El), (Mg, Ml)):
        d = np.mean(x) - np.mean(y)
        err = np.sqrt(np.var(x) / len(x) + np.var(y) / len(y)) + 1e-12
        assert abs(d) < 5 * err, (np.mean(x), np.mean(y), err)
