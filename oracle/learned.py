"""Learned slice proposal: plain FP64 reference definitions.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the GPU path never
imports this module.

The proposal is not in the paper; it is added to the method: a small
network q_theta(phi_tau | phi_{tau-1}, phi_{tau+1}) over one imaginary-time
slice of the Hubbard-Stratonovich field, whose moves are
accepted by the exact Metropolis-Hastings test of the fermion weight
(Methods, Eq. weight and the determinant ratio of the local update), so the
sampled distribution is the paper's.

Network (all layers dense, row-major weights, x = [phi_{tau-1}, phi_{tau+1}]
of length 2 nf, nf = 4 N_q real fields per slice):
    a1 = W1 x + b1,  h1 = silu(a1)              W1: H x 2nf
    a2 = W2 h1 + b2, h2 = silu(a2)              W2: H x H
    o  = W3 h2 + b3                             W3: 2nf x H
    mu = o[:nf],  s = o[nf:]  (log sigma)
silu(a) = a / (1 + exp(-a)).
Parameters are packed as one vector in the order W1, b1, W2, b2, W3, b3.

Training loss: Gaussian negative log likelihood of the slice given its
neighbours, averaged over the batch and summed over fields, without the
constant (1/2) log 2 pi:
    loss = mean_b sum_f [ (1/2) ((y - mu) exp(-s))^2 + s ].
Optimiser: Adam (Kingma & Ba, 2015) with bias correction, optionally with
decoupled weight decay of the weight matrices (Loshchilov & Hutter, 2019).

Move (preconditioned Crank-Nicolson around the learned Gaussian
N(mu, diag sigma^2), sigma = exp(s), 0 <= rho < 1):
    phi' = mu + rho (phi - mu) + sqrt(1 - rho^2) sigma xi,  xi ~ N(0, 1).
It is reversible with respect to N(mu, sigma^2), whose parameters depend
only on the neighbours, so for the target pi(phi) = w(phi) exp(-|phi|^2/2)
    log A = 2 Re log R - (|phi'|^2 - |phi|^2)/2 - [log N(phi') - log N(phi)],
    log N(x) = -(1/2) sum_f ((x_f - mu_f)/sigma_f)^2 + const,
with log R the determinant ratio of the slice update (the same ratio as the
Langevin update).  rho = 0 is an independence proposal.
"""
from __future__ import annotations

import numpy as np


def shapes(nf: int, H: int):
    return [("W1", (H, 2 * nf)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
            ("W3", (2 * nf, H)), ("b3", (2 * nf,))]


def n_params(nf: int, H: int) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(nf, H))


def unpack(theta: np.ndarray, nf: int, H: int) -> dict:
    out, k = {}, 0
    for name, s in shapes(nf, H):
        n = int(np.prod(s))
        out[name] = theta[k:k + n].reshape(s)
        k += n
    assert k == len(theta)
    return out


def pack(p: dict, nf: int, H: int) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=float).ravel() for name, _ in shapes(nf, H)])


def _sig(a):
    return 1.0 / (1.0 + np.exp(-a))


def silu(a):
    return a * _sig(a)


def silu_grad(a):
    s = _sig(a)
    return s * (1.0 + a * (1.0 - s))


def forward(theta, X, nf, H):
    """X: (B, 2nf) -> (mu, s) each (B, nf), plus the activations."""
    p = unpack(np.asarray(theta, float), nf, H)
    X = np.asarray(X, float)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = silu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(a2)
    o = h2 @ p["W3"].T + p["b3"]
    return o[:, :nf], o[:, nf:], (X, a1, h1, a2, h2)


def loss_and_grad(theta, X, Y, nf, H):
    """Gaussian NLL (module docstring) and its gradient by the chain rule."""
    mu, s, (X, a1, h1, a2, h2) = forward(theta, X, nf, H)
    Y = np.asarray(Y, float)
    B = X.shape[0]
    r = (Y - mu) * np.exp(-s)
    loss = float(np.sum(0.5 * r * r + s) / B)
    dmu = -r * np.exp(-s) / B
    ds = (1.0 - r * r) / B
    do = np.concatenate([dmu, ds], axis=1)
    p = unpack(np.asarray(theta, float), nf, H)
    g = {}
    g["W3"] = do.T @ h2
    g["b3"] = do.sum(0)
    dh2 = do @ p["W3"]
    da2 = dh2 * silu_grad(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * silu_grad(a1)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(0)
    return loss, pack(g, nf, H)


def weight_mask(nf, H):
    """1 on the entries of W1, W2, W3 and 0 on the biases."""
    return np.concatenate([np.full(int(np.prod(s)), 0.0 if name.startswith("b") else 1.0)
                           for name, s in shapes(nf, H)])


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0, mask=None):
    """One Adam step (t = 1 for the first); returns new (theta, m, v).  wd is
    decoupled weight decay (Loshchilov & Hutter, 2019) on the entries where
    mask is 1: theta -= lr * wd * theta, from the value before the step."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    decay = 0.0 if mask is None else wd * mask * theta
    return theta - lr * (mh / (np.sqrt(vh) + eps) + decay), m, v


def pcn_move(mu, s, phi, rho, xi):
    """phi' and log N(phi') - log N(phi) of the module docstring."""
    sig = np.exp(s)
    php = mu + rho * (phi - mu) + np.sqrt(1.0 - rho * rho) * sig * xi
    lq = -0.5 * np.sum(((php - mu) / sig) ** 2) + 0.5 * np.sum(((phi - mu) / sig) ** 2)
    return php, lq
