"""Pins of the oracle's time-displaced Green's functions and structure factors
(the groundwork of the SO(5) gap measurement; GPU kernels for them come
later).

Fixed by: the boundary values G(beta,0) = 1 - G and Gbar(0,beta) = G
(antiperiodicity), the exact identities G(t,0) = [B(t,0)^-1 + B(beta,t)]^-1
and Gbar(0,t) = [B(t,0) + B(beta,t)^-1]^-1 evaluated from the raw slice
products, the equal-time limit, periodicity S(beta) = S(0), the free limit
(no dynamics), and exact diagonalisation of the transformed Hamiltonian.
"""
import math

import numpy as np
import pytest

from oracle import ed as E
from oracle import model as M
from oracle import oracle as O
from tests.sphere_units import sphere_u


def _chain(beta=1.0, dtau=0.1, u=2.0, al=0.2, seed=3, g=None):
    ch = O.Chain(M.TORUS, 2, beta, dtau, u, al, seed, n_stab=5, g=g)
    ch.sweep(20)
    return ch


def _prod(ch, t1, t2):
    """B(t2, t1) = B_t2 ... B_{t1+1} from the stored slice propagators"""
    P = np.eye(ch.N, dtype=complex)
    for t in range(t1 + 1, t2 + 1):
        P = ch.B(t)[0] @ P
    return P


def test_boundary_values_and_identities():
    ch = _chain()
    G = ch.green()
    L, I = ch.L, np.eye(ch.N)
    Gt0, Gb, Gtt = ch.green_tau(0)
    assert np.abs(Gt0 - G).max() < 1e-14 and np.abs(Gb - (I - G)).max() < 1e-14
    Gt0, Gb, Gtt = ch.green_tau(L)
    assert np.abs(Gt0 - (I - G)).max() < 1e-10       # G(beta, 0) = 1 - G
    assert np.abs(Gb - G).max() < 1e-10              # Gbar(0, beta) = G
    assert np.abs(Gtt - G).max() < 1e-10
    for t in (1, 3, L // 2, L - 1):
        Gt0, Gb, Gtt = ch.green_tau(t)
        Bt0, Bbt = _prod(ch, 0, t), _prod(ch, t, L)
        assert np.abs(Gt0 - np.linalg.inv(np.linalg.inv(Bt0) + Bbt)).max() < 1e-10
        assert np.abs(Gb - np.linalg.inv(Bt0 + np.linalg.inv(Bbt))).max() < 1e-10
        assert np.abs(Gtt - ch.green_bruteforce(t)).max() < 1e-10


def test_equal_time_limit_and_periodicity():
    ch = _chain()
    S = ch.measure_tau([0, ch.L])
    eq = ch.measure()[1:6]
    assert np.abs(S[0] - eq).max() < 1e-12 * max(1.0, np.abs(eq).max())
    assert np.abs(S[1] - S[0]).max() < 1e-10
    # spin SO(3): the three spin components agree at every tau
    S = ch.measure_tau([1, 4, 7])
    assert np.all(S[:, 2] == S[:, 3]) and np.all(S[:, 3] == S[:, 4])


def test_free_limit_has_no_dynamics():
    ch = _chain(g=np.zeros(4))
    S = ch.measure_tau(list(range(ch.L + 1)))
    assert np.abs(S - S[0]).max() < 1e-14


def _mean_err(x, nbin=50):
    b = np.array_split(np.asarray(x), nbin)
    m = np.array([v.mean() for v in b])
    return m.mean(), m.std(ddof=1) / math.sqrt(nbin)


def test_time_displaced_structure_factor_matches_exact_diagonalisation():
    """torus N_phi = 2, u = 4, alpha = 0.3, beta = 2, dtau = 0.05: Monte Carlo
    S^1_0(tau) and S^3_0(tau) at tau = 0.5 and 1 within 4 sigma of ED."""
    m = M.Model(M.TORUS, 2)
    beta, dtau = 2.0, 0.05
    ed = E.ED(m, M.couplings(4.0, 0.3), beta)
    ch = O.Chain(M.TORUS, 2, beta, dtau, 4.0, 0.3, seed=7, n_stab=5, n_adapt=150, model=m)
    ch.sweep(150)
    taus = [10, 20]
    rec = []
    for _ in range(2500):
        ch.sweep(1)
        rec.append(ch.measure_tau(taus))
    rec = np.array(rec)
    q0 = m.q0()
    for k, t in enumerate(taus):
        for gi, col in ((0, 0), (2, 2)):
            ref = ed.structure_factor_tau(gi, q0, t * dtau)
            mu, err = _mean_err(rec[:, k, col])
            assert abs(mu - ref) < 4 * err, (t, gi, mu, ref, err)
    # and S(tau) really decays away from tau = 0 in this model
    assert ed.structure_factor_tau(0, q0, 1.0) < ed.structure_factor_tau(0, q0, 0.0)


def test_stable_form_equals_plain_propagation_at_small_beta():
    ch = _chain(beta=1.0)
    for t in (0, 1, 4, 7, ch.L):
        for a, b in zip(ch.green_tau(t), ch.green_tau_stable(t)):
            assert np.abs(a - b).max() < 1e-10, t


def test_stable_form_at_large_beta():
    """beta = 10 (L = 100), u = 2: the boundary values, the sweep's own
    stabilised G at t = 0, and the one-slice relations G(t+1,0) = B G(t,0),
    Gbar(0,t+1) = Gbar(0,t) B^-1, G(t+1,t+1) = B G(t,t) B^-1 (each product a
    single well-conditioned slice) hold to rounding."""
    ch = O.Chain(M.TORUS, 2, 10.0, 0.1, 2.0, 0.2, 5, n_stab=5)
    ch.sweep(10)
    G, I, L = ch.green(), np.eye(ch.N), ch.L
    Gt0, Gb, Gtt = ch.green_tau_stable(0)
    assert np.abs(Gtt - G).max() < 1e-10 and np.abs(Gt0 - G).max() < 1e-10
    Gt0, Gb, Gtt = ch.green_tau_stable(L)
    assert np.abs(Gt0 - (I - G)).max() < 1e-9 and np.abs(Gb - G).max() < 1e-9
    prev = ch.green_tau_stable(37)
    cur = ch.green_tau_stable(38)
    B, Bi = ch.B(38)
    assert np.abs(cur[0] - B @ prev[0]).max() < 1e-9
    assert np.abs(cur[1] - prev[1] @ Bi).max() < 1e-9
    assert np.abs(cur[2] - B @ prev[2] @ Bi).max() < 1e-9
    # all three are O(1): Green's functions, however large B(t,0) is
    assert max(np.abs(m).max() for m in cur) < 10


def test_stable_structure_factors():
    """S^i_0(tau) from the stable Green's functions equals the plain
    propagation at beta = 1, and at beta = 10 starts at the equal-time
    record and is periodic, S(beta) = S(0)."""
    ch = _chain(beta=1.0)
    taus = [0, 1, 4, 5, 7, 10]
    a, b = ch.measure_tau(taus), ch.measure_tau(taus, stable=True)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    ch = O.Chain(M.TORUS, 2, 10.0, 0.1, 2.0, 0.2, 3, n_stab=5)
    ch.sweep(3)
    S = ch.measure_tau([0, 37, ch.L], stable=True)
    eq = ch.measure()[1:6]
    assert np.abs(S[0] - eq).max() < 1e-10 * np.abs(eq).max()
    assert np.abs(S[2] - S[0]).max() < 1e-9 * np.abs(eq).max()
    assert np.all(S[1, 2:] < S[0, 2:])


def _stable_triple(QR, DR, WR, QL, DL, WL):
    Db, Ds = np.maximum, np.minimum
    J = (QR.conj().T @ QL) / Db(DR, 1)[:, None] / Db(DL, 1)[None, :] \
        + Ds(DR, 1)[:, None] * (WR @ WL.conj().T) * Ds(DL, 1)[None, :]
    Ji = np.linalg.inv(J)
    X = (QL / Db(DL, 1)[None, :]) @ Ji
    R = QR.conj().T / Db(DR, 1)[:, None]
    return X @ (Ds(DR, 1)[:, None] * WR), (WL.conj().T * Ds(DL, 1)[None, :]) @ Ji @ R, X @ R


@pytest.mark.parametrize("nphi,beta,nstab", [(4, 2.0, 5), (5, 1.3, 4), (4, 10.0, 10)])
def test_stabilisation_point_scheme(nphi, beta, nstab):
    """The scheme of the GPU's time-displaced measurement: the left UDV stack
    of B(beta, sp_k)^H built downward, the right UDV of B(sp_k, 0) advanced
    upward, the stable triple at each stabilisation point and plain
    propagation by one slice in between, reproduces the stable form at every
    slice (to 1e-12 at beta = 10)."""
    ch = O.Chain(M.TORUS, nphi, beta, 0.1, 1.5, 0.1, 3, n_stab=nstab)
    ch.sweep(2)
    N, L = ch.N, ch.L
    sp = list(range(nstab, L, nstab)) + [L]
    nsp = len(sp)
    LQ, LD, LW = [None] * (nsp + 1), [None] * (nsp + 1), [None] * (nsp + 1)
    LQ[nsp - 1], LD[nsp - 1], LW[nsp - 1] = np.eye(N), np.ones(N), np.eye(N)
    for k in range(nsp - 1, -1, -1):
        X = LQ[k] * LD[k][None, :]
        for t in range(sp[k], sp[k - 1] if k > 0 else 0, -1):
            X = ch.B(t)[0].conj().T @ X
        Q, D, V = O.udv(X)
        dst = k - 1 if k > 0 else nsp
        LQ[dst], LD[dst], LW[dst] = Q, D, V @ LW[k]
    RQ, RD, RW = np.eye(N, dtype=complex), np.ones(N), np.eye(N, dtype=complex)
    cur = _stable_triple(RQ, RD, RW, LQ[nsp], LD[nsp], LW[nsp])
    k, prev = 0, 0
    for t in range(L + 1):
        if t > 0:
            B, Bi = ch.B(t)
            if t == sp[k]:
                X = RQ * RD[None, :]
                for u in range(prev + 1, t + 1):
                    X = ch.B(u)[0] @ X
                Q, D, V = O.udv(X)
                RQ, RD, RW = Q, D, V @ RW
                cur = _stable_triple(RQ, RD, RW, LQ[k], LD[k], LW[k])
                prev, k = t, k + 1
            else:
                cur = (B @ cur[0], cur[1] @ Bi, B @ cur[2] @ Bi)
        ref = ch.green_tau_stable(t)
        for a, b in zip(cur, ref):
            assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(b).max()), t


def test_sphere_time_displaced_structure_factor_matches_ed():
    """Sphere n_orb = 2, u = 79, alpha = 15.8 (strong coupling, tests/sphere_units.py),
    beta = 2, dtau = 0.05: Monte
    Carlo S^1_0(tau) and S^3_0(tau) (l = 0) at tau = 0.1 and 0.25 within 4
    sigma of ED (the sphere's form factors in the time-displaced Wick
    contractions)."""
    m = M.Model(M.SPHERE, 2)
    beta, dtau = 2.0, 0.05
    us, als = sphere_u(1.0, 2), sphere_u(0.2, 2)
    ed = E.ED(m, M.couplings(us, als), beta)
    ch = O.Chain(M.SPHERE, 2, beta, dtau, us, als, seed=7, n_stab=5, n_adapt=150, model=m)
    ch.sweep(150)
    taus = [2, 5]
    rec = []
    for _ in range(2500):
        ch.sweep(1)
        rec.append(ch.measure_tau(taus))
    rec = np.array(rec)
    for k, t in enumerate(taus):
        for gi, col in ((0, 0), (2, 2)):
            ref = ed.structure_factor_tau(gi, 0, t * dtau)
            mu, err = _mean_err(rec[:, k, col])
            assert abs(mu - ref) < 4 * err and err < 0.3 * ref, (t, gi, mu, ref, err)
    assert ed.structure_factor_tau(0, 0, 0.25) < ed.structure_factor_tau(0, 0, 0.1)
