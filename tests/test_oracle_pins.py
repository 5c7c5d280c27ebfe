"""Pins of the FP64 oracle against things other than itself.

Each test fixes one piece of the oracle with something the paper or the
mathematics determines independently: published known-answer vectors, the
magnetic-translation algebra, exact 3j symbols, operator identities on a
Fock space, brute-force determinants, finite differences, closed forms at zero
coupling, and library routines.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as st

from oracle import model as M
from oracle import oracle as O
from tests.sphere_units import sphere_u

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ RNG ----
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        assert O.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


def test_box_muller_normals_are_standard():
    x = np.concatenate([O.normals(s, 3, 7, 1, 50000) for s in range(4)])
    assert abs(x.mean()) < 5 / math.sqrt(len(x))
    assert abs(x.var() - 1) < 5 * math.sqrt(2.0 / len(x))
    assert st.kstest(x, "norm").pvalue > 1e-4
    # different purposes / sweeps give independent streams
    a = O.normals(0, 0, 0, 0, 2000)
    b = O.normals(0, 0, 0, 1, 2000)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.1


# --------------------------------------------------------- form factors ---
@pytest.mark.parametrize("nphi", [2, 3, 4, 8, 36, 140])
def test_torus_momentum_set_is_the_gaussian_disk(nphi):
    qs = M.torus_momenta(nphi)
    r = 60
    qx, qy = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1))
    inside = np.exp(-2 * np.pi * (qx ** 2 + qy ** 2) / (4 * nphi)) > 0.01
    assert len(qs) == int(inside.sum())
    assert len(set(qs)) == len(qs)
    assert all((-a, -b) in set(qs) for a, b in qs)


def _T(nphi, q):
    """magnetic translation F_q / pref(q) as a dense matrix"""
    val, col = M.torus_form_factors(nphi, [q])
    pref = math.exp(-2 * math.pi * (q[0] ** 2 + q[1] ** 2) / (4 * nphi)) / (4 * math.pi * math.sqrt(nphi))
    T = np.zeros((nphi, nphi), complex)
    for r in range(nphi):
        T[r, col[0, r]] = val[0, r] / pref
    return T


@pytest.mark.parametrize("nphi", [3, 5, 8])
def test_torus_form_factor_obeys_magnetic_translation_algebra(nphi):
    """Girvin-MacDonald-Platzman algebra: T_q T_q' = exp(i q^q'/2) T_{q+q'}
    with q^q' = (2 pi / N_phi)(q_x q'_y - q_y q'_x).  A wrong sign or factor
    in the phase of the torus form factor breaks it."""
    rng = np.random.default_rng(nphi)
    for _ in range(20):
        q = tuple(int(v) for v in rng.integers(-4, 5, 2))
        p = tuple(int(v) for v in rng.integers(-4, 5, 2))
        lhs = _T(nphi, q) @ _T(nphi, p)
        wedge = 2 * math.pi / nphi * (q[0] * p[1] - q[1] * p[0])
        rhs = np.exp(0.5j * wedge) * _T(nphi, (q[0] + p[0], q[1] + p[1]))
        assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("geom,size", [(M.TORUS, 4), (M.TORUS, 7), (M.SPHERE, 3), (M.SPHERE, 4)])
def test_density_operators_hermitian_pairs(geom, size):
    m = M.Model(geom, size)
    for q in range(m.nq):
        assert np.abs(m.dense_F(q).conj().T - m.dense_F(int(m.partner[q]))).max() < 1e-14


@pytest.mark.parametrize("nphi", [4, 9])
def test_torus_form_factor_is_scaled_unitary(nphi):
    m = M.Model(M.TORUS, nphi)
    for q, (qx, qy) in enumerate(m.qs):
        pref = math.exp(-2 * math.pi * (qx * qx + qy * qy) / (4 * nphi)) / (4 * math.pi * math.sqrt(nphi))
        F = m.dense_F(q)
        assert np.abs(F @ F.conj().T - pref ** 2 * np.eye(nphi)).max() < 1e-15


def test_wigner3j_matches_sympy():
    from fractions import Fraction as Fr
    from sympy.physics.wigner import wigner_3j
    cases = []
    for j2 in range(0, 5):
        for s2 in (1, 3, 5):
            s = Fr(s2, 2)
            for m1 in [Fr(k, 2) for k in range(-s2, s2 + 1, 2)]:
                for m2 in range(-j2, j2 + 1):
                    cases.append((s, j2, s, -m1, -m2, m1 + m2))
    for c in cases:
        ref = float(wigner_3j(*[x if isinstance(x, int) else __import__("sympy").Rational(x.numerator, x.denominator) for x in c]))
        assert abs(M.wigner3j(*c) - ref) < 1e-14


@pytest.mark.parametrize("norb", [3, 4, 7])
def test_sphere_F00_closed_form_and_rotation_invariance(norb):
    """F_{0,0} = (-1)^{2s} I / (4 pi sqrt(n_orb)), the torus's q = 0 table
    (the printed (-1)^{2s} I / 2 times the normalisation 1/(2 pi sqrt(n_orb)));
    sum_m F_{l,m} F_{l,m}^dagger is proportional to the identity for every l
    (rotation invariance, the addition theorem for the monopole-harmonic
    matrix elements)."""
    m = M.Model(M.SPHERE, norb)
    s2 = norb - 1
    F00 = m.dense_F(m.qs.index((0, 0)))
    assert np.abs(F00 - ((-1) ** s2) / (4 * math.pi * math.sqrt(norb)) * np.eye(norb)).max() < 1e-15
    for l in range(norb):
        S = sum(m.dense_F(m.qs.index((l, mm))) @ m.dense_F(m.qs.index((l, mm))).conj().T
                for mm in range(-l, l + 1))
        assert np.abs(S - S[0, 0] * np.eye(norb)).max() < 1e-12 * max(1, abs(S[0, 0]))


@pytest.mark.parametrize("norb", [2, 5, 8])
def test_sphere_weight_per_orbital_matches_the_torus(norb):
    """sum_q ||F_q||_F^2 / n_orb = 1/(16 pi^2) exactly on the sphere: for each
    l, sum_m of the squared 3j symbols (s l s; -m_k -m m_k+m) over the pairs
    is 1/(2s+1) per row (3j orthogonality), and sum_l (2l+1)
    (s l s; -s 0 s)^2 = 1.  On the torus the same sum is
    sum_q pref(q)^2 = 1/(16 pi^2) up to the cut of the Gaussian (~1e-4 at
    N_phi >= 8), so both geometries carry the same weight per orbital at
    every size."""
    m = M.Model(M.SPHERE, norb)
    w = sum(np.linalg.norm(m.dense_F(q)) ** 2 for q in range(m.nq)) / norb
    assert abs(w * 16 * math.pi ** 2 - 1) < 1e-13
    t = M.Model(M.TORUS, 4 * norb)
    wt = sum(np.linalg.norm(t.dense_F(q)) ** 2 for q in range(t.nq)) / t.norb
    assert abs(wt * 16 * math.pi ** 2 - 1) < 1e-3


def test_background_is_half_the_four_flavour_trace():
    """b_q = 2 Tr F_q; on the torus for N_phi >= 3 only q = 0 carries it and
    it equals the literal 2 N_phi pref(0) of Eq. torus_density_operator."""
    for nphi in (3, 4, 8):
        m = M.Model(M.TORUS, nphi)
        nz = [q for q in range(m.nq) if abs(m.bg[q]) > 1e-14]
        assert nz == [m.q0()]
        assert abs(m.bg[m.q0()] - 2 * nphi / (4 * math.pi * math.sqrt(nphi))) < 1e-14


# ---------------------------------------------------- operator identities --
def _jw(nmodes):
    """Jordan-Wigner annihilators on a 2^nmodes Fock space."""
    a = np.array([[0, 1], [0, 0]], complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    I2 = np.eye(2, dtype=complex)
    cs = []
    for x in range(nmodes):
        ops = [Z] * x + [a] + [I2] * (nmodes - x - 1)
        m = ops[0]
        for o in ops[1:]:
            m = np.kron(m, o)
        cs.append(m)
    return cs


def _bilinear(cs, h):
    out = 0
    for x in range(len(cs)):
        for y in range(len(cs)):
            if h[x, y] != 0:
                out = out + h[x, y] * cs[x].conj().T @ cs[y]
    return out


def test_fierz_identity_fixes_the_couplings():
    """On one orbital (valley x spin, 4 modes): the Gamma-form interaction of
    Eq. model equals sum_i g_i (c^dag O^i c - 2 delta_i0)^2 up to a constant,
    with the g_i of Eq. newmodel."""
    cs = _jw(4)
    P = {k: v for k, v in zip("Ixyz", [np.eye(2), [[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]])}
    T = lambda a, b: np.kron(np.array(P[a], complex), np.array(P[b], complex))  # valley (x) spin
    n = lambda A: _bilinear(cs, A)
    Id = np.eye(16)
    for u, al in [(1.0, 0.0), (0.7, 0.3), (2.0, -0.2)]:
        UN, UK = u + al / math.sqrt(2), u - al / math.sqrt(2)
        H = (n(T("I", "I")) - 2 * Id) @ (n(T("I", "I")) - 2 * Id)
        H = H - UK * (n(T("x", "I")) @ n(T("x", "I")) + n(T("y", "I")) @ n(T("y", "I")))
        H = H - UN * sum(n(T("z", s)) @ n(T("z", s)) for s in "xyz")
        g = M.couplings(u, al)
        Hf = sum(g[i] * (n(T(v, "I")) - (2 * Id if i == 0 else 0)) @ (n(T(v, "I")) - (2 * Id if i == 0 else 0))
                 for i, v in enumerate("Ixyz"))
        D = H - Hf
        assert np.abs(D - D[0, 0] * Id).max() < 1e-12


@pytest.mark.parametrize("g", [1.3, -0.7])
def test_hs_identity_by_quadrature(g):
    """int dphi e^{-phi^2/2}/sqrt(2 pi) e^{alpha phi Q} = e^{-dtau g Q^2/2}
    with alpha = sqrt(-dtau g) (Eq. hs_transform), for both signs of g."""
    rng = np.random.default_rng(1)
    A = rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))
    Q = (A + A.conj().T) / 4
    dtau = 0.1
    alpha = M.hs_alpha(np.array([g]), dtau)[0]
    x, w = np.polynomial.hermite_e.hermegauss(80)
    lhs = sum(wk * sla.expm(alpha * xk * Q) for xk, wk in zip(x, w)) / math.sqrt(2 * math.pi)
    rhs = sla.expm(-dtau * g * Q @ Q / 2)
    assert np.abs(lhs - rhs).max() < 1e-12


def test_sum_of_squares_field_parametrisation():
    """sum_q n_q n_qbar = sum_r Q_r^2 / 2 with Q_r = d(sum_q z_q n_q)/d phi_r,
    i.e. the z_q(phi) map of the real fields reproduces Eq.
    interaction_squares with exactly N_q real fields per channel."""
    for geom, size in [(M.TORUS, 2), (M.SPHERE, 2)]:
        m = M.Model(geom, size)
        cs = _jw(m.N)
        nq = [_bilinear(cs, np.kron(np.array([[0, 1], [1, 0]], complex), m.dense_F(q))) for q in range(m.nq)]
        lhs = sum(nq[q] @ nq[int(m.partner[q])] for q in range(m.nq))
        rhs = 0
        for r in range(m.nq):
            e = np.zeros(m.nq)
            e[r] = 1.0
            z = M.z_from_phi(m, e)
            Qr = sum(z[q] * nq[q] for q in range(m.nq))
            assert np.abs(Qr - Qr.conj().T).max() < 1e-13
            rhs = rhs + Qr @ Qr / 2
        assert np.abs(lhs - rhs).max() < 1e-12


def _fock_log_bracket(ch, m, dtau, g):
    """log of Tr_Fock prod_t prod_j e^{c^dag X_j c} * prod_t e^{-Tr W0/2} for
    one spin block, built independently of the oracle from the model tables."""
    cs = _jw(m.N)
    alpha = M.hs_alpha(g, dtau)
    Ov = [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.diag([1, -1])]
    order = [(0, .5), (1, .5), (2, .5), (3, 1.0), (2, .5), (1, .5), (0, .5)]
    phi = ch.phi()
    U = np.eye(2 ** m.N, dtype=complex)
    bg = 0
    for t in range(ch.L):
        W = []
        for i in range(4):
            z = M.z_from_phi(m, phi[t, i])
            F = sum(z[q] * m.dense_F(q) for q in range(m.nq))
            W.append(alpha[i] * np.kron(Ov[i], F))
        Bt = np.eye(2 ** m.N, dtype=complex)
        for i, c in order:
            Bt = Bt @ sla.expm(_bilinear(cs, c * W[i]))
        U = Bt @ U
        bg += -0.5 * np.trace(W[0])
    return np.log(np.trace(U)) + bg


@pytest.mark.parametrize("u,al", [(1.0, 0.0), (3.0, 0.2)])
def test_determinant_equals_fock_trace_and_is_real(u, al):
    """det(1 + B(beta,0)) = Tr_Fock prod e^{c^dag X c} for one spin block,
    with the seven-factor symmetric slice of Eq. trotter_decomposition; the
    bracket including the background is real (sign-free weight)."""
    m = M.Model(M.TORUS, 2)
    ch = O.Chain(M.TORUS, 2, 0.3, 0.1, u, al, seed=5, model=m)
    lb = ch.log_bracket()
    ref = _fock_log_bracket(ch, m, 0.1, M.couplings(u, al))
    assert abs(lb.real - ref.real) < 1e-10
    assert abs(math.sin(lb.imag)) < 1e-10
    assert abs(math.sin(ref.imag)) < 1e-10


@pytest.mark.parametrize("geom,size,u,al", [(M.TORUS, 4, 5.0, 0.3), (M.TORUS, 3, 0.5, -0.2), (M.SPHERE, 3, sphere_u(1.0, 3), sphere_u(0.1, 3))])
def test_weight_is_sign_free_on_random_fields(geom, size, u, al):
    for seed in range(3):
        ch = O.Chain(geom, size, 1.0, 0.1, u, al, seed=seed)
        lb = ch.log_bracket()
        assert abs(math.sin(lb.imag)) < 1e-9


# ---------------------------------------------------------- derivatives ---
@pytest.mark.parametrize("geom,size,u,al,t", [(M.TORUS, 2, 2.0, 0.3, 2), (M.TORUS, 4, 1.0, 0.0, 3), (M.SPHERE, 2, sphere_u(1.0, 2), sphere_u(0.2, 2), 1)])
def test_gradient_matches_finite_differences(geom, size, u, al, t):
    ch = O.Chain(geom, size, 0.5, 0.1, u, al, seed=11)
    g = ch.gradient(t)
    p0 = ch.phi()[t - 1].copy()

    def S():
        return 0.5 * np.sum(ch.phi() ** 2) - 2 * ch.log_bracket().real
    h = 1e-5
    fd = np.zeros_like(g)
    for i in range(4):
        for r in range(ch.nq):
            p = p0.copy(); p[i, r] += h; ch.set_slice_phi(t, p); sp = S()
            p = p0.copy(); p[i, r] -= h; ch.set_slice_phi(t, p); sm = S()
            fd[i, r] = (sp - sm) / (2 * h)
    ch.set_slice_phi(t, p0)
    assert np.abs(fd - g).max() < 1e-6 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("u,al", [(1.0, 0.0), (4.0, -0.3)])
def test_ratio_and_green_update_match_brute_force(u, al):
    """log R via M = 1 + (Delta-1)(1-G) equals the brute-force log ratio of
    determinants, and G M^-1 equals the brute-force new Green's function."""
    ch = O.Chain(M.TORUS, 4, 1.0, 0.1, u, al, seed=2)
    rng = np.random.default_rng(0)
    for t in (1, 4, 10):
        before = ch.log_bracket()
        p0 = ch.phi()[t - 1].copy()
        p1 = p0 + 0.3 * rng.normal(size=p0.shape)
        logR, Gp = ch.ratio_at(t, p1)
        ch.set_slice_phi(t, p1)
        after = ch.log_bracket()
        assert abs(logR.real - (after - before).real) < 1e-10
        assert abs(math.sin(logR.imag)) < 1e-10
        Gb = ch.green_bruteforce(t)
        assert np.abs(Gp - Gb).max() < 1e-10 * np.abs(Gb).max()


def test_stabilised_green_matches_brute_force_and_stays_fresh():
    ch = O.Chain(M.TORUS, 4, 2.0, 0.1, 3.0, 0.2, seed=4, n_stab=5)
    obs = ch.sweep(5)
    assert np.abs(ch.green() - ch.green_bruteforce(ch.L)).max() < 1e-11
    assert obs[:, 15].max() < 1e-9          # |G_wrap - G_stable| / max|G|
    # long beta: stabilisation keeps the wrapped G within 1e-9 of a fresh one
    ch2 = O.Chain(M.SPHERE, 3, 20.0, 0.1, sphere_u(1.0, 3), 0.0, seed=1, n_stab=10)
    obs2 = ch2.sweep(1)
    assert obs2[:, 15].max() < 1e-8
    assert obs2[:, 16].max() < 1e-8


def test_linear_algebra_helpers_against_numpy():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(9, 9)) + 1j * rng.normal(size=(9, 9))
    H = A + A.conj().T
    w, V = O.eigh(H)
    assert np.abs(np.sort(w) - np.linalg.eigvalsh(H)).max() < 1e-12
    assert np.abs(V @ np.diag(w) @ V.conj().T - H).max() < 1e-12
    Q, D, W = O.udv(A)
    assert np.abs(Q @ np.diag(D) @ W - A).max() < 1e-12
    assert np.abs(Q.conj().T @ Q - np.eye(9)).max() < 1e-13
    assert np.all(np.diff(D) <= 1e-12)
    sign, ld = np.linalg.slogdet(A)
    got = O.logdet(A)
    assert abs(got.real - ld) < 1e-12
    assert abs(np.exp(1j * got.imag) - sign) < 1e-12


# ------------------------------------------------------- closed forms ------
def test_zero_coupling_closed_form():
    """All g_i = 0: B = 1, G = 1/2, every ratio is 1, S^i_q = N_phi pref(q)^2
    and m^2 = 1 / (16 pi^2 N_phi^2); the MH log-acceptance of every proposal
    equals the closed form of MALA on a standard Gaussian target."""
    nphi = 4
    ch = O.Chain(M.TORUS, nphi, 2.0, 0.1, 0, 0, seed=9, g=np.zeros(4), eps0=0.6, n_adapt=0)
    assert np.abs(ch.green() - 0.5 * np.eye(2 * nphi)).max() < 1e-13
    ch.enable_trace(100)
    obs = ch.sweep(1)[0]
    pref0 = 1 / (4 * math.pi * math.sqrt(nphi))
    assert abs(obs[0] - 1 / (16 * math.pi ** 2 * nphi ** 2)) < 1e-15
    assert np.allclose(obs[1:6], nphi * pref0 ** 2, rtol=1e-13, atol=0)
    pref1 = math.exp(-2 * math.pi / (4 * nphi)) / (4 * math.pi * math.sqrt(nphi))
    assert np.allclose(obs[6:11], nphi * pref1 ** 2, rtol=1e-13, atol=0)
    tr = ch.trace()
    assert np.abs(tr[:, 2]).max() < 1e-13
    nf = 4 * ch.nq
    eps = 0.6
    for row in tr:
        t = int(row[1])
        phi = O.normals(9, t - 1, 0, 0, nf)
        xi = O.normals(9, t - 1, 0, 1, nf)
        php = phi - 0.5 * eps ** 2 * phi + eps * xi
        fw = np.sum((php - phi + 0.5 * eps ** 2 * phi) ** 2)
        bw = np.sum((phi - php + 0.5 * eps ** 2 * php) ** 2)
        logA = -0.5 * (np.sum(php ** 2) - np.sum(phi ** 2)) - bw / (2 * eps ** 2) + fw / (2 * eps ** 2)
        assert abs(row[4] - logA) < 1e-10 * max(1, abs(logA))
        assert row[6] == (row[5] < row[4])


def test_zero_coupling_samples_standard_normal():
    ch = O.Chain(M.TORUS, 2, 1.0, 0.1, 0, 0, seed=3, g=np.zeros(4), n_adapt=50)
    ch.sweep(50)
    xs = []
    for _ in range(300):
        ch.sweep(1)
        xs.append(ch.phi().ravel())
    x = np.array(xs)
    assert abs(x.mean()) < 0.03
    assert abs(x.var() - 1) < 0.05


# ------------------------------------------------------ checkpointing ---
@pytest.mark.parametrize("n_adapt", [-1, 6])
def test_resumed_chain_is_bit_identical(n_adapt):
    """Fields, step and sweep index are the whole state: a chain rebuilt from
    a checkpoint continues exactly as the uninterrupted one (Philox is
    counter based; propagators and G are recomputed as the sweep does)."""
    a = O.Chain(M.TORUS, 3, 1.0, 0.1, 2.0, 0.1, 9, n_stab=4, n_adapt=n_adapt)
    a.sweep(4)
    st = a.get_state()
    ref = a.sweep(5)
    b = O.Chain(M.TORUS, 3, 1.0, 0.1, 2.0, 0.1, 9, n_stab=4, n_adapt=n_adapt)
    b.set_state(st)
    got = b.sweep(5)
    assert np.array_equal(got, ref)
    assert np.array_equal(a.phi(), b.phi()) and a.eps == b.eps
    with pytest.raises(ValueError):
        b.set_state(st[:-1])


def test_momentum_counts():
    """N_q = (N_phi + 1)^2 = n_orb^2 on the sphere (all angular momentum
    channels) and N_q proportional to N_phi on the torus: the disk
    e^{-2 pi |q|^2 / (4 N_phi)} > 0.01 has area 2 N_phi ln 100
    (Results, model section; Methods, toric and spherical regularisation)."""
    for norb in (2, 3, 7, 16):
        assert len(M.sphere_momenta(norb)) == norb ** 2
    for nphi, nq in ((4, 37), (36, 333)):
        assert len(M.torus_momenta(nphi)) == nq
    r = [len(M.torus_momenta(n)) / n for n in (36, 64, 140)]
    assert all(abs(x / (2 * math.log(100.0)) - 1) < 0.02 for x in r), r


def test_sign_free_region_is_u_n_nonnegative():
    """The weight is sign-free wherever U_N = u + alpha/sqrt(2) >= 0, U_K
    of either sign (g_1 = g_2 = -2u <= 0, g_0, g_3 >= 0); with U_N < 0 the
    bracket acquires a phase, which is why qmc_create rejects that region."""
    rng = np.random.default_rng(12)
    for _ in range(6):
        u = rng.uniform(0.05, 3.0)
        al = rng.uniform(-math.sqrt(2) * u, 3.0)
        ch = O.Chain(M.TORUS, 3, 1.0, 0.1, u, al, seed=int(rng.integers(100)))
        assert abs(math.sin(ch.log_bracket().imag)) < 1e-10, (u, al)
    for u, al in ((1.0, -2.0), (0.2, -0.5)):
        assert u + al / math.sqrt(2) < 0
        devs = [abs(math.sin(O.Chain(M.TORUS, 3, 1.0, 0.1, u, al, seed=s).log_bracket().imag))
                for s in range(3)]
        assert max(devs) > 1e-5, (u, al, devs)
