"""Model tables for the CF-DQMC oracle (plain numpy, FP64).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.

What is built here, and the passage each piece follows:

* couplings g_i of the Fierz-transformed Hamiltonian (Results, "Theoretical
  model ..."; Methods, Eq. newmodel): U_0 = 1, U_N = u + a/sqrt(2),
  U_K = u - a/sqrt(2) (Results, "Universal phase diagram"),
  g = (U_0 + U_N, -(U_K + U_N), -(U_K + U_N), 2 U_N).  The Methods copy of
  this equation writes "N_N" where U_N is meant; U_N is used.
* HS amplitudes alpha_i = sqrt(-dtau g_i) (Methods, Eq. hs_transform), taken
  as the principal complex square root: real for g_i <= 0, i*sqrt(dtau g_i)
  for g_i > 0.
* torus momenta and LLL form factors (Methods, Eq. torus_density_operator):
  all integer (q_x, q_y) with exp(-2 pi |q|^2 / (4 N_phi)) > 0.01, and
  (F_q)[k, k - q_y mod N_phi] = pref(q) exp(i/2 (2k - q_y) q_x 2 pi / N_phi)
  with k = 1..N_phi as in the paper, pref = exp(-2 pi |q|^2/(4 N_phi)) /
  (4 pi sqrt(N_phi)).
* sphere monopole-harmonic form factors (Methods,
  Eq. sphere_density_operator), with orbital label m_k = k - 1 - s
  substituted for the literal "k" inside the 3j symbol and the phase, with
  n_{l,-m} taken as n_{l,m}^dagger, and scaled by 1/(2 pi sqrt(n_orb)) so that
  the sphere carries the torus's normalisation (see ``sphere_form_factors``).
* the real-field parametrisation of the sum of squares (Methods,
  Eq. interaction_squares): for a self-conjugate q, Q = sqrt(2) n_q; for a
  pair (q, qbar) with F_qbar = F_q^dagger, Q_A = n_q + n_qbar and
  Q_B = i (n_q - n_qbar), so sum_q n_q n_qbar = sum Q^2 / 2 with exactly
  N_q real fields per channel.  In complex form z_q = phi_A + i phi_B,
  z_qbar = conj(z_q), z_q = sqrt(2) phi for self-conjugate q.
* the particle-hole background of channel 0 (Methods, Eq.
  torus_density_operator, term -2 delta_{q_y,0} delta_{i,0}):
  b_q = 2 Tr F_q, i.e. half of the four-flavour trace of F_q (x) I_4.

Field ordering (shared by nothing: the CUDA path derives it independently
from the same rule): walk K in its stored order; a self-conjugate q takes the
next field index, the first member q of a pair takes the next two (A, B).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

TORUS = 0
SPHERE = 1


# --------------------------------------------------------------------------
# couplings
# --------------------------------------------------------------------------
def couplings(u: float, anis: float) -> np.ndarray:
    """g_0..g_3 of H = sum_i g_i H_i (Eq. newmodel) from (u, alpha)."""
    un = u + anis / math.sqrt(2.0)
    uk = u - anis / math.sqrt(2.0)
    return np.array([1.0 + un, -(uk + un), -(uk + un), 2.0 * un])


def hs_alpha(g: np.ndarray, dtau: float) -> np.ndarray:
    """alpha_i = sqrt(-dtau g_i) (Eq. hs_transform), principal branch."""
    return np.sqrt((-dtau * np.asarray(g, dtype=float)).astype(complex))


# --------------------------------------------------------------------------
# torus
# --------------------------------------------------------------------------
def torus_momenta(nphi: int) -> list[tuple[int, int]]:
    """Integer (q_x, q_y) with exp(-2 pi (q_x^2+q_y^2)/(4 N_phi)) > 0.01.

    Order: q_y ascending (outer), q_x ascending (inner)."""
    r = int(math.isqrt(int(4 * nphi * math.log(100.0) / (2 * math.pi)))) + 2
    out = []
    for qy in range(-r, r + 1):
        for qx in range(-r, r + 1):
            if math.exp(-2 * math.pi * (qx * qx + qy * qy) / (4 * nphi)) > 0.01:
                out.append((qx, qy))
    return out


def torus_form_factors(nphi: int, qs):
    """val[q, row], col[q, row] of the shifted-diagonal F_q (Eq.
    torus_density_operator).  Row = orbital of c^dagger (k - 1), column =
    orbital of c (k - q_y mod N_phi)."""
    nq = len(qs)
    val = np.zeros((nq, nphi), dtype=complex)
    col = np.zeros((nq, nphi), dtype=np.int32)
    for iq, (qx, qy) in enumerate(qs):
        pref = math.exp(-2 * math.pi * (qx * qx + qy * qy) / (4 * nphi)) / (
            4 * math.pi * math.sqrt(nphi))
        for k in range(1, nphi + 1):
            ph = 0.5 * (2 * k - qy) * qx * (2 * math.pi / nphi)
            val[iq, k - 1] = pref * complex(math.cos(ph), math.sin(ph))
            col[iq, k - 1] = (k - 1 - qy) % nphi
    return val, col


def torus_partner(qs) -> np.ndarray:
    idx = {q: i for i, q in enumerate(qs)}
    return np.array([idx[(-qx, -qy)] for (qx, qy) in qs], dtype=np.int32)


# --------------------------------------------------------------------------
# sphere: exact Wigner 3j by the Racah formula in rational arithmetic
# --------------------------------------------------------------------------
_FACT = [1]


def _fact(n: int) -> int:
    while len(_FACT) <= n:
        _FACT.append(_FACT[-1] * len(_FACT))
    return _FACT[n]


def wigner3j(j1: Fraction, j2: Fraction, j3: Fraction,
             m1: Fraction, m2: Fraction, m3: Fraction) -> float:
    """Wigner 3j symbol from the Racah formula, evaluated exactly.

    All arguments are integers or half-integers (Fractions).  The value is
    s * sqrt(P) with s an exact rational sum and P an exact rational; it is
    returned as sign(s) * sqrt(s^2 P), so the only rounding is the final
    conversion to float."""
    j1, j2, j3, m1, m2, m3 = map(Fraction, (j1, j2, j3, m1, m2, m3))
    if m1 + m2 + m3 != 0:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    ints = [j1 + j2 - j3, j1 - j2 + j3, -j1 + j2 + j3, j1 + m1, j1 - m1,
            j2 + m2, j2 - m2, j3 + m3, j3 - m3, j1 + j2 + j3 + 1]
    for v in ints:
        if v.denominator != 1:
            return 0.0
    a, b, c, d, e, f, g, h, i, big = (int(v) for v in ints)
    # triangle coefficient times the (j +- m)! product
    P = Fraction(_fact(a) * _fact(b) * _fact(c), _fact(big))
    P *= _fact(d) * _fact(e) * _fact(f) * _fact(g) * _fact(h) * _fact(i)
    # Racah sum over t
    k1 = int(j3 - j2 + m1)
    k2 = int(j3 - j1 - m2)
    n1 = int(j1 + j2 - j3)
    n2 = int(j1 - m1)
    n3 = int(j2 + m2)
    tmin = max(0, -k1, -k2)
    tmax = min(n1, n2, n3)
    s = Fraction(0)
    for t in range(tmin, tmax + 1):
        den = (_fact(t) * _fact(k1 + t) * _fact(k2 + t) * _fact(n1 - t)
               * _fact(n2 - t) * _fact(n3 - t))
        s += Fraction((-1) ** t, den)
    ph = j1 - j2 - m3
    assert ph.denominator == 1
    if int(ph) % 2:
        s = -s
    if s == 0:
        return 0.0
    mag = math.sqrt(float(s * s * P))
    return mag if s > 0 else -mag


def sphere_momenta(norb: int) -> list[tuple[int, int]]:
    """(l, m) with l = 0..2s, m = -l..l, 2s + 1 = norb: N_q = norb^2."""
    return [(l, m) for l in range(norb) for m in range(-l, l + 1)]


def sphere_form_factors(norb: int, qs):
    """F_{l,m}[k, k+m] (Eq. sphere_density_operator).

    Reading of the garbled passage: the orbital label inside the 3j symbol and
    the phase is m_k = k - 1 - s (the paper's "k"), so for 0-based row r,
    m_k = r - s and the phase (-1)^{s + m_k + m} = (-1)^{r + m}.  The paper's
    formula obeys F_{l,-m} = (-1)^m F_{l,m}^dagger; the rotation-invariant
    interaction sum_m n_{l,m} n_{l,m}^dagger is used, i.e. for m < 0 the table
    holds F_{l,|m|}^dagger.

    Normalisation.  As printed, F_{0,0} = (-1)^{2s}/2 I and (3j orthogonality)
    sum_q ||F_q||_F^2 = n_orb^2 / 4: the weight per orbital grows with the
    system, so the effective coupling would grow with n_orb.  The
    torus of Eq. torus_density_operator has F_0 = I / (4 pi sqrt(N_phi)) and
    a size-independent weight 1/(16 pi^2) per orbital, and the paper finds
    one critical coupling for all sphere sizes N_phi = 15..59 (u_c ~ 0.17,
    finite-size scaling in Results), close to the torus's 0.20 (Supp.
    Fig. S4): both need a size-independent scale, matching the torus's.  Reading: the printed expression times 1/(2 pi sqrt(n_orb)),
    which makes F_{0,0} = (-1)^{2s} I / (4 pi sqrt(n_orb)) and the weight
    exactly 1/(16 pi^2) per orbital, the torus's values."""
    s2 = norb - 1                      # 2s
    s = Fraction(s2, 2)
    nq = len(qs)
    val = np.zeros((nq, norb), dtype=complex)
    col = np.full((nq, norb), -1, dtype=np.int32)
    kappa = 1.0 / (2.0 * math.pi * math.sqrt(norb))
    red = {}
    for l in range(norb):
        red[l] = wigner3j(s, l, s, -s, 0, s)
    cache = {}
    for iq, (l, m) in enumerate(qs):
        if m >= 0:
            for r in range(norb):
                c = r + m
                if c >= norb:
                    continue
                mk = Fraction(r) - s
                w = wigner3j(s, l, s, -mk, -m, mk + m)
                sign = -1.0 if (r + m) % 2 else 1.0
                v = sign * (s2 + 1) * math.sqrt(2 * l + 1) / 2.0 * w * red[l] * kappa
                val[iq, r] = v
                col[iq, r] = c
            cache[(l, m)] = iq
    for iq, (l, m) in enumerate(qs):
        if m < 0:
            jp = cache[(l, -m)]
            # adjoint of a shifted-diagonal matrix: entry (r, r+|m|) -> (r+|m|, r)
            for r in range(norb):
                c = col[jp, r]
                if c >= 0:
                    val[iq, c] = np.conj(val[jp, r])
                    col[iq, c] = r
    return val, col


def sphere_partner(qs) -> np.ndarray:
    idx = {q: i for i, q in enumerate(qs)}
    return np.array([idx[(l, -m)] for (l, m) in qs], dtype=np.int32)


# --------------------------------------------------------------------------
# assembled model
# --------------------------------------------------------------------------
class Model:
    """Everything the oracle sweep needs besides the couplings and seeds."""

    def __init__(self, geom: int, size: int):
        self.geom = geom
        if geom == TORUS:
            self.norb = size
            self.qs = torus_momenta(size)
            self.val, self.col = torus_form_factors(size, self.qs)
            self.partner = torus_partner(self.qs)
        elif geom == SPHERE:
            self.norb = size
            self.qs = sphere_momenta(size)
            self.val, self.col = sphere_form_factors(size, self.qs)
            self.partner = sphere_partner(self.qs)
        else:
            raise ValueError(geom)
        self.nq = len(self.qs)
        self.N = 2 * self.norb
        self.field_map = field_map(self.partner)
        self.bg = 2.0 * np.array([self.trace_F(q) for q in range(self.nq)])

    def dense_F(self, q: int) -> np.ndarray:
        F = np.zeros((self.norb, self.norb), dtype=complex)
        for r in range(self.norb):
            c = self.col[q, r]
            if c >= 0:
                F[r, c] += self.val[q, r]
        return F

    def trace_F(self, q: int) -> complex:
        return complex(np.trace(self.dense_F(q)))

    def delta_q(self) -> list[int]:
        """Indices of the smallest non-zero momenta used by the correlation
        ratio: torus (+-1, 0), (0, +-1); sphere l = 1, all m."""
        if self.geom == TORUS:
            want = {(1, 0), (-1, 0), (0, 1), (0, -1)}
        else:
            want = {(1, -1), (1, 0), (1, 1)}
        return [i for i, q in enumerate(self.qs) if q in want]

    def q0(self) -> int:
        return self.qs.index((0, 0))


def field_map(partner: np.ndarray):
    """Per q: (kind, rA, rB).  kind 0: self-conjugate, z = sqrt(2) phi[rA];
    kind 1: first of a pair, z = phi[rA] + i phi[rB]; kind 2: second of a
    pair, z = phi[rA] - i phi[rB]."""
    nq = len(partner)
    out = [None] * nq
    r = 0
    for q in range(nq):
        p = int(partner[q])
        if p == q:
            out[q] = (0, r, -1)
            r += 1
        elif p > q:
            out[q] = (1, r, r + 1)
            out[p] = (2, r, r + 1)
            r += 2
    assert r == nq
    return out


def z_from_phi(model: Model, phi_c: np.ndarray) -> np.ndarray:
    """z_q for one channel from its N_q real fields."""
    z = np.zeros(model.nq, dtype=complex)
    for q, (kind, a, b) in enumerate(model.field_map):
        if kind == 0:
            z[q] = math.sqrt(2.0) * phi_c[a]
        elif kind == 1:
            z[q] = phi_c[a] + 1j * phi_c[b]
        else:
            z[q] = phi_c[a] - 1j * phi_c[b]
    return z
