"""ctypes front end of the plain FP64 CPU oracle (``cfdqmc_oracle.c``).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never imports the
product package and the product package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import model as M

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cfdqmc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
NOBS = 20
NTRACE = 8
OBS_NAMES = ["m2", "S1_0", "S2_0", "S3_0", "S4_0", "S5_0", "S1_dq", "S2_dq",
             "S3_dq", "S4_dq", "S5_dq", "R", "E", "acc", "eps", "stab_err",
             "sign_dev", "n_acc", "_", "_"]

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (portable flags, no -march)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fcx-limited-range", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, dp, ip, ip, C.c_int, C.c_int,
                                 C.c_double, dp, C.c_uint64, C.c_double, C.c_double,
                                 C.c_double, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_sweep.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_sweep_learned.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, dp, C.c_double]
        L.orc_mlp_forward.argtypes = [C.c_int, C.c_int, dp, C.c_int, dp, dp]
        L.orc_green_tau.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.orc_green_tau_stable.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        L.orc_measure_tau.argtypes = [C.c_void_p, C.c_int, ip, dp]
        L.orc_measure_tau_stable.argtypes = [C.c_void_p, C.c_int, ip, dp]
        L.orc_measure.argtypes = [C.c_void_p, dp]
        L.orc_set_measure_q.argtypes = [C.c_void_p, C.c_int, ip, C.c_int]
        L.orc_set_skip_energy.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_trace.argtypes = [C.c_void_p, dp, C.c_long]
        L.orc_trace_count.restype = C.c_long
        L.orc_trace_count.argtypes = [C.c_void_p]
        L.orc_get_green.argtypes = [C.c_void_p, dp]
        L.orc_get_phi.argtypes = [C.c_void_p, dp]
        L.orc_get_eps.restype = C.c_double
        L.orc_get_eps.argtypes = [C.c_void_p]
        L.orc_set_eps.argtypes = [C.c_void_p, C.c_double]
        L.orc_get_sweep.restype = C.c_uint
        L.orc_get_sweep.argtypes = [C.c_void_p]
        L.orc_get_B.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_set_slice_phi.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_log_bracket.argtypes = [C.c_void_p, dp]
        L.orc_green_bruteforce.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_gradient_at.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_slice_factors.restype = C.c_int
        L.orc_slice_factors.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_state_size.restype = C.c_long
        L.orc_state_size.argtypes = [C.c_void_p]
        L.orc_get_state.argtypes = [C.c_void_p, dp]
        L.orc_set_state.argtypes = [C.c_void_p, dp]
        L.orc_set_variant.restype = C.c_int
        L.orc_set_variant.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_fields_per_slice.restype = C.c_int
        L.orc_fields_per_slice.argtypes = [C.c_void_p]
        L.orc_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                  C.c_int, dp]
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                        C.POINTER(C.c_uint32)]
        L.orc_eigh.argtypes = [C.c_int, dp, dp, dp]
        L.orc_udv.argtypes = [C.c_int, dp, dp, dp, dp]
        L.orc_logdet.argtypes = [C.c_int, dp, dp]
        L.orc_ratio_at.argtypes = [C.c_void_p, C.c_int, dp, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _cplx(a):
    return np.ascontiguousarray(a).view(np.complex128)


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def normals(seed, slice_, sweep, purpose, n):
    out = np.zeros(n)
    lib().orc_normals(seed, slice_, sweep, purpose, n, _dp(out))
    return out


def eigh(H):
    H = np.ascontiguousarray(H, dtype=complex)
    n = H.shape[0]
    V = np.zeros((n, n), complex)
    w = np.zeros(n)
    lib().orc_eigh(n, _dp(H.view(float)), _dp(V.view(float)), _dp(w))
    return w, V


def udv(X):
    X = np.ascontiguousarray(X, dtype=complex)
    n = X.shape[0]
    Q = np.zeros((n, n), complex)
    V = np.zeros((n, n), complex)
    D = np.zeros(n)
    lib().orc_udv(n, _dp(X.view(float)), _dp(Q.view(float)), _dp(D), _dp(V.view(float)))
    return Q, D, V


def logdet(A):
    A = np.ascontiguousarray(A, dtype=complex)
    out = np.zeros(2)
    lib().orc_logdet(A.shape[0], _dp(A.view(float)), _dp(out))
    return complex(out[0], out[1])


SLICE_SYM, SLICE_SINGLE, SLICE_INDEP = 0, 1, 2
DRIFT_EXACT, DRIFT_FIRST = 0, 1


class Chain:
    """One Markov chain of the oracle.

    geom/size select the model (torus N_phi or sphere orbital count);
    u, anis give the couplings; L = beta/dtau slices.  slice_kind picks the
    discretisation of a slice (SLICE_SYM: the paper's seven factors with
    shared fields; SLICE_SINGLE: one exponential of the four channels;
    SLICE_INDEP: seven factors with a field set each) and drift_kind the
    Langevin drift (DRIFT_EXACT, or DRIFT_FIRST: each factor's derivative
    taken as Tr[(1-G) dX])."""

    def __init__(self, geom, size, beta, dtau, u, anis, seed, n_stab=5,
                 eps0=0.5, deps=0.1, r0=0.574, n_adapt=-1, g=None, model=None,
                 slice_kind=SLICE_SYM, drift_kind=DRIFT_EXACT):
        self.model = model if model is not None else M.Model(geom, size)
        L = int(round(beta / dtau))
        if abs(L * dtau - beta) > 1e-9 * max(1.0, beta):
            raise ValueError("beta / dtau is not an integer")
        self.L = L
        self.dtau = dtau
        self.g = np.asarray(g if g is not None else M.couplings(u, anis), float)
        m = self.model
        self.nq, self.norb, self.N = m.nq, m.norb, m.N
        self._ffval = np.ascontiguousarray(m.val, dtype=complex)
        self._ffcol = np.ascontiguousarray(m.col, dtype=np.int32)
        self._partner = np.ascontiguousarray(m.partner, dtype=np.int32)
        self._g = np.ascontiguousarray(self.g)
        self.h = lib().orc_create(m.norb, m.nq, _dp(self._ffval.view(float)),
                                  _ip(self._ffcol), _ip(self._partner), L, n_stab,
                                  dtau, _dp(self._g), seed, eps0, deps, r0, n_adapt)
        if (slice_kind, drift_kind) != (SLICE_SYM, DRIFT_EXACT):
            if lib().orc_set_variant(self.h, slice_kind, drift_kind) != 0:
                raise ValueError("unknown slice or drift variant")
        self.slice_kind, self.drift_kind = slice_kind, drift_kind
        self.nfs = lib().orc_fields_per_slice(self.h) // m.nq
        dq = np.array(m.delta_q(), dtype=np.int32)
        lib().orc_set_measure_q(self.h, m.q0() if m.geom == M.TORUS else 0,
                                _ip(dq), len(dq))
        self._trace = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def enable_trace(self, cap):
        self._trace = np.zeros((cap, NTRACE))
        lib().orc_set_trace(self.h, _dp(self._trace), cap)

    def trace(self):
        n = lib().orc_trace_count(self.h)
        return self._trace[:n].copy()

    def sweep(self, n=1):
        obs = np.zeros((n, NOBS))
        lib().orc_sweep(self.h, n, _dp(obs))
        return obs

    def sweep_learned(self, n, theta, H, rho):
        """n sweeps of learned slice moves (oracle/learned.py) with the
        network parameters theta (packed FP64) of hidden width H."""
        if self.L < 2:
            raise ValueError("learned moves need L >= 2")
        theta = np.ascontiguousarray(theta, dtype=float)
        obs = np.zeros((n, NOBS))
        lib().orc_sweep_learned(self.h, n, _dp(obs), H, _dp(theta), float(rho))
        return obs

    def green_tau(self, t):
        """(G(t,0), Gbar(0,t), G(t,t)) of the current configuration from the
        time origin 0, t in slices (plain propagation: small beta)."""
        out = [np.zeros((self.N, self.N), complex) for _ in range(3)]
        lib().orc_green_tau(self.h, int(t), *[_dp(a.view(float)) for a in out])
        return tuple(out)

    def green_tau_stable(self, t):
        """The same three matrices as green_tau, from UDV decompositions of
        B(t,0) and B(beta,t): stable at any beta."""
        out = [np.zeros((self.N, self.N), complex) for _ in range(3)]
        lib().orc_green_tau_stable(self.h, int(t), *[_dp(a.view(float)) for a in out])
        return tuple(out)

    def measure_tau(self, taus, stable=False):
        """S^i_{q=0}(tau) for i = 1..5 at slice offsets taus (time origin 0):
        array (len(taus), 5); from plain propagation (small beta) or, with
        stable=True, from the stable UDV form of the Green's functions."""
        t = np.ascontiguousarray(taus, dtype=np.int32)
        out = np.zeros((len(t), 5))
        f = lib().orc_measure_tau_stable if stable else lib().orc_measure_tau
        f(self.h, len(t), _ip(t), _dp(out))
        return out

    def measure(self):
        obs = np.zeros(NOBS)
        lib().orc_measure(self.h, _dp(obs))
        return obs

    def skip_energy(self, skip=True):
        """Leave the energy column (12) of later records at 0: its Wick sum
        over every momentum costs O(N_q N^3) per record, minutes at N = 280."""
        lib().orc_set_skip_energy(self.h, 1 if skip else 0)

    def green(self):
        G = np.zeros((self.N, self.N), complex)
        lib().orc_get_green(self.h, _dp(G.view(float)))
        return G

    def green_bruteforce(self, t):
        G = np.zeros((self.N, self.N), complex)
        lib().orc_green_bruteforce(self.h, t, _dp(G.view(float)))
        return G

    def phi(self):
        p = np.zeros((self.L, self.nfs, self.nq))
        lib().orc_get_phi(self.h, _dp(p))
        return p

    def set_slice_phi(self, t, phis):
        phis = np.ascontiguousarray(phis, dtype=float).reshape(self.nfs * self.nq)
        lib().orc_set_slice_phi(self.h, t, _dp(phis))

    def B(self, t):
        B = np.zeros((self.N, self.N), complex)
        Bi = np.zeros((self.N, self.N), complex)
        lib().orc_get_B(self.h, t, _dp(B.view(float)), _dp(Bi.view(float)))
        return B, Bi

    def factors(self, t):
        E = np.zeros((7, self.N, self.N), complex)
        tw = np.zeros(2)
        n = lib().orc_slice_factors(self.h, t, _dp(E.view(float)), _dp(tw))
        return E[:n], complex(tw[0], tw[1])

    def log_bracket(self):
        out = np.zeros(2)
        lib().orc_log_bracket(self.h, _dp(out))
        return complex(out[0], out[1])

    def gradient(self, t):
        g = np.zeros((self.nfs, self.nq))
        lib().orc_gradient_at(self.h, t, _dp(g))
        return g

    def ratio_at(self, t, phis):
        """(log R, G') for replacing slice t's fields by phis (G by brute force)."""
        phis = np.ascontiguousarray(phis, dtype=float).reshape(self.nfs * self.nq)
        out = np.zeros(2)
        Gp = np.zeros((self.N, self.N), complex)
        lib().orc_ratio_at(self.h, t, _dp(phis), _dp(out), _dp(Gp.view(float)))
        return complex(out[0], out[1]), Gp

    def get_state(self):
        """checkpoint: fields, Langevin step, sweep index (orc_get_state)"""
        out = np.zeros(lib().orc_state_size(self.h))
        lib().orc_get_state(self.h, _dp(out))
        return out

    def set_state(self, state):
        """resume from get_state() of a chain built with the same arguments"""
        state = np.ascontiguousarray(state, dtype=float)
        if len(state) != lib().orc_state_size(self.h):
            raise ValueError("state size does not match this chain")
        lib().orc_set_state(self.h, _dp(state))

    @property
    def eps(self):
        return lib().orc_get_eps(self.h)

    @eps.setter
    def eps(self, v):
        lib().orc_set_eps(self.h, v)

    @property
    def sweep_index(self):
        return lib().orc_get_sweep(self.h)


def mlp_forward(theta, X, nf, H):
    """The C oracle's network forward: (B, 2nf) -> (B, 2nf) = [mu, log sigma]."""
    theta = np.ascontiguousarray(theta, dtype=float)
    X = np.ascontiguousarray(X, dtype=float)
    out = np.zeros((X.shape[0], 2 * nf))
    lib().orc_mlp_forward(nf, H, _dp(theta), X.shape[0], _dp(X), _dp(out))
    return out
