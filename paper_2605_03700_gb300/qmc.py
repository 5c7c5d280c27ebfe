"""Thin ctypes binding of libqmc (include/qmc.h).

Argument marshalling only: every step of the sweep runs in the CUDA library.
The functions carry the C names; ``Chain`` is a small convenience wrapper.
There is no CPU fallback: if libqmc.so is missing or no CUDA device is
present, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libqmc.so")

QMC_TORUS = 0
QMC_SPHERE = 1
QMC_NOBS = 20
QMC_NTRACE = 8
QMC_DRIFT_EXACT, QMC_DRIFT_FIRST = 0, 1
QMC_SLICE_SHARED, QMC_SLICE_INDEP = 0, 2
OBS_NAMES = ["m2", "S1_0", "S2_0", "S3_0", "S4_0", "S5_0", "S1_dq", "S2_dq",
             "S3_dq", "S4_dq", "S5_dq", "R", "E", "acc", "eps", "stab_err",
             "sign_dev", "n_acc", "_", "_"]


class qmc_opts(C.Structure):
    _fields_ = [
        ("n_stab", C.c_int),
        ("precision", C.c_int),
        ("eps0", C.c_double),
        ("deps", C.c_double),
        ("r0", C.c_double),
        ("n_adapt", C.c_int),
        ("n_orb_sphere", C.c_int),
        ("n_chains", C.c_int),
        ("couplings", C.POINTER(C.c_double)),
        ("anisotropies", C.POINTER(C.c_double)),
        ("seeds", C.POINTER(C.c_uint64)),
        ("series_capacity", C.c_int),
        ("trace_capacity", C.c_int),
        ("stab_tol", C.c_double),
        ("sign_tol", C.c_double),
        ("drift", C.c_int),
        ("slice_kind", C.c_int),
    ]


QMC_CKPT_MAGIC = 0x4B434D51
QMC_CKPT_VERSION = 1


class qmc_checkpoint_header(C.Structure):
    _fields_ = [
        ("magic", C.c_uint32),
        ("version", C.c_uint32),
        ("geometry", C.c_int32),
        ("n_orb", C.c_int32),
        ("L", C.c_int32),
        ("n_q", C.c_int32),
        ("n_chains", C.c_int32),
        ("precision", C.c_int32),
        ("drift", C.c_int32),
        ("n_stab", C.c_int32),
        ("beta", C.c_double),
        ("dtau", C.c_double),
        ("params_hash", C.c_uint64),
        ("n_doubles", C.c_uint64),
    ]


class QMCError(RuntimeError):
    pass


_lib = None


def lib():
    """Load libqmc.so (built by paper_2605_03700_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise QMCError(f"{LIB} is missing: run paper_2605_03700_gb300.build.build() first")
        L = C.CDLL(LIB)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.qmc_state_size.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.qmc_get_state.argtypes = [vp, dp, C.c_size_t]
        L.qmc_set_state.argtypes = [vp, dp, C.c_size_t]
        hp = C.POINTER(qmc_checkpoint_header)
        L.qmc_checkpoint_header_of.argtypes = [vp, hp]
        L.qmc_checkpoint_write.argtypes = [C.c_char_p, hp, dp]
        L.qmc_checkpoint_read_header.argtypes = [C.c_char_p, hp]
        L.qmc_checkpoint_read.argtypes = [C.c_char_p, hp, dp, C.c_size_t]
        L.qmc_measure_tau.argtypes = [vp, C.c_int, C.POINTER(C.c_int), dp]
        L.qmc_default_opts.argtypes = [C.POINTER(qmc_opts)]
        L.qmc_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_double, C.c_double,
                                 C.c_double, C.c_double, C.c_uint64, C.POINTER(qmc_opts)]
        L.qmc_destroy.argtypes = [vp]
        L.qmc_set_stream.argtypes = [vp, vp]
        L.qmc_sweep.argtypes = [vp, C.c_int]
        L.qmc_sweep_graph.argtypes = [vp, C.c_int]
        fp = C.POINTER(C.c_float)
        L.qmc_net_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_longlong, C.c_uint64]
        L.qmc_net_destroy.argtypes = [vp]
        L.qmc_net_set_stream.argtypes = [vp, vp]
        L.qmc_net_num_params.restype = C.c_longlong
        L.qmc_net_num_params.argtypes = [vp]
        L.qmc_net_dataset_size.restype = C.c_longlong
        L.qmc_net_dataset_size.argtypes = [vp]
        L.qmc_net_get_params.argtypes = [vp, fp, C.c_size_t]
        L.qmc_net_set_params.argtypes = [vp, fp, C.c_size_t]
        L.qmc_net_collect.argtypes = [vp, vp]
        L.qmc_net_train.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, dp]
        L.qmc_net_forward.argtypes = [vp, fp, C.c_int, fp]
        L.qmc_net_loss_grad.argtypes = [vp, fp, fp, C.c_int, dp, fp]
        L.qmc_sweep_learned.argtypes = [vp, vp, C.c_int, C.c_double]
        L.qmc_sweep_learned_graph.argtypes = [vp, vp, C.c_int, C.c_double]
        L.qmc_sweep_prior.argtypes = [vp, C.c_int, C.c_double]
        L.qmc_sweep_prior_graph.argtypes = [vp, C.c_int, C.c_double]
        L.qmc_group_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int]
        L.qmc_group_sweep.argtypes = [vp, C.c_int]
        L.qmc_group_sync.argtypes = [vp]
        L.qmc_group_destroy.argtypes = [vp]
        L.qmc_sync.argtypes = [vp]
        L.qmc_measure.argtypes = [vp, dp]
        L.qmc_get_series.argtypes = [vp, C.c_int, dp]
        L.qmc_series_length.argtypes = [vp]
        L.qmc_get_green.argtypes = [vp, C.c_int, dp, C.c_size_t]
        L.qmc_get_green_block.argtypes = [vp, C.c_int, dp, C.c_size_t]
        L.qmc_get_fields.argtypes = [vp, C.c_int, dp, C.c_size_t]
        L.qmc_get_trace.argtypes = [vp, C.c_int, dp, C.c_size_t, C.POINTER(C.c_long)]
        L.qmc_sizes.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int)]
        L.qmc_get_eps.argtypes = [vp, dp]
        L.qmc_get_propagator.argtypes = [vp, C.c_int, C.c_int, dp, dp, C.c_size_t]
        L.qmc_tau_int.restype = C.c_double
        L.qmc_tau_int.argtypes = [dp, C.c_int]
        L.qmc_strerror.restype = C.c_char_p
        L.qmc_strerror.argtypes = [C.c_int]
        L.qmc_last_error.restype = C.c_char_p
        L.qmc_last_error.argtypes = [vp]
        L.qmc_copy_latest_async.argtypes = [vp, dp]
        L.qmc_ratio_update.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp]
        L.qmc_ratio_update_noalloc.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp]
        L.qmc_gemm_tile.argtypes = [C.c_int, C.c_int]
        L.qmc_launch_count.restype = C.c_longlong
        L.qmc_launch_count.argtypes = []
        L.qmc_profile_gemm.argtypes = [C.c_int, dp, C.POINTER(C.c_longlong), dp]
        L.qmc_peak_fma.argtypes = [C.c_int, C.c_int, dp]
        L.qmc_profile_tensor.argtypes = [dp, C.POINTER(C.c_longlong), dp, dp]
        L.qmc_cgemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, C.c_int, vp, vp,
                                C.c_int, C.c_int, C.c_int, vp]
        L.qmc_eigh.argtypes = [C.c_int, C.c_int, vp, vp, vp, C.c_int, vp]
        L.qmc_udv.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(code, h=None):
    if code != 0:
        msg = lib().qmc_strerror(code).decode()
        if h:
            msg += ": " + lib().qmc_last_error(h).decode()
        raise QMCError(f"libqmc error {code}: {msg}")


def qmc_default_opts() -> qmc_opts:
    o = qmc_opts()
    _check(lib().qmc_default_opts(C.byref(o)))
    return o


def checkpoint_write(path, header, state):
    """Write a checkpoint file (qmc_checkpoint_write)."""
    state = np.ascontiguousarray(state, dtype=float)
    if state.size != header.n_doubles:
        raise QMCError("state length differs from the header's n_doubles")
    _check(lib().qmc_checkpoint_write(os.fsencode(path), C.byref(header), _dp(state)))


def checkpoint_read_header(path):
    h = qmc_checkpoint_header()
    _check(lib().qmc_checkpoint_read_header(os.fsencode(path), C.byref(h)))
    return h


def checkpoint_read(path, expect=None):
    """The state stored in a checkpoint file; with expect (a header) the file
    must belong to a run built the same way."""
    h = checkpoint_read_header(path)
    out = np.zeros(h.n_doubles)
    _check(lib().qmc_checkpoint_read(os.fsencode(path), C.byref(expect) if expect is not None else None,
                                     _dp(out), out.size))
    return out


def qmc_gemm_tile(n: int, precision: int) -> int:
    return int(lib().qmc_gemm_tile(n, precision))


def qmc_launch_count() -> int:
    return int(lib().qmc_launch_count())


def qmc_profile_gemm(enable: bool):
    """Start (True) or stop (False) GEMM event timing; stop returns
    (total_ms, launches, flops)."""
    ms, n, fl = C.c_double(), C.c_longlong(), C.c_double()
    _check(lib().qmc_profile_gemm(1 if enable else 0, C.byref(ms), C.byref(n), C.byref(fl)))
    return None if enable else (ms.value, n.value, fl.value)


def qmc_profile_tensor():
    """(ms, launches, needed flops, issued flops) of the tensor-core MMA
    kernel in the last qmc_profile_gemm window."""
    ms, fl, iss = C.c_double(), C.c_double(), C.c_double()
    n = C.c_longlong()
    lib().qmc_profile_tensor(C.byref(ms), C.byref(n), C.byref(fl), C.byref(iss))
    return ms.value, n.value, fl.value, iss.value


def qmc_peak_fma(fp64: bool = True, iters: int = 4096) -> float:
    """Measured FMA rate of the current device in TFLOP/s (FP64 or FP32)."""
    v = C.c_double()
    _check(lib().qmc_peak_fma(1 if fp64 else 0, int(iters), C.byref(v)))
    return v.value


def qmc_cgemm(M, N, K, batch, A_ptr, opA, B_ptr, opB, d_ptr, C_ptr, negate=0, add_identity=0,
              digits=7, stream=0):
    """Batched complex product on device pointers (qmc_cgemm); digits 0 = FP64
    CUDA cores, 1..8 = tensor cores from that many bfloat16 digits."""
    _check(lib().qmc_cgemm(M, N, K, batch, C.c_void_p(A_ptr), opA, C.c_void_p(B_ptr), opB,
                           C.c_void_p(d_ptr) if d_ptr else None, C.c_void_p(C_ptr), negate,
                           add_identity, digits, C.c_void_p(stream) if stream else None))


def qmc_eigh(n, batch, A_ptr, U_ptr, w_ptr, precision=1, stream=0):
    """Eigenpairs of a batch of Hermitian matrices on device pointers
    (qmc_eigh); precision 0 = FP64 Jacobi, 1 = FP32 + FP64 refinement,
    2 = refinement products on the tensor cores."""
    _check(lib().qmc_eigh(n, batch, C.c_void_p(A_ptr), C.c_void_p(U_ptr), C.c_void_p(w_ptr),
                          precision, C.c_void_p(stream) if stream else None))


def qmc_udv(n, batch, X_ptr, Q_ptr, logD_ptr, V_ptr, logscale_ptr=0, stream=0):
    """X diag(e^c) = Q diag(e^d) V on device pointers (qmc_udv): c the
    optional column log scales, d = log D returned."""
    _check(lib().qmc_udv(n, batch, C.c_void_p(X_ptr),
                         C.c_void_p(logscale_ptr) if logscale_ptr else None, C.c_void_p(Q_ptr),
                         C.c_void_p(logD_ptr), C.c_void_p(V_ptr),
                         C.c_void_p(stream) if stream else None))


def qmc_ratio_update(N, batch, G_ptr, Delta_ptr, Gp_ptr, logdet_ptr, stream=0):
    """Device pointers (ints) of complex128 buffers; see include/qmc.h."""
    _check(lib().qmc_ratio_update(N, batch, C.c_void_p(G_ptr), C.c_void_p(Delta_ptr),
                                  C.c_void_p(Gp_ptr), C.c_void_p(logdet_ptr), C.c_void_p(stream)))


def qmc_tau_int(x) -> float:
    x = np.ascontiguousarray(x, dtype=float)
    return lib().qmc_tau_int(_dp(x), len(x))


class Chain:
    """A batch of independent CF-DQMC chains resident on the current GPU."""

    def __init__(self, geometry, N_phi, beta, dtau, coupling, anisotropy=0.0, seed=0, *,
                 n_chains=1, couplings=None, anisotropies=None, seeds=None, n_stab=10,
                 eps0=0.5, deps=0.1, r0=0.574, n_adapt=-1, series_capacity=4096,
                 trace_capacity=0, stab_tol=1e-6, sign_tol=1e-6, precision=0, n_orb_sphere=0,
                 drift=0, slice_kind=0, stream=None):
        o = qmc_default_opts()
        o.n_stab = n_stab
        o.drift = drift
        o.slice_kind = slice_kind
        o.n_orb_sphere = n_orb_sphere
        o.precision = precision
        o.eps0, o.deps, o.r0, o.n_adapt = eps0, deps, r0, n_adapt
        o.n_chains = n_chains
        o.series_capacity = series_capacity
        o.trace_capacity = trace_capacity
        o.stab_tol, o.sign_tol = stab_tol, sign_tol
        self._keep = []
        if couplings is not None:
            a = np.ascontiguousarray(couplings, dtype=float)
            self._keep.append(a)
            o.couplings = _dp(a)
        if anisotropies is not None:
            a = np.ascontiguousarray(anisotropies, dtype=float)
            self._keep.append(a)
            o.anisotropies = _dp(a)
        if seeds is not None:
            a = np.ascontiguousarray(seeds, dtype=np.uint64)
            self._keep.append(a)
            o.seeds = a.ctypes.data_as(C.POINTER(C.c_uint64))
        h = C.c_void_p()
        _check(lib().qmc_create(C.byref(h), geometry, N_phi, beta, dtau, coupling, anisotropy,
                                seed, C.byref(o)))
        self.h = h
        if stream is not None:
            self.set_stream(stream)
        n_orb, n_q, L, nb = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        lib().qmc_sizes(h, C.byref(n_orb), C.byref(n_q), C.byref(L), C.byref(nb))
        self.n_orb, self.n_q, self.L, self.n_chains = n_orb.value, n_q.value, L.value, nb.value
        self.N = 2 * self.n_orb
        self.trace_capacity = trace_capacity
        # field sets per slice: 4 (one per channel) or 7 (one per factor)
        self.n_sets = 7 if slice_kind == QMC_SLICE_INDEP else 4

    def close(self):
        if getattr(self, "h", None):
            lib().qmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a cudaStream_t handle as int (e.g. torch.cuda.Stream().cuda_stream)."""
        _check(lib().qmc_set_stream(self.h, C.c_void_p(int(stream))), self.h)

    def sweep(self, n=1, graph=False):
        """Enqueue n sweeps of all chains; graph=True replays one captured
        sweep (qmc_sweep_graph) instead of launching every kernel."""
        f = lib().qmc_sweep_graph if graph else lib().qmc_sweep
        _check(f(self.h, n), self.h)

    def sweep_learned(self, net, n=1, rho=0.0, graph=False):
        """n sweeps of learned slice moves with network `net` (qmc_sweep_learned);
        graph=True replays one captured learned sweep (qmc_sweep_learned_graph)."""
        f = lib().qmc_sweep_learned_graph if graph else lib().qmc_sweep_learned
        _check(f(self.h, net.h, n, float(rho)), self.h)

    def sweep_prior(self, n=1, rho=0.0, graph=False):
        """n sweeps of whole-slice moves around N(0, 1) (qmc_sweep_prior)."""
        f = lib().qmc_sweep_prior_graph if graph else lib().qmc_sweep_prior
        _check(f(self.h, n, float(rho)), self.h)

    def sync(self):
        _check(lib().qmc_sync(self.h), self.h)

    def measure(self):
        out = np.zeros((self.n_chains, QMC_NOBS))
        _check(lib().qmc_measure(self.h, _dp(out)), self.h)
        return out

    def get_state(self):
        """checkpoint: fields, Langevin steps and sweep number (qmc_get_state)"""
        n = C.c_size_t()
        _check(lib().qmc_state_size(self.h, C.byref(n)), self.h)
        out = np.zeros(n.value)
        _check(lib().qmc_get_state(self.h, _dp(out), n.value), self.h)
        return out

    def set_state(self, state):
        """resume from get_state() of a context built with the same arguments"""
        n = C.c_size_t()
        _check(lib().qmc_state_size(self.h, C.byref(n)), self.h)
        state = np.ascontiguousarray(state, dtype=float)
        if state.size != n.value:
            raise QMCError(f"state has {state.size} values, this context needs {n.value}")
        _check(lib().qmc_set_state(self.h, _dp(state), n.value), self.h)

    def checkpoint_header(self):
        h = qmc_checkpoint_header()
        _check(lib().qmc_checkpoint_header_of(self.h, C.byref(h)), self.h)
        return h

    def save(self, path):
        """checkpoint to a file: header, state, checksum"""
        checkpoint_write(path, self.checkpoint_header(), self.get_state())

    def load(self, path):
        """resume from a file written by save() of a context built the same way"""
        self.set_state(checkpoint_read(path, self.checkpoint_header()))

    def measure_tau(self, taus):
        """S^i_{q=0}(tau) of the current configuration, i = 1..5, at the
        ascending slice offsets taus from the time origin: array
        (n_chains, len(taus), 5) (qmc_measure_tau)."""
        t = np.ascontiguousarray(taus, dtype=np.int32)
        out = np.zeros((self.n_chains, len(t), 5))
        _check(lib().qmc_measure_tau(self.h, len(t), t.ctypes.data_as(C.POINTER(C.c_int)),
                                     _dp(out)), self.h)
        return out

    def series(self, count=None):
        n = lib().qmc_series_length(self.h)
        count = n if count is None else count
        out = np.zeros((self.n_chains, count, QMC_NOBS))
        _check(lib().qmc_get_series(self.h, count, _dp(out)), self.h)
        return out

    def copy_latest_async(self, host_ptr):
        """Enqueue the D2H copy of the newest records into host memory at
        host_ptr (an int address of n_chains * QMC_NOBS doubles, pinned)."""
        _check(lib().qmc_copy_latest_async(self.h, C.cast(C.c_void_p(host_ptr),
                                                           C.POINTER(C.c_double))), self.h)

    def green(self, chain=0, block=True):
        if block:
            G = np.zeros((self.N, self.N), complex)
            _check(lib().qmc_get_green_block(self.h, chain, _dp(G.view(float)), 2 * G.size), self.h)
        else:
            G = np.zeros((2 * self.N, 2 * self.N), complex)
            _check(lib().qmc_get_green(self.h, chain, _dp(G.view(float)), 2 * G.size), self.h)
        return G

    def propagator(self, slice_, chain=0):
        """(B_tau, B_tau^-1) of a slice (1-based) as complex128 arrays."""
        B = np.zeros((self.N, self.N), complex)
        Bi = np.zeros((self.N, self.N), complex)
        _check(lib().qmc_get_propagator(self.h, chain, slice_, _dp(B.view(float)),
                                        _dp(Bi.view(float)), 2 * B.size), self.h)
        return B, Bi

    def fields(self, chain=0):
        p = np.zeros((self.L, self.n_sets, self.n_q))
        _check(lib().qmc_get_fields(self.h, chain, _dp(p), p.size), self.h)
        return p

    def trace(self, chain=0):
        cap = max(self.trace_capacity, 1)
        buf = np.zeros((cap, QMC_NTRACE))
        cnt = C.c_long()
        _check(lib().qmc_get_trace(self.h, chain, _dp(buf), buf.size, C.byref(cnt)), self.h)
        return buf[: cnt.value].copy()

    def eps(self):
        out = np.zeros(self.n_chains)
        _check(lib().qmc_get_eps(self.h, _dp(out)), self.h)
        return out


class Group:
    """Several Chain objects (any sizes) swept together as one CUDA graph per
    sweep, each on its own graph branch (qmc_group_*).  The chains must stay
    open while the group lives."""

    def __init__(self, chains):
        self.chains = list(chains)
        arr = (C.c_void_p * len(self.chains))(*[c.h.value for c in self.chains])
        h = C.c_void_p()
        _check(lib().qmc_group_create(C.byref(h), arr, len(self.chains)))
        self.h = h

    def sweep(self, n=1):
        _check(lib().qmc_group_sweep(self.h, n))

    def sync(self):
        code = lib().qmc_group_sync(self.h)
        if code != 0:
            for c in self.chains:
                c.sync()
            _check(code)

    def close(self):
        if getattr(self, "h", None):
            lib().qmc_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Net:
    """The learned slice proposal's network (qmc_net_*): nf = 4 N_q fields per
    slice, hidden width `width`, a device-resident ring of `capacity`
    configurations for training, allocated on the first collect() as
    capacity x L x nf FP32 values (N_phi = 36, L = 360: 1.9 MB each)."""

    def __init__(self, nf, width=256, capacity=1000, seed=0):
        h = C.c_void_p()
        _check(lib().qmc_net_create(C.byref(h), int(nf), int(width), int(capacity), int(seed)))
        self.h = h
        self.nf, self.width = int(nf), int(width)

    @property
    def num_params(self):
        return int(lib().qmc_net_num_params(self.h))

    @property
    def dataset_size(self):
        return int(lib().qmc_net_dataset_size(self.h))

    def get_params(self):
        out = np.zeros(self.num_params, dtype=np.float32)
        _check(lib().qmc_net_get_params(self.h, _fp(out), out.size))
        return out

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().qmc_net_set_params(self.h, _fp(a), a.size))

    def collect(self, chain):
        _check(lib().qmc_net_collect(self.h, chain.h), chain.h)

    def train(self, steps, batch=256, lr=1e-3, weight_decay=0.0):
        loss = np.zeros(steps)
        _check(lib().qmc_net_train(self.h, int(steps), int(batch), float(lr),
                                   float(weight_decay), _dp(loss)))
        return loss

    def forward(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        out = np.zeros((X.shape[0], 2 * self.nf), dtype=np.float32)
        _check(lib().qmc_net_forward(self.h, _fp(X), X.shape[0], _fp(out)))
        return out

    def loss_grad(self, X, Y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        loss = C.c_double()
        g = np.zeros(self.num_params, dtype=np.float32)
        _check(lib().qmc_net_loss_grad(self.h, _fp(X), _fp(Y), X.shape[0], C.byref(loss),
                                       _fp(g)))
        return loss.value, g

    def close(self):
        if getattr(self, "h", None):
            lib().qmc_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
