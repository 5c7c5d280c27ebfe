"""Exact diagonalisation of the Fierz-transformed projected Hamiltonian.

TEST INFRASTRUCTURE ONLY (pins the oracle; see the oracle package header).

H = sum_{i=0..3} g_i sum_{q in K} n^{O^i}_q n^{O^i}_qbar  (Methods, Eq. newmodel)
with n^{M}_q = sum c^dagger (M (x) F_q) c - b_q delta_{i,0} over the four
flavours (valley x spin) and b_q = 2 Tr F_q (the particle-hole background of
Eq. torus_density_operator).  The grand-canonical ensemble at zero chemical
potential is what det(1 + B) samples.  The Hamiltonian conserves the particle
number of each spin separately (the O^i act as identity on spin), so it is
block-diagonalised by (N_up, N_down) and each block is diagonalised densely.

Mode order: spin (outer), valley, orbital (inner): mode = s*N + v*norb + k.
This construction works directly with fermion operators on bit strings
(Jordan-Wigner signs); it uses none of the oracle's Wick formulas.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import model as M

PAULI = {
    "I": np.eye(2, dtype=complex),
    "x": np.array([[0, 1], [1, 0]], dtype=complex),
    "y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "z": np.array([[1, 0], [0, -1]], dtype=complex),
}
O_VALLEY = [PAULI["I"], PAULI["x"], PAULI["y"], PAULI["z"]]
# Gamma^1..5 = tau_x I, tau_y I, tau_z sigma_x, tau_z sigma_y, tau_z sigma_z
GAMMA = [("x", "I"), ("y", "I"), ("z", "x"), ("z", "y"), ("z", "z")]


def one_body(model: M.Model, q: int, valley: np.ndarray, spin: np.ndarray) -> np.ndarray:
    """Single-particle matrix of spin (x) valley (x) F_q on 2N modes."""
    return np.kron(spin, np.kron(valley, model.dense_F(q)))


class Fock:
    """Spin-resolved particle-number blocks of the 2^(2N) Fock space."""

    def __init__(self, nmodes_per_spin: int):
        self.n = nmodes_per_spin
        self.nm = 2 * nmodes_per_spin
        self.blocks = {}
        for nu in range(self.n + 1):
            for nd in range(self.n + 1):
                up = [sum(1 << b for b in c) for c in itertools.combinations(range(self.n), nu)]
                dn = [sum(1 << (b + self.n) for b in c) for c in itertools.combinations(range(self.n), nd)]
                states = [a | b for a in up for b in dn]
                self.blocks[(nu, nd)] = (states, {s: i for i, s in enumerate(states)})

    def op(self, h: np.ndarray, key, src=None):
        """Matrix of sum_{xy} h_xy c^dagger_x c_y from block `src` (default:
        `key`) into block `key`; transitions landing elsewhere are dropped."""
        states, index = self.blocks[key]
        sstates = self.blocks[src if src is not None else key][0]
        out = np.zeros((len(states), len(sstates)), dtype=complex)
        nz = np.argwhere(np.abs(h) > 0)
        for col, s in enumerate(sstates):
            for x, y in nz:
                if not (s >> y) & 1:
                    continue
                s1 = s & ~(1 << y)
                sign = -1 if bin(s & ((1 << y) - 1)).count("1") % 2 else 1
                if (s1 >> x) & 1:
                    continue
                s2 = s1 | (1 << x)
                if bin(s1 & ((1 << x) - 1)).count("1") % 2:
                    sign = -sign
                if s2 in index:
                    out[index[s2], col] += sign * h[x, y]
        return out


class ED:
    """Thermal averages of the transformed Hamiltonian at inverse temperature beta."""

    def __init__(self, model: M.Model, g, beta: float):
        self.model = model
        self.g = np.asarray(g, float)
        self.beta = beta
        N = model.N
        self.fock = Fock(N)
        nq = model.nq
        I2 = PAULI["I"]
        self.blocks = {}
        for key in self.fock.blocks:
            dim = len(self.fock.blocks[key][0])
            nops = {}
            for i in range(4):
                for q in range(nq):
                    A = self.fock.op(one_body(model, q, O_VALLEY[i], I2), key)
                    if i == 0:
                        A = A - model.bg[q] * np.eye(dim)
                    nops[(i, q)] = A
            H = np.zeros((dim, dim), dtype=complex)
            for i in range(4):
                for q in range(nq):
                    H += self.g[i] * nops[(i, q)] @ nops[(i, int(model.partner[q]))]
            assert np.abs(H - H.conj().T).max() < 1e-10
            w, V = np.linalg.eigh(H)
            self.blocks[key] = (w, V, nops)
        emin = min(b[0].min() for b in self.blocks.values())
        self.emin = emin
        self.Z = sum(np.exp(-beta * (b[0] - emin)).sum() for b in self.blocks.values())

    def thermal(self, opfun) -> float:
        """<O> with O given blockwise by opfun(key, nops)."""
        tot = 0.0
        for key, (w, V, nops) in self.blocks.items():
            Ob = opfun(key, nops)
            Od = np.einsum("ij,jk,ki->i", V.conj().T, Ob, V)
            tot += np.sum(np.exp(-self.beta * (w - self.emin)) * Od).real
        return tot / self.Z

    def energy(self) -> float:
        def f(key, nops):
            w, V, _ = self.blocks[key]
            return (V * w) @ V.conj().T
        return self.thermal(f)

    def structure_factor(self, gi: int, q: int) -> float:
        """S^i_q = <n^{Gamma^i}_q n^{Gamma^i}_qbar> for Gamma index gi = 0..4."""
        tv, ts = GAMMA[gi]
        m = self.model
        hq = one_body(m, q, PAULI[tv], PAULI[ts])
        hp = one_body(m, int(m.partner[q]), PAULI[tv], PAULI[ts])

        def f(key, nops):
            nu, nd = key
            out = 0
            # intermediate blocks reachable by one spin flip (or none)
            for mid in [(nu, nd), (nu + 1, nd - 1), (nu - 1, nd + 1)]:
                if mid in self.fock.blocks:
                    out = out + self.fock.op(hq, key, mid) @ self.fock.op(hp, mid, key)
            return out
        return self.thermal(f)

    def structure_factor_tau(self, gi: int, q: int, tau: float) -> float:
        """S^i_q(tau) = <n^{Gamma^i}_q(tau) n^{Gamma^i}_qbar(0)>
        = Tr[e^{-(beta - tau) H} n_q e^{-tau H} n_qbar] / Z, 0 <= tau <= beta."""
        tv, ts = GAMMA[gi]
        m = self.model
        hq = one_body(m, q, PAULI[tv], PAULI[ts])
        hp = one_body(m, int(m.partner[q]), PAULI[tv], PAULI[ts])
        tot = 0.0
        for key, (w, V, _) in self.blocks.items():
            nu, nd = key
            left = (V * np.exp(-(self.beta - tau) * (w - self.emin))) @ V.conj().T
            for mid in [(nu, nd), (nu + 1, nd - 1), (nu - 1, nd + 1)]:
                if mid not in self.blocks:
                    continue
                wm, Vm, _ = self.blocks[mid]
                prop = (Vm * np.exp(-tau * (wm - self.emin))) @ Vm.conj().T
                A = self.fock.op(hq, key, mid)
                B = self.fock.op(hp, mid, key)
                tot += np.trace(left @ A @ prop @ B).real
        return tot / self.Z

    def gap(self, gi: int, q: int, rel_tol: float = 1e-10) -> float:
        """Lowest excitation energy E_n - E_0 reachable from the ground state
        by n^{Gamma^i}_q (spectral weight |<n| n_q |0>|^2 above rel_tol of
        the total): the rate of the long-time decay of S^i_q(tau) at zero
        temperature (Supplementary Note 2).  Needs a unique ground state."""
        tv, ts = GAMMA[gi]
        hq = one_body(self.model, q, PAULI[tv], PAULI[ts])
        levels = sorted((w[k], key, k) for key, (w, _, _) in self.blocks.items() for k in range(len(w)))
        e0, key0, k0 = levels[0]
        if levels[1][0] - e0 < 1e-9 * max(1.0, abs(e0)):
            raise ValueError("degenerate ground state")
        psi0 = self.blocks[key0][1][:, k0]
        nu, nd = key0
        found = []
        for mid in [(nu, nd), (nu + 1, nd - 1), (nu - 1, nd + 1)]:
            if mid not in self.blocks:
                continue
            wm, Vm, _ = self.blocks[mid]
            amp = Vm.conj().T @ (self.fock.op(hq, mid, key0) @ psi0)
            found += [(e, abs(a) ** 2) for e, a in zip(wm, amp)]
        tot = sum(a for _, a in found)
        exc = [e - e0 for e, a in found if a > rel_tol * tot and e - e0 > 1e-9]
        return float(min(exc))

    def observables(self) -> dict:
        m = self.model
        q0 = m.q0() if m.geom == M.TORUS else 0
        dq = m.delta_q()
        S0 = np.array([self.structure_factor(i, q0) for i in range(5)])
        Sd = np.array([np.mean([self.structure_factor(i, q) for q in dq]) for i in range(5)])
        return {
            "E": self.energy(),
            "S0": S0,
            "Sdq": Sd,
            "m2": S0.sum() / (5.0 * m.norb ** 2),
            "R": 1.0 - Sd.sum() / S0.sum(),
        }
