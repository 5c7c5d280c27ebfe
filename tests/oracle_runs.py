"""Oracle chains for the GPU parity tests at the benchmark's matrix size,
run in spawned worker processes (started before or independently of any
GPU work) so the slow FP64 CPU chains overlap the GPU side.  Each function
returns plain arrays: the per-update trace, the per-sweep observable
records, the fields and G after every sweep."""
import numpy as np


def langevin_chain(nphi, beta, dtau, u, anis, seed, n_stab, eps0, nsweeps):
    """Plain Langevin (MALA) sweeps of the FP64 oracle; G and the fields are
    recorded after every sweep."""
    from oracle import model as M
    from oracle import oracle as O
    m = M.Model(M.TORUS, nphi)
    o = O.Chain(M.TORUS, nphi, beta, dtau, u, anis, seed, n_stab=n_stab, eps0=eps0, model=m)
    o.enable_trace(nsweeps * o.L)
    obs, greens = [], []
    for _ in range(nsweeps):
        obs.append(o.sweep(1))
        greens.append(o.green())
    return {"trace": o.trace(), "obs": np.concatenate(obs), "green": np.array(greens),
            "phi": o.phi(), "L": o.L}


def scheduled_chain(nphi, beta, dtau, u, anis, seed, n_stab, eps0, schedule, theta, H, rho):
    """Sweeps in the given order: 'P' a Langevin sweep, 'N' a learned sweep
    with the network parameters theta (hidden width H) at pCN correlation
    rho; G and the fields after every sweep."""
    from oracle import model as M
    from oracle import oracle as O
    m = M.Model(M.TORUS, nphi)
    o = O.Chain(M.TORUS, nphi, beta, dtau, u, anis, seed, n_stab=n_stab, eps0=eps0, model=m)
    o.enable_trace(len(schedule) * o.L)
    obs, greens, phis = [], [], []
    for kind in schedule:
        if kind == "P":
            obs.append(o.sweep(1))
        else:
            obs.append(o.sweep_learned(1, theta, H, rho))
        greens.append(o.green())
        phis.append(o.phi())
    return {"trace": o.trace(), "obs": np.concatenate(obs), "green": np.array(greens),
            "phi": np.array(phis), "L": o.L}


def plain_chain(geom, size, beta, dtau, u, anis, seed, n_stab, eps0, nsweeps, schedule=None,
                energy=True):
    """Sweeps of the oracle in either geometry (geom: oracle model code):
    Langevin sweeps, or the given schedule ('P' Langevin, '0' a whole-slice
    move around N(0, 1), i.e. the learned move with a zero network);
    energy=False leaves the records' energy column at 0.  Trace, records, G
    and fields at the end."""
    import numpy as np
    from oracle import learned as LN
    from oracle import model as M
    from oracle import oracle as O
    m = M.Model(geom, size)
    o = O.Chain(geom, size, beta, dtau, u, anis, seed, n_stab=n_stab, eps0=eps0, model=m)
    if not energy:
        o.skip_energy()
    schedule = schedule or "P" * nsweeps
    o.enable_trace(len(schedule) * o.L)
    th = np.zeros(LN.n_params(4 * o.nq, 2))
    obs = np.concatenate([o.sweep(1) if k == "P" else o.sweep_learned(1, th, 2, 0.0)
                          for k in schedule])
    return {"trace": o.trace(), "obs": obs, "green": o.green(), "phi": o.phi(), "L": o.L}
