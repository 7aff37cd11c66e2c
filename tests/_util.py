"""Shared helpers for the GPU parity tests (case construction, device round trips)."""
import dataclasses

import numpy as np

from paper_1912_07921_gb300 import inputs as I


def ragged_molecule(prec, fd_order=8, n_orb=5, **kw):
    """Grid sizes that are not multiples of any tile, atoms whose spheres touch the faces."""
    s = I.SystemSpec(nx=37, ny=21, nz=19, h=0.3, fd_order=fd_order, prec=prec, n_orb=n_orb, n_atoms=4,
                     projectors=True, gauge=I.GAUGE_LENGTH, amp=0.02, omega=0.2, envelope=I.ENV_SIN2,
                     t_total=3.0, dt=0.02, seed=21)
    return dataclasses.replace(s, **kw)


def bloch_cell(prec, fd_order=4, n_orb=3, n_k=3, **kw):
    s = I.SystemSpec(nx=13, ny=12, nz=10, h=0.35, fd_order=fd_order, bc=I.BC_BLOCH, prec=prec,
                     n_orb=n_orb, n_k=n_k, n_atoms=2, projectors=True, gauge=I.GAUGE_VELOCITY,
                     amp=0.3, omega=0.4, pol=(0.2, 0.3, 0.9), dt=0.01, seed=31)
    return dataclasses.replace(s, **kw)


def bloch_inputs(spec):
    inp = I.make_inputs(spec)
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    # spheres crossing the cell faces (wrapped images, Bloch phases)
    inp.pos = np.array([[0.2, 0.3, 0.5 * L[2]], [L[0] - 0.4, 0.6 * L[1], L[2] - 0.1]])[: spec.n_atoms]
    return inp


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def small_uneven_batch(prec, n=5, seed=7):
    """Uneven finite boxes (edges 17..33, 3..11 orbitals, 0..3 atoms with projectors) that
    share FD order 4, h = 0.25, dt = 0.015 and one sub-step, as the batched workload does."""
    rng = I.SplitMix64(seed)
    out = []
    for i in range(n):
        nx, ny, nz = (rng.randint(17, 33) for _ in range(3))
        n_orb = rng.randint(3, 11)
        n_atoms = rng.randint(0, 3)
        out.append(I.SystemSpec(nx=nx, ny=ny, nz=nz, h=0.25, fd_order=4, prec=prec, n_orb=n_orb,
                                n_atoms=n_atoms, projectors=n_atoms > 0, gauge=I.GAUGE_LENGTH,
                                amp=0.01 * (i + 1), omega=0.2, envelope=I.ENV_SIN2 if i % 2 else I.ENV_NONE,
                                t_total=0.5, dt=0.015, substeps=1, seed=(seed << 8) + i))
    return out


def horizon_molecule(prec):
    """The medium molecule's physics on a smaller grid, for the 1000-step FP32 check: order-8
    FD at h = 0.25 on 32^3, 8 orbitals, 16 atoms with Gaussian wells and 4 Kleinman-Bylander
    projectors each, LDA exchange, the sin^2 pulse E0 = 0.005, omega = 0.057 over T = 1000 dt,
    dt = 0.05 as 4 Taylor-4 sub-steps."""
    return I.medium_molecule(prec=prec, nx=32, ny=32, nz=32, n_orb=8, n_steps=1000)


def horizon_cell(prec):
    """The periodic cell's physics on a smaller grid, for the 1000-step FP32 check: side
    10.2 bohr on 32^3 (h = 0.319), order-4 FD, 8 diamond atoms with wells and projectors,
    2 seeded k-points x 8 bands, velocity gauge A0 = 0.2, omega = 0.03, dt = 0.04 as 2
    Taylor-4 sub-steps (the automatic count at this spacing)."""
    return I.periodic_cell(n_k=2, prec=prec, nx=32, ny=32, nz=32, h=10.2 / 32, n_orb=8, n_steps=1000,
                           substeps=2)


HORIZON_CASES = {"molecule": horizon_molecule, "cell": horizon_cell}


def read_horizon_golden(path):
    """Records [n_steps, 8] of a stored oracle trajectory (see make_fp32_horizon.py)."""
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return np.array([[float(x) for x in r[1:]] for r in rows])
