"""Seeded synthetic inputs for the real-time TDDFT propagation path.

Both the CUDA library and the FP64 oracle consume what this module makes; it is the
only module the two sides share, and it holds no step of the propagator itself
(no stencil, no Hamiltonian, no Taylor series, no density, no exchange term).  It
draws numbers from one counter-free generator (SplitMix64, Steele, Lea and Flood,
OOPSLA 2014) and builds the *inputs* the paper's workloads would read from files:

* atom positions and Kleinman-Bylander strengths D_aj (drawn);
* a local potential of attractive Gaussian wells, sampled on the grid;
* initial orbitals: Gaussians of width 1 bohr at drawn centres, orthonormalised with
  the grid inner product (modified Gram-Schmidt in index order, done as a QR with a
  positive diagonal, which is the same factorisation);
* k-points and their weights for the periodic cell.

The paper's molecules and solids (Sec. "GPUs", Fig. gpuscaling: beta-cyclodextrin,
chlorophyll; Sec. "New propagators": benzene) are not available; these seeded
systems stand in for them with the grid sizes, orbital counts and atom counts of the
workloads the library is measured on.

Orbitals use the library's host layout: complex128, shape [n_k, nz, ny, nx, n_orb]
(the state index innermost, as in the paper's packed batch layout, Sec. "Memory
layout").
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator from its published definition (64-bit state, golden-ratio
    increment, two xor-shift-multiply mixing rounds)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1)) if hi > lo else lo

    def exponential(self, rate: float) -> float:
        return -math.log(1.0 - self.uniform()) / rate


# Field gauges and envelopes (same integer codes as the C interface).
GAUGE_NONE, GAUGE_LENGTH, GAUGE_VELOCITY = 0, 1, 2
ENV_NONE, ENV_SIN2 = 0, 1
BC_ZERO, BC_BLOCH = 0, 1
PREC_C128, PREC_C64 = 0, 1
XC_NONE, XC_LDA_X, XC_LDA_X_HARTREE = 0, 1, 2


@dataclasses.dataclass
class SystemSpec:
    """One propagation problem: grid, orbitals, atoms, field, time stepping."""

    nx: int
    ny: int
    nz: int
    h: float
    fd_order: int = 4
    bc: int = BC_ZERO
    prec: int = PREC_C128
    n_orb: int = 4
    n_k: int = 1
    n_atoms: int = 0
    projectors: bool = False
    wells: bool = True
    well_depth: float = 2.0
    well_width: float = 0.8
    orb_width: float = 1.0
    r_c: float = 0.6
    r_cut: float = 2.0
    xc: int = XC_LDA_X
    occ: float = 2.0
    gauge: int = GAUGE_LENGTH
    pol: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    amp: float = 0.0
    omega: float = 0.0
    envelope: int = ENV_NONE
    t_total: float = 0.0
    dt: float = 0.02
    n_steps: int = 1
    substeps: int = 1
    seed: int = 1
    lattice: str = "random"  # "random" (molecule) or "diamond" (periodic cell)

    @property
    def n_points(self) -> int:
        return self.nx * self.ny * self.nz

    def describe(self) -> str:
        prec = "c128" if self.prec == PREC_C128 else "c64"
        bc = "zero" if self.bc == BC_ZERO else "bloch"
        return (f"{self.nx}x{self.ny}x{self.nz} h={self.h} order={self.fd_order} bc={bc} {prec} "
                f"orb={self.n_orb} k={self.n_k} atoms={self.n_atoms} proj={int(self.projectors)} "
                f"dt={self.dt} steps={self.n_steps} substeps={self.substeps} seed={self.seed}")


# ---------------------------------------------------------------------------
# Named workloads (synthetic stand-ins for the paper's systems)
# ---------------------------------------------------------------------------

def tiny_molecule(**kw) -> SystemSpec:
    """24^3 grid, h=0.3, 4th-order FD, 4 complex128 orbitals, 2 Gaussian wells, no
    projectors, LDA exchange, E0=0.01 along z at omega=0.1, 100 Taylor steps dt=0.02."""
    s = SystemSpec(nx=24, ny=24, nz=24, h=0.3, fd_order=4, prec=PREC_C128, n_orb=4,
                   n_atoms=2, projectors=False, gauge=GAUGE_LENGTH, amp=0.01, omega=0.1,
                   dt=0.02, n_steps=100, substeps=1, seed=1)
    return dataclasses.replace(s, **kw)


def medium_molecule(prec: int = PREC_C64, **kw) -> SystemSpec:
    """96^3 grid, h=0.25, 8th-order FD, 64 orbitals, 16 atoms with Gaussian wells and 4
    Kleinman-Bylander projectors each (radius 2.0), sin^2 pulse E0=0.005, omega=0.057
    over 1000 steps of dt=0.05 (4 sub-steps per step keep the Taylor series stable)."""
    s = SystemSpec(nx=96, ny=96, nz=96, h=0.25, fd_order=8, prec=prec, n_orb=64,
                   n_atoms=16, projectors=True, gauge=GAUGE_LENGTH, amp=0.005, omega=0.057,
                   envelope=ENV_SIN2, t_total=1000 * 0.05, dt=0.05, n_steps=1000,
                   substeps=4, seed=2)
    return dataclasses.replace(s, **kw)


def periodic_cell(n_k: int = 32, **kw) -> SystemSpec:
    """64^3 cubic cell of side 10.2 bohr, 8 atoms on a diamond lattice, n_k seeded
    k-points x 16 bands in complex64, Bloch phases folded into the periodic boundaries,
    velocity-gauge A(t) = 0.2 sin(0.03 t) along z, 2000 steps of dt=0.04."""
    n = 64
    s = SystemSpec(nx=n, ny=n, nz=n, h=10.2 / n, fd_order=4, bc=BC_BLOCH, prec=PREC_C64,
                   n_orb=16, n_k=n_k, n_atoms=8, projectors=True, gauge=GAUGE_VELOCITY,
                   amp=0.2, omega=0.03, dt=0.04, n_steps=2000, substeps=6, seed=4,
                   lattice="diamond")
    return dataclasses.replace(s, **kw)


def batched_systems(n_systems: int = 256, seed: int = 3, **kw) -> List[SystemSpec]:
    """Uneven independent molecules: edges U[32,80] per axis, 4..32 orbitals, 0..12 atoms
    with 4 projectors each, complex64, h=0.25, 4th-order FD, dt=0.015, 500 steps."""
    rng = SplitMix64(seed)
    out = []
    for i in range(n_systems):
        nx, ny, nz = (rng.randint(32, 80) for _ in range(3))
        n_orb = rng.randint(4, 32)
        n_atoms = rng.randint(0, 12)
        s = SystemSpec(nx=nx, ny=ny, nz=nz, h=0.25, fd_order=4, prec=PREC_C64, n_orb=n_orb,
                       n_atoms=n_atoms, projectors=n_atoms > 0, wells=True,
                       gauge=GAUGE_LENGTH, amp=0.005, omega=0.057, dt=0.015, n_steps=500,
                       substeps=1, seed=(seed << 20) + i)
        out.append(dataclasses.replace(s, **kw))
    return out


# ---------------------------------------------------------------------------
# Input synthesis
# ---------------------------------------------------------------------------

def _axis(n: int, h: float, bc: int) -> np.ndarray:
    if bc == BC_ZERO:
        return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * h
    return np.arange(n, dtype=np.float64) * h


def atom_positions(spec: SystemSpec) -> np.ndarray:
    """[n_atoms, 3] positions.  Molecules: uniform over the inner half of the box.
    Periodic cell: fcc sites plus the (1/4,1/4,1/4) basis (diamond)."""
    if spec.n_atoms == 0:
        return np.zeros((0, 3))
    if spec.lattice == "diamond":
        L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
        fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
        frac = np.concatenate([fcc, fcc + 0.25])[: spec.n_atoms]
        return frac * L
    rng = SplitMix64(spec.seed * 1000003 + 17)
    half = np.array([(spec.nx - 1), (spec.ny - 1), (spec.nz - 1)]) * spec.h / 2.0
    pos = np.empty((spec.n_atoms, 3))
    for a in range(spec.n_atoms):
        for d in range(3):
            pos[a, d] = rng.uniform(-half[d] / 2.0, half[d] / 2.0)
    return pos


def projector_strengths(spec: SystemSpec) -> np.ndarray:
    """[n_atoms, 4] real Kleinman-Bylander strengths D_aj ~ U[-1, 1] Ha."""
    rng = SplitMix64(spec.seed * 1000003 + 29)
    return np.array([[rng.uniform(-1.0, 1.0) for _ in range(4)] for _ in range(spec.n_atoms)],
                    dtype=np.float64).reshape(spec.n_atoms, 4)


def kpoints(spec: SystemSpec) -> Tuple[np.ndarray, np.ndarray]:
    """[n_k, 3] k-points drawn uniformly in the first zone [-pi/L, pi/L)^3, equal weights.
    Finite systems get k = 0, weight 1."""
    if spec.bc == BC_ZERO:
        return np.zeros((1, 3)), np.ones(1)
    rng = SplitMix64(spec.seed * 1000003 + 43)
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    k = np.array([[rng.uniform(-math.pi / L[d], math.pi / L[d]) for d in range(3)]
                  for _ in range(spec.n_k)])
    return k, np.full(spec.n_k, 1.0 / spec.n_k)


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def local_potential(spec: SystemSpec, pos: Optional[np.ndarray] = None) -> np.ndarray:
    """V_loc(r) = -depth * sum_a exp(-|r - R_a|^2 / (2 w^2)) on the grid, shape [nz,ny,nx]."""
    if pos is None:
        pos = atom_positions(spec)
    x, y, z = (_axis(n, spec.h, spec.bc) for n in (spec.nx, spec.ny, spec.nz))
    v = np.zeros((spec.nz, spec.ny, spec.nx))
    if not spec.wells:
        return v
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    for a in range(pos.shape[0]):
        dx, dy, dz = x - pos[a, 0], y - pos[a, 1], z - pos[a, 2]
        if spec.bc == BC_BLOCH:
            dx, dy, dz = _min_image(dx, L[0]), _min_image(dy, L[1]), _min_image(dz, L[2])
        r2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        v -= spec.well_depth * np.exp(-r2 / (2.0 * spec.well_width ** 2))
    return v


def orbital_centres(spec: SystemSpec) -> np.ndarray:
    rng = SplitMix64(spec.seed * 1000003 + 7)
    if spec.bc == BC_ZERO:
        half = np.array([(spec.nx - 1), (spec.ny - 1), (spec.nz - 1)]) * spec.h / 2.0
        return np.array([[rng.uniform(-half[d] / 2.0, half[d] / 2.0) for d in range(3)]
                         for _ in range(spec.n_orb)]).reshape(spec.n_orb, 3)
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    return np.array([[rng.uniform(0.0, L[d]) for d in range(3)]
                     for _ in range(spec.n_orb)]).reshape(spec.n_orb, 3)


def initial_orbitals(spec: SystemSpec) -> np.ndarray:
    """Orthonormal (h^3 inner product) Gaussian orbitals, complex128 [n_k,nz,ny,nx,n_orb].

    Periodic cells: the Gaussians are summed over the nearest images, orthonormalised,
    then multiplied by exp(i k.r) per k-point, so each orbital obeys the Bloch condition
    psi(r + L e_a) = exp(i k_a L) psi(r) on the grid.
    """
    c = orbital_centres(spec)
    x, y, z = (_axis(n, spec.h, spec.bc) for n in (spec.nx, spec.ny, spec.nz))
    L = np.array([spec.nx, spec.ny, spec.nz]) * spec.h
    N = spec.n_points
    A = np.empty((N, spec.n_orb))
    w2 = 2.0 * spec.orb_width ** 2
    for i in range(spec.n_orb):
        dx, dy, dz = x - c[i, 0], y - c[i, 1], z - c[i, 2]
        if spec.bc == BC_BLOCH:
            gx = sum(np.exp(-(dx + s * L[0]) ** 2 / w2) for s in (-1, 0, 1))
            gy = sum(np.exp(-(dy + s * L[1]) ** 2 / w2) for s in (-1, 0, 1))
            gz = sum(np.exp(-(dz + s * L[2]) ** 2 / w2) for s in (-1, 0, 1))
        else:
            gx, gy, gz = np.exp(-dx ** 2 / w2), np.exp(-dy ** 2 / w2), np.exp(-dz ** 2 / w2)
        A[:, i] = (gz[:, None, None] * gy[None, :, None] * gx[None, None, :]).reshape(N)
    q, r = np.linalg.qr(A)
    q *= np.sign(np.diag(r))[None, :]
    q /= math.sqrt(spec.h ** 3)
    k, _ = kpoints(spec)
    out = np.empty((k.shape[0], spec.nz, spec.ny, spec.nx, spec.n_orb), dtype=np.complex128)
    q = q.reshape(spec.nz, spec.ny, spec.nx, spec.n_orb)
    for ik in range(k.shape[0]):
        if spec.bc == BC_BLOCH:
            ph = np.exp(1j * (k[ik, 2] * z[:, None, None] + k[ik, 1] * y[None, :, None]
                              + k[ik, 0] * x[None, None, :]))
            out[ik] = q * ph[..., None]
        else:
            out[ik] = q
    return out


@dataclasses.dataclass
class Inputs:
    vloc: np.ndarray      # [nz, ny, nx] float64
    psi0: np.ndarray      # [n_k, nz, ny, nx, n_orb] complex128
    pos: np.ndarray       # [n_atoms, 3]
    D: np.ndarray         # [n_atoms, 4]
    kpts: np.ndarray      # [n_k, 3]
    kw: np.ndarray        # [n_k]


def make_inputs(spec: SystemSpec, with_orbitals: bool = True) -> Inputs:
    pos = atom_positions(spec)
    k, kw = kpoints(spec)
    return Inputs(vloc=local_potential(spec, pos),
                  psi0=initial_orbitals(spec) if with_orbitals else None,
                  pos=pos, D=projector_strengths(spec), kpts=k, kw=kw)


def random_orbitals(spec: SystemSpec, seed: int) -> np.ndarray:
    """Unstructured complex test vectors (for Hermiticity and parity of single H
    applications), drawn from SplitMix64-seeded numpy streams."""
    rng = np.random.Generator(np.random.PCG64(SplitMix64(seed).next_u64()))
    shape = (spec.n_k, spec.nz, spec.ny, spec.nx, spec.n_orb)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
