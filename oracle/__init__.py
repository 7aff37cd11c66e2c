"""FP64 CPU oracle: Python entry points over ``tdks_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU baseline
are the only callers; the product library never imports this package.  The oracle is
compiled with gcc (``build()``) into ``oracle/_build/liboracle.so``.

Every array argument uses the host layout of the seeded inputs: orbitals complex128
[n_k, nz, ny, nx, n_orb]; fields float64 [nz, ny, nx].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdks_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Sys(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("h", ctypes.c_double), ("fd_order", ctypes.c_int), ("bc", ctypes.c_int),
        ("n_orb", ctypes.c_int), ("n_k", ctypes.c_int),
        ("kpts", ctypes.c_void_p), ("kw", ctypes.c_void_p), ("vloc", ctypes.c_void_p),
        ("xc", ctypes.c_int), ("occ", ctypes.c_double), ("gauge", ctypes.c_int),
        ("pol", ctypes.c_double * 3), ("amp", ctypes.c_double), ("omega", ctypes.c_double),
        ("envelope", ctypes.c_int), ("t_total", ctypes.c_double),
        ("n_atoms", ctypes.c_int), ("pos", ctypes.c_void_p), ("D", ctypes.c_void_p),
        ("r_c", ctypes.c_double), ("r_cut", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
        S = ctypes.POINTER(_Sys)
        _lib.oracle_fd_laplacian_weights.argtypes = [I, P]
        _lib.oracle_fd_gradient_weights.argtypes = [I, P]
        _lib.oracle_field.argtypes = [S, D, P, P]
        _lib.oracle_density.argtypes = [S, P, P]
        _lib.oracle_lda_x.argtypes = [S, P, P]
        _lib.oracle_lda_x.restype = D
        _lib.oracle_apply_H.argtypes = [S, D, P, P, P]
        _lib.oracle_taylor_substep.argtypes = [S, D, D, P]
        _lib.oracle_observables.argtypes = [S, D, D, P, P]
        _lib.oracle_propagate.argtypes = [S, D, D, I, I, P, P]
        _lib.oracle_sphere_count.argtypes = [S, I]
        _lib.oracle_sphere_count.restype = I
        _lib.oracle_propagate_cfm4.argtypes = [S, D, D, I, I, P, P]
        _lib.oracle_cfm4_weights.argtypes = [I, P, P]
        _lib.oracle_cfm4_constants.argtypes = [P, P]
        _lib.oracle_propagate_emr.argtypes = [S, D, D, I, I, P, P]
        _lib.oracle_propagate_aetrs.argtypes = [S, D, D, I, I, P, P]
        _lib.oracle_propagate_etrs.argtypes = [S, D, D, I, I, P, P]
        _lib.oracle_propagate_rk4.argtypes = [S, D, D, I, I, P, P]
        _lib.oracle_hartree.argtypes = [S, P, P]
        _lib.oracle_hartree.restype = D
        _lib.oracle_hartree_self_cell.argtypes = []
        _lib.oracle_set_threads.argtypes = [I]
        _lib.oracle_band_energy.argtypes = [S, P, P]
        _lib.oracle_band_energy.restype = D
        _lib.oracle_velocity_expectation.argtypes = [S, P, P, I, P]
        _lib.oracle_set_threads.restype = I
        _lib.oracle_tsurff_flux.argtypes = [S, P, I, P, P, P, D, D, P, P]
        _lib.oracle_heat_current.argtypes = [S, P, P, P]
        _lib.oracle_volkov_step.argtypes = [S, D, D, P]
        _lib.oracle_tsurff_propagate.argtypes = [S, P, I, P, D, D, I, I, P, P, P, P, P]
        _lib.oracle_hartree_self_cell.restype = D
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class System:
    """An oracle view of one problem.  Holds contiguous copies of the inputs so the C
    struct's pointers stay valid for the object's lifetime."""

    def __init__(self, spec, inputs, *, xc=None, gauge=None, projectors=None, vloc=None):
        self.spec = spec
        self.N = spec.n_points
        self.vloc = np.ascontiguousarray(inputs.vloc if vloc is None else vloc, dtype=np.float64)
        self.kpts = np.ascontiguousarray(inputs.kpts, dtype=np.float64)
        self.kw = np.ascontiguousarray(inputs.kw, dtype=np.float64)
        self.pos = np.ascontiguousarray(inputs.pos, dtype=np.float64).reshape(-1, 3)
        self.D = np.ascontiguousarray(inputs.D, dtype=np.float64).reshape(-1, 4)
        use_proj = spec.projectors if projectors is None else projectors
        s = _Sys()
        s.nx, s.ny, s.nz, s.h = spec.nx, spec.ny, spec.nz, spec.h
        s.fd_order, s.bc, s.n_orb = spec.fd_order, spec.bc, spec.n_orb
        s.n_k = self.kpts.shape[0]
        s.kpts, s.kw, s.vloc = _ptr(self.kpts), _ptr(self.kw), _ptr(self.vloc)
        s.xc = spec.xc if xc is None else xc
        s.occ = spec.occ
        s.gauge = spec.gauge if gauge is None else gauge
        s.pol = (ctypes.c_double * 3)(*spec.pol)
        s.amp, s.omega, s.envelope, s.t_total = spec.amp, spec.omega, spec.envelope, spec.t_total
        s.n_atoms = self.pos.shape[0] if use_proj else 0
        s.pos, s.D = _ptr(self.pos), _ptr(self.D)
        s.r_c, s.r_cut = spec.r_c, spec.r_cut
        self._s = s
        self.lib = _load()
        self.shape = (s.n_k, spec.nz, spec.ny, spec.nx, spec.n_orb)

    @property
    def ref(self):
        return ctypes.byref(self._s)

    def _psi(self, psi) -> np.ndarray:
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        assert a.shape == self.shape, (a.shape, self.shape)
        return a

    def field(self, t):
        E, A = np.zeros(3), np.zeros(3)
        self.lib.oracle_field(self.ref, t, _ptr(E), _ptr(A))
        return E, A

    def density(self, psi) -> np.ndarray:
        psi = self._psi(psi)
        n = np.empty(self.N)
        self.lib.oracle_density(self.ref, _ptr(psi), _ptr(n))
        return n.reshape(self.spec.nz, self.spec.ny, self.spec.nx)

    def lda_x(self, n):
        n = np.ascontiguousarray(n, dtype=np.float64)
        vx = np.empty_like(n)
        ex = self.lib.oracle_lda_x(self.ref, _ptr(n), _ptr(vx))
        return ex, vx

    def hartree(self, n):
        """(E_H, v_H) of the density n: a direct sum over grid cells in a finite box, the
        exact plane-wave Poisson solve with a neutralising background in a periodic cell."""
        n = np.ascontiguousarray(n, dtype=np.float64)
        vh = np.empty_like(n)
        eh = self.lib.oracle_hartree(self.ref, _ptr(n), _ptr(vh))
        return eh, vh

    def band_energy(self, A, psi) -> float:
        """sum_k w_k f <phi|H(A)|phi> h^3 at an explicit vector potential A (no exchange)."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        return self.lib.oracle_band_energy(self.ref, _ptr(A), _ptr(self._psi(psi)))

    def velocity(self, A, psi, with_nonlocal=True) -> np.ndarray:
        """sum_k w_k f <phi| i[H, r] |phi> h^3 per axis at vector potential A; the projector
        commutator included when `with_nonlocal` is set."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        out = np.empty(3)
        self.lib.oracle_velocity_expectation(self.ref, _ptr(A), _ptr(self._psi(psi)), int(with_nonlocal), _ptr(out))
        return out

    def apply_H(self, psi, t=0.0, vx=None) -> np.ndarray:
        """H[vx, t] psi.  vx=None applies no exchange term; pass vx explicitly (e.g. from
        ``vx_of(psi_state)``) to apply the Hamiltonian of a given state's density."""
        psi = self._psi(psi)
        out = np.empty_like(psi)
        vptr = None
        if vx is not None:
            vx = np.ascontiguousarray(vx, dtype=np.float64)
            vptr = _ptr(vx)
        self.lib.oracle_apply_H(self.ref, t, vptr, _ptr(psi), _ptr(out))
        return out

    def vx_of(self, psi):
        """The density-dependent potential of psi's density: v_x (xc 1), v_x + v_H (xc 2)."""
        if self._s.xc not in (1, 2):
            return None
        n = self.density(psi)
        v = self.lda_x(n)[1]
        return v + self.hartree(n.ravel())[1].reshape(v.shape) if self._s.xc == 2 else v

    def taylor_substep(self, psi, t, dt) -> np.ndarray:
        psi = self._psi(psi).copy()
        self.lib.oracle_taylor_substep(self.ref, t, dt, _ptr(psi))
        return psi

    def observables(self, psi, t_state, t_field) -> np.ndarray:
        psi = self._psi(psi)
        obs = np.empty(8)
        self.lib.oracle_observables(self.ref, t_state, t_field, _ptr(psi), _ptr(obs))
        return obs

    def propagate(self, psi, t0, dt, n_steps, substeps, record=True):
        psi = self._psi(psi).copy()
        obs = np.empty((n_steps, 8)) if record else None
        self.lib.oracle_propagate(self.ref, t0, dt, n_steps, substeps, _ptr(psi),
                                  _ptr(obs) if record else None)
        return psi, obs

    def propagate_cfm4(self, psi, t0, dt, n_steps, substeps, record=True):
        """CFM4 (two exponentials per sub-step, v_x extrapolated from the last four
        sub-steps); length gauge or no field."""
        psi = self._psi(psi).copy()
        obs = np.empty((n_steps, 8)) if record else None
        self.lib.oracle_propagate_cfm4(self.ref, t0, dt, n_steps, substeps, _ptr(psi),
                                       _ptr(obs) if record else None)
        return psi, obs

    def propagate_emr(self, psi, t0, dt, n_steps, substeps, record=True):
        """Exponential midpoint rule, v_x extrapolated to the sub-step midpoint; length gauge
        or no field."""
        psi = self._psi(psi).copy()
        obs = np.empty((n_steps, 8)) if record else None
        self.lib.oracle_propagate_emr(self.ref, t0, dt, n_steps, substeps, _ptr(psi),
                                      _ptr(obs) if record else None)
        return psi, obs

    def propagate_aetrs(self, psi, t0, dt, n_steps, substeps, record=True):
        """Approximate enforced time-reversal symmetry: half exponentials with H at t and at
        t + ds (v_x extrapolated there); length gauge or no field."""
        psi = self._psi(psi).copy()
        obs = np.empty((n_steps, 8)) if record else None
        self.lib.oracle_propagate_aetrs(self.ref, t0, dt, n_steps, substeps, _ptr(psi),
                                        _ptr(obs) if record else None)
        return psi, obs

    def propagate_etrs(self, psi, t0, dt, n_steps, substeps, record=True):
        """Enforced time-reversal symmetry: H at t + ds from the density of the trial state
        exp(-i ds H[t]) psi; half exponentials with H at t and at t + ds; length gauge or no
        field."""
        psi = self._psi(psi).copy()
        obs = np.empty((n_steps, 8)) if record else None
        self.lib.oracle_propagate_etrs(self.ref, t0, dt, n_steps, substeps, _ptr(psi),
                                       _ptr(obs) if record else None)
        return psi, obs

    def propagate_rk4(self, psi, t0, dt, n_steps, substeps, record=True):
        """Classical Runge-Kutta 4 with the density rebuilt at every stage; any gauge."""
        psi = self._psi(psi).copy()
        obs = np.empty((n_steps, 8)) if record else None
        self.lib.oracle_propagate_rk4(self.ref, t0, dt, n_steps, substeps, _ptr(psi),
                                      _ptr(obs) if record else None)
        return psi, obs

    def tsurff_flux(self, psi, box, p, a=(0.0, 0.0, 0.0), alpha=(0.0, 0.0, 0.0), beta=0.0, t_rel=0.0):
        """t-SURFF flux F[i, p] = oint_S n . <chi_p| j |phi_i> ds of the orbitals psi through the
        box surface `box` = (i0, i1, j0, j1, k0, k1) (grid planes), for momenta p [n_p, 3], with
        the Volkov parameters a(t), alpha(t), beta(t) and the time t_rel since the accumulation
        started.  Finite boxes, one k-point."""
        psi = self._psi(psi)
        box = np.ascontiguousarray(box, dtype=np.int32)
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
        a, alpha = np.ascontiguousarray(a, dtype=np.float64), np.ascontiguousarray(alpha, dtype=np.float64)
        F = np.zeros((self.spec.n_orb, p.shape[0]), dtype=np.complex128)
        self.lib.oracle_tsurff_flux(self.ref, _ptr(box), p.shape[0], _ptr(p), _ptr(a), _ptr(alpha), float(beta),
                                    float(t_rel), _ptr(psi), _ptr(F))
        return F

    def volkov_step(self, vol, t, dt):
        """(a, alpha, beta) = vol[0:3], vol[3:6], vol[6] advanced from t to t + dt (RK4)."""
        vol = np.ascontiguousarray(vol, dtype=np.float64).copy()
        self.lib.oracle_volkov_step(self.ref, t, dt, _ptr(vol))
        return vol

    def propagate_tsurff(self, psi, t0, dt, n_steps, substeps, box, p, vol=None, t_rel=0.0, b=None, record=True):
        """Taylor-4 propagation with the t-SURFF amplitudes b[i, p] accumulated by the trapezoid
        rule over the configured steps.  Returns (psi, records, b, vol, t_rel); pass vol, t_rel
        and b back in to continue an accumulation."""
        psi = self._psi(psi).copy()
        box = np.ascontiguousarray(box, dtype=np.int32)
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
        vol = np.zeros(7) if vol is None else np.ascontiguousarray(vol, dtype=np.float64).copy()
        b = (np.zeros((self.spec.n_orb, p.shape[0]), dtype=np.complex128) if b is None
             else np.ascontiguousarray(b, dtype=np.complex128).copy())
        tr = ctypes.c_double(t_rel)
        obs = np.empty((n_steps, 8)) if record else None
        self.lib.oracle_tsurff_propagate(self.ref, _ptr(box), p.shape[0], _ptr(p), t0, dt, n_steps, substeps,
                                         _ptr(psi), _ptr(obs) if record else None, _ptr(vol), ctypes.byref(tr),
                                         _ptr(b))
        return psi, obs, b, vol, tr.value

    def heat_current(self, A, psi) -> np.ndarray:
        """Macroscopic kinetic heat current (1/Omega) sum_k w_k f int J_t at vector potential A
        (the printed kinetic term with its last pair antisymmetric; covariant derivatives)."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        out = np.empty(3)
        self.lib.oracle_heat_current(self.ref, _ptr(A), _ptr(self._psi(psi)), _ptr(out))
        return out

    def sphere_count(self, a: int) -> int:
        return self.lib.oracle_sphere_count(self.ref, a)


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops from now on; returns the previous count."""
    return _load().oracle_set_threads(n)


def hartree_self_cell() -> float:
    """c0 = integral of 1/|r| over the unit cube centred at 0 (a cell's own Coulomb term)."""
    return _load().oracle_hartree_self_cell()


def fd_weights(M: int):
    lib = _load()
    c, d = np.zeros(M + 1), np.zeros(M + 1)
    lib.oracle_fd_laplacian_weights(M, _ptr(c))
    lib.oracle_fd_gradient_weights(M, _ptr(d))
    return c, d


def cfm4_weights(nh: int):
    """Weights of the newest nh v_x (newest first) in the effective potentials of the
    first and second CFM4 exponentials."""
    lib = _load()
    wf, ws = np.zeros(4), np.zeros(4)
    lib.oracle_cfm4_weights(nh, _ptr(wf), _ptr(ws))
    return wf[:nh], ws[:nh]


def cfm4_constants():
    """(a1, a2), (theta1, theta2) of CFM4."""
    lib = _load()
    a, th = np.zeros(2), np.zeros(2)
    lib.oracle_cfm4_constants(_ptr(a), _ptr(th))
    return a, th
