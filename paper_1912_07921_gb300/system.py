"""Python view of one propagation system of the C library (argument marshalling only).

Device memory for ``apply_H`` operands and streams come from PyTorch; every step of the
propagation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _lib
from .inputs import (BC_BLOCH, PREC_C64, GAUGE_NONE, SystemSpec, Inputs)

RECORD = 8


def _dp(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def shape_count() -> int:
    n = ctypes.c_int()
    _lib.check(_lib.load().tdks_sweep_shape_info(0, ctypes.byref(n), None, None, None, None))
    return n.value


def shape_info(shape: int):
    """(tx, ty, rows, warps) of a TMA sweep tile shape: tx x ty points per work item, rows
    y-adjacent points per consumer thread, `warps` consumer warps."""
    tx, ty, rows, warps = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _lib.check(_lib.load().tdks_sweep_shape_info(shape, None, ctypes.byref(tx), ctypes.byref(ty),
                                                  ctypes.byref(rows), ctypes.byref(warps)))
    return tx.value, ty.value, rows.value, warps.value


class System:
    """One TDKS system resident on the current CUDA device."""

    def __init__(self, spec: SystemSpec, inputs: Optional[Inputs] = None, stream: Optional[int] = None,
                 orbitals: Optional[np.ndarray] = None, xc: Optional[int] = None,
                 projectors: Optional[bool] = None, gauge: Optional[int] = None):
        self.lib = _lib.load()
        self.spec = spec
        kpts = np.ascontiguousarray(inputs.kpts if inputs is not None else np.zeros((1, 3)), dtype=np.float64)
        kw = np.ascontiguousarray(inputs.kw if inputs is not None else np.ones(1), dtype=np.float64)
        self.n_k = kpts.shape[0]
        h = ctypes.c_void_p()
        _lib.check(self.lib.tdks_create_grid(spec.nx, spec.ny, spec.nz, spec.h, spec.fd_order, spec.bc,
                                             spec.prec, spec.n_orb, self.n_k, _dp(kpts), _dp(kw),
                                             ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        self.shape = (self.n_k, spec.nz, spec.ny, spec.nx, spec.n_orb)
        if inputs is not None:
            self.set_local_potential(inputs.vloc)
            use_proj = spec.projectors if projectors is None else projectors
            if use_proj and inputs.pos.shape[0] > 0:
                self.set_projectors(inputs.pos, inputs.D, spec.r_c, spec.r_cut)
        self.set_field(spec.gauge if gauge is None else gauge, spec.pol, spec.amp, spec.omega, spec.envelope,
                       spec.t_total)
        self.set_xc(spec.xc if xc is None else xc, spec.occ)
        psi = orbitals if orbitals is not None else (inputs.psi0 if inputs is not None else None)
        if psi is not None:
            self.set_orbitals(psi)

    # -- setters ---------------------------------------------------------------------
    def set_local_potential(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        _lib.check(self.lib.tdks_set_local_potential(self.h, _dp(v)))

    def set_projectors(self, pos, D, r_c, r_cut):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1, 4)
        _lib.check(self.lib.tdks_set_atoms_projectors(self.h, pos.shape[0], _dp(pos), _dp(D), r_c, r_cut))

    def set_field(self, gauge, pol, amp, omega, envelope, t_total):
        pol = np.ascontiguousarray(pol, dtype=np.float64)
        _lib.check(self.lib.tdks_set_field(self.h, gauge, _dp(pol), amp, omega, envelope, t_total))

    def set_xc(self, xc, occ):
        _lib.check(self.lib.tdks_set_xc(self.h, xc, occ))

    def set_orbitals(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        assert psi.shape == self.shape, (psi.shape, self.shape)
        _lib.check(self.lib.tdks_set_orbitals(self.h, _dp(psi)))

    def set_orbitals_ptr(self, host_ptr: int):
        """Orbitals from a host buffer (e.g. pinned memory) in the host layout."""
        _lib.check(self.lib.tdks_set_orbitals(self.h, ctypes.c_void_p(host_ptr)))

    def set_upload_buffers(self, n: int):
        """1 (default) or 2: with two, each upload packs into a second state buffer while
        the work enqueued before it runs (a stream of uploads); such a system joins no batch."""
        _lib.check(self.lib.tdks_set_upload_buffers(self.h, n))

    def set_tile(self, tx, ty, zc=0):
        _lib.check(self.lib.tdks_set_tile(self.h, tx, ty, zc))

    def heat_current(self, t_field: float) -> np.ndarray:
        """Macroscopic kinetic heat current of the current state (periodic cells), with the
        vector potential at t_field."""
        out = np.empty(3)
        _lib.check(self.lib.tdks_heat_current(self.h, t_field, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def set_tsurff(self, box, p):
        """t-SURFF amplitudes through the surface of the box of grid planes `box` =
        (i0, i1, j0, j1, k0, k1) for momenta p [n_p, 3], accumulated from the next propagation
        on; an empty p turns it off."""
        box = np.ascontiguousarray(box, dtype=np.int32)
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
        self._ts_np = p.shape[0]
        _lib.check(self.lib.tdks_set_tsurff(self.h, _dp(box), p.shape[0], _dp(p)))

    def tsurff(self):
        """(b [n_orb, n_p] complex128, time since the accumulation started)."""
        b = np.empty((self.spec.n_orb, self._ts_np), dtype=np.complex128)
        t = ctypes.c_double(0.0)
        _lib.check(self.lib.tdks_get_tsurff(self.h, _dp(b), ctypes.byref(t)))
        return b, t.value

    def set_failure_injection(self, withhold: bool):
        """Failure injection (tests): the TMA sweeps' producers withhold every copy, so the
        consumers' bounded waits run out (~2 s) and the next synchronising call raises
        TDKS_ETIMEOUT; False restores normal sweeps."""
        _lib.check(self.lib.tdks_set_failure_injection(self.h, int(bool(withhold))))

    def set_sweep_path(self, path: int):
        """0: TMA-fed warp-specialised sweep where it applies (finite boxes, 16x8 tiles);
        1: general sweep; 2: TMA-fed sweep with all warps of a CTA in lockstep."""
        _lib.check(self.lib.tdks_set_sweep_path(self.h, path))

    def set_sweep_shape(self, sweep: int, shape: int):
        """Tile shape of one Taylor-term sweep (0..3; -1: all) of the TMA sweep."""
        _lib.check(self.lib.tdks_set_sweep_shape(self.h, sweep, shape))

    def sweep_shapes(self):
        """The tile shape of each of the four Taylor-term sweeps."""
        out = []
        for i in range(4):
            v = ctypes.c_int()
            _lib.check(self.lib.tdks_get_sweep_shape(self.h, i, ctypes.byref(v)))
            out.append(v.value)
        return out

    def autotune(self, reps: int = 5) -> np.ndarray:
        """Time every tile shape on each Taylor-term sweep of this system and keep the
        fastest per sweep; returns the mean ms per launch as [shape][sweep] (-1 where the
        system does not take the TMA sweep)."""
        n = shape_count()
        ms = np.zeros(n * 4, dtype=np.float64)
        _lib.check(self.lib.tdks_autotune(self.h, reps, ms.ctypes.data_as(_lib.PD)))
        return ms.reshape(n, 4)

    # -- queries ---------------------------------------------------------------------
    def get_orbitals(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.complex128)
        _lib.check(self.lib.tdks_get_orbitals(self.h, _dp(out)))
        return out

    def layout(self):
        bs, nb, eb, nbytes = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _lib.check(self.lib.tdks_layout(self.h, ctypes.byref(bs), ctypes.byref(nb), ctypes.byref(eb),
                                        ctypes.byref(nbytes)))
        return bs.value, nb.value, eb.value, nbytes.value

    def pack(self, psi: np.ndarray) -> np.ndarray:
        """Host layout [k][z][y][x][orb] -> packed layout [k][b][z][y][x][BS] (zero-padded),
        complex64 for complex64 systems."""
        bs, nb, eb, _ = self.layout()
        k, z, y, x, o = self.shape
        pad = np.zeros((k, z, y, x, nb * bs), dtype=np.complex128)
        pad[..., :o] = psi
        out = pad.reshape(k, z, y, x, nb, bs).transpose(0, 4, 1, 2, 3, 5)
        return np.ascontiguousarray(out, dtype=np.complex64 if eb == 8 else np.complex128)

    def unpack(self, packed: np.ndarray) -> np.ndarray:
        bs, nb, _, _ = self.layout()
        k, z, y, x, o = self.shape
        a = np.asarray(packed).reshape(k, nb, z, y, x, bs).transpose(0, 2, 3, 4, 1, 5)
        return a.reshape(k, z, y, x, nb * bs)[..., :o].astype(np.complex128)

    def apply_H(self, t: float, dev_in: int, dev_out: int):
        """dev_in / dev_out: device pointers (e.g. torch tensor .data_ptr()) in the packed layout."""
        self._xcheck(self.lib.tdks_apply_H(self.h, t, ctypes.c_void_p(dev_in), ctypes.c_void_p(dev_out)))

    def set_propagator(self, propagator: int):
        """0: Taylor-4 (default); 1: CFM4 (two exponentials per sub-step); 2: exponential
        midpoint rule; 3: approximate enforced time-reversal symmetry (two half exponentials);
        4: classical Runge-Kutta 4 (complex128); 5: enforced time-reversal symmetry with its
        trial state (three exponentials per sub-step)."""
        _lib.check(self.lib.tdks_set_propagator(self.h, propagator))

    def set_exchange(self, fn):
        """Make this system one rank of a state-parallel run (tdks_set_exchange).

        ``fn(ptr, n, stream) -> None`` must replace the n doubles at device address ``ptr``
        with their sum over all ranks, ordered after the work already on the CUDA stream
        handle ``stream`` and before what is enqueued there later (see
        ``sharding.allreduce_exchange``).  ``None`` detaches the hook.  An exception in ``fn``
        makes the library call that invoked it fail with TDKS_EDEVICE.
        """
        if fn is None:
            _lib.check(self.lib.tdks_set_exchange(self.h, None, None))
            self._xcb = None
            return

        def hook(ptr, n, stream, ctx):
            try:
                fn(ptr, n, stream)
                return 0
            except BaseException as exc:  # reported through the library's status code
                self._x_error = exc
                return 1

        cb = _lib.EXCHANGE_FN(hook)
        _lib.check(self.lib.tdks_set_exchange(self.h, ctypes.cast(cb, ctypes.c_void_p), None))
        self._xcb = cb  # the C side keeps only the pointer
        self._x_error = None

    def _xcheck(self, code: int):
        """check() that chains the exchange hook's exception when the hook failed."""
        exc, self._x_error = getattr(self, "_x_error", None), None
        if code != 0 and exc is not None:
            raise _lib.TdksError(code, _lib.load().tdks_last_error().decode()) from exc
        _lib.check(code)

    def propagate(self, t0: float, dt: float, n_steps: int, substeps: int = 0):
        self._xcheck(self.lib.tdks_propagate_n(self.h, t0, dt, n_steps, substeps))

    def auto_substeps(self, dt: float) -> int:
        s = ctypes.c_int()
        _lib.check(self.lib.tdks_auto_substeps(self.h, dt, ctypes.byref(s)))
        return s.value

    def step_count(self) -> int:
        c = ctypes.c_longlong()
        _lib.check(self.lib.tdks_step_count(self.h, ctypes.byref(c)))
        return c.value

    def reductions(self, step_from: int = 0, n: Optional[int] = None) -> np.ndarray:
        if n is None:
            n = self.step_count() - step_from
        out = np.empty((n, RECORD))
        _lib.check(self.lib.tdks_reductions(self.h, step_from, n, _dp(out)))
        return out

    def observe(self, t_state: float, t_field: float) -> np.ndarray:
        out = np.empty(RECORD)
        self._xcheck(self.lib.tdks_observe(self.h, t_state, t_field, _dp(out)))
        return out

    def set_profiling(self, on: bool):
        _lib.check(self.lib.tdks_set_profiling(self.h, int(on)))

    def kernel_time(self, kind: int = 0):
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        _lib.check(self.lib.tdks_kernel_time(self.h, kind, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def launch_count(self) -> int:
        c = ctypes.c_longlong()
        _lib.check(self.lib.tdks_launch_count(self.h, ctypes.byref(c)))
        return c.value

    def set_clock(self, t: float, dt: float, substeps: int):
        _lib.check(self.lib.tdks_set_clock(self.h, t, dt, substeps))

    def clock(self):
        t, n = ctypes.c_double(), ctypes.c_longlong()
        _lib.check(self.lib.tdks_get_clock(self.h, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    # -- checkpoint / resume ----------------------------------------------------------
    def save(self, path: str):
        """Write a checkpoint (tdks_save): the loaded system continues bit for bit."""
        _lib.check(self.lib.tdks_save(self.h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, stream: Optional[int] = None) -> "System":
        """A system restored from a checkpoint of tdks_save (tdks_load), on `stream`.  The
        spec reflects the file's grid, precision and counts (header fields 0..7 and 11 are
        nx, ny, nz, FD order, bc, precision, orbitals, k-points and atoms; double 0 is h)."""
        with open(path, "rb") as f:
            head = f.read(8 + 32 * 8 + 16 * 8)
        if len(head) < 8 + 32 * 8 + 16 * 8:
            raise _lib.TdksError(1, f"{path}: not a checkpoint file")
        ints = np.frombuffer(head, dtype="<i8", count=32, offset=8)
        dbl = np.frombuffer(head, dtype="<f8", count=16, offset=8 + 32 * 8)
        self = cls.__new__(cls)
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self.lib.tdks_load(os.fsencode(path), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        self.h = h
        nx, ny, nz, order, bc, prec, n_orb, n_k = (int(v) for v in ints[:8])
        self.spec = SystemSpec(nx=nx, ny=ny, nz=nz, h=float(dbl[0]), fd_order=order, bc=bc, prec=prec,
                               n_orb=n_orb, n_k=n_k, n_atoms=int(ints[11]))
        self.n_k = n_k
        self.shape = (n_k, nz, ny, nx, n_orb)
        return self

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tdks_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many finite-box systems advanced together (one persistent sweep launch per Taylor
    term over all of them, replayed as a CUDA graph).  The systems must use the batch's
    stream and share FD order, precision and sub-step count."""

    def __init__(self, systems, stream: Optional[int] = None):
        self.lib = _lib.load()
        self.systems = list(systems)
        arr = (ctypes.c_void_p * len(self.systems))(*[s.h.value for s in self.systems])
        h = ctypes.c_void_p()
        _lib.check(self.lib.tdks_batch_create(arr, len(self.systems), ctypes.c_void_p(stream or 0),
                                              ctypes.byref(h)))
        self.h = h

    def propagate(self, n_steps: int, use_graph: bool = True):
        _lib.check(self.lib.tdks_batch_propagate(self.h, n_steps, int(use_graph)))

    def launch_count(self) -> int:
        c = ctypes.c_longlong()
        _lib.check(self.lib.tdks_batch_launch_count(self.h, ctypes.byref(c)))
        return c.value

    def set_shape(self, term: int, shape: int):
        """Sweep tile shape of one Taylor term (0..3; -1: all) of the batched sweep."""
        _lib.check(self.lib.tdks_batch_set_shape(self.h, term, shape))

    def shapes(self):
        out = []
        for k in range(4):
            v = ctypes.c_int()
            _lib.check(self.lib.tdks_batch_get_shape(self.h, k, ctypes.byref(v)))
            out.append(v.value)
        return out

    def autotune(self, reps: int = 3) -> np.ndarray:
        """Time every tile shape on each Taylor term's batched sweep and keep the fastest;
        returns the mean ms per launch as [shape][term]."""
        n = shape_count()
        ms = np.zeros(n * 4, dtype=np.float64)
        _lib.check(self.lib.tdks_batch_autotune(self.h, reps, ms.ctypes.data_as(_lib.PD)))
        return ms.reshape(n, 4)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tdks_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
