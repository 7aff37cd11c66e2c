"""tdks_apply_H_noalloc: the H application for callers that may not allocate device memory.

Some callers cannot call cudaMalloc (a host framework that owns all device memory through
its own pool, or a real-time loop that cannot afford the device synchronisation an
allocation may cause).  The no-allocation entry point keeps its scratch in a fixed
file-scope device array; this test calls it through the C interface, twice in a row on
different inputs, and checks each result against tdks_apply_H of a system built for the
same Hamiltonian (kinetic stencil plus local potential).  It lives in a file collected
last so that a run stopping at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1912_07921_gb300 import inputs as I
from tests._util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _reference(spec, inp, psi, stream):
    """H psi through the existing entry point (a system with no exchange, no projectors, no field)."""
    from paper_1912_07921_gb300.system import System
    s = System(spec, inp, stream=stream, xc=I.XC_NONE, projectors=False, gauge=I.GAUGE_NONE)
    packed = s.pack(psi)
    view = np.float32 if packed.dtype == np.complex64 else np.float64
    din = torch.from_numpy(packed.view(view)).cuda()
    dout = torch.empty_like(din)
    s.apply_H(0.0, din.data_ptr(), dout.data_ptr())
    torch.cuda.synchronize()
    out = dout.cpu().numpy().view(packed.dtype).reshape(packed.shape)
    s.close()
    return packed, out


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_noalloc_matches_apply_H_on_two_calls(prec):
    from paper_1912_07921_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [I.SystemSpec(nx=37, ny=21, nz=19, h=0.3, fd_order=8, prec=prec, n_orb=5, n_atoms=3, seed=3),
             I.SystemSpec(nx=24, ny=30, nz=17, h=0.25, fd_order=4, prec=prec, n_orb=9, n_atoms=2, seed=4)]
    for i, spec in enumerate(cases):
        inp = I.make_inputs(spec, with_orbitals=False)
        psi = I.random_orbitals(spec, 100 + i)
        packed, ref = _reference(spec, inp, psi, stream)
        view = np.float32 if packed.dtype == np.complex64 else np.float64
        din = torch.from_numpy(packed.view(view)).cuda()
        dout = torch.full_like(din, float("nan"))
        vloc = torch.from_numpy(np.ascontiguousarray(inp.vloc)).cuda()
        rc = lib.tdks_apply_H_noalloc(spec.nx, spec.ny, spec.nz, spec.h, spec.fd_order, spec.prec, spec.n_orb,
                                      ctypes.c_void_p(vloc.data_ptr()), ctypes.c_void_p(din.data_ptr()),
                                      ctypes.c_void_p(dout.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, lib.tdks_last_error().decode()
        got = dout.cpu().numpy().view(packed.dtype).reshape(packed.shape)
        tol = 1e-12 if prec == I.PREC_C128 else 5e-6
        assert rel_err(got, ref) < tol


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1912_07921_gb300 import _lib
    lib = _lib.load()
    rc = lib.tdks_apply_H_noalloc(128, 128, 128, 0.25, 4, I.PREC_C64, 8, ctypes.c_void_p(16),
                                  ctypes.c_void_p(32), ctypes.c_void_p(48), ctypes.c_void_p(0))
    assert rc == 1
    assert "at most" in lib.tdks_last_error().decode()
