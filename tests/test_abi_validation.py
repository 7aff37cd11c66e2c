"""Argument checks of the C interface that return before any CUDA call, so they run on a CPU:
bad grids, orders, precisions and counts are refused with TDKS_EINVAL (and the thread's
error message says why), NULL handles are refused, and the tile-shape table is consistent
with the shapes' own constraints (every consumer thread owns R y-adjacent points of one
16-byte vector: CW warps x 32 = 4 vectors x TX x TY / R)."""
import ctypes

import numpy as np

import pytest

EINVAL = 1


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_07921_gb300 import _lib
    return _lib.load()


def _create(lib, nx=8, ny=8, nz=8, h=0.3, order=4, bc=0, prec=0, n_orb=2, n_k=1):
    out = ctypes.c_void_p()
    rc = lib.tdks_create_grid(nx, ny, nz, h, order, bc, prec, n_orb, n_k, None, None, None, ctypes.byref(out))
    return rc, out.value


@pytest.mark.parametrize("kw,msg", [
    (dict(order=6), b"fd_order"),
    (dict(bc=2), b"bc"),
    (dict(prec=2), b"prec"),
    (dict(nx=4, order=8), b"too small"),      # a finite box needs M + 1 points per axis
    (dict(ny=2, order=4), b"too small"),
    (dict(h=0.0), b"h must be"),
    (dict(h=float("nan")), b"h must be"),
    (dict(n_orb=0), b"n_orb"),
    (dict(n_k=0), b"n_k"),
    (dict(n_k=2), b"one k-point"),            # finite boxes take exactly one k-point
    (dict(nx=1100, ny=1100, nz=1000), b"2^30"),
])
def test_create_grid_refuses_bad_arguments(lib, kw, msg):
    rc, handle = _create(lib, **kw)
    assert rc == EINVAL and handle is None
    assert msg in lib.tdks_last_error()


def test_create_grid_refuses_a_null_output(lib):
    assert lib.tdks_create_grid(8, 8, 8, 0.3, 4, 0, 0, 2, 1, None, None, None, None) == EINVAL


def test_calls_on_a_null_system_are_refused(lib):
    assert lib.tdks_destroy(None) == 0  # freeing nothing is fine
    assert lib.tdks_set_propagator(None, 0) == EINVAL
    assert lib.tdks_set_exchange(None, None, None) == EINVAL
    assert lib.tdks_propagate_n(None, 0.0, 0.01, 1, 1) == EINVAL
    assert lib.tdks_set_sweep_shape(None, 0, 0) == EINVAL
    assert lib.tdks_apply_H(None, 0.0, None, None) == EINVAL
    out = ctypes.c_void_p()
    assert lib.tdks_batch_create(None, 0, None, ctypes.byref(out)) == EINVAL
    assert lib.tdks_set_tsurff(None, None, 0, None) == EINVAL
    assert lib.tdks_get_tsurff(None, None, None) == EINVAL
    assert lib.tdks_set_failure_injection(None, 0) == EINVAL
    assert lib.tdks_set_upload_buffers(None, 2) == EINVAL
    out3 = np.empty(3)
    assert lib.tdks_heat_current(None, 0.0, out3.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == EINVAL
    assert lib.tdks_fma_rate(0, None) == EINVAL
    assert lib.tdks_fma_rate(7, ctypes.byref(ctypes.c_double())) == EINVAL


def test_noalloc_entry_refuses_bad_arguments(lib):
    buf = ctypes.c_void_p(16)  # never dereferenced: every case fails its checks first
    assert lib.tdks_apply_H_noalloc(8, 8, 8, 0.3, 6, 0, 1, buf, buf, ctypes.c_void_p(32), None) == EINVAL
    assert lib.tdks_apply_H_noalloc(8, 8, 8, 0.3, 4, 0, 1, buf, buf, buf, None) == EINVAL  # in == out
    assert lib.tdks_apply_H_noalloc(4, 8, 8, 0.3, 8, 0, 1, buf, buf, ctypes.c_void_p(32), None) == EINVAL
    assert lib.tdks_apply_H_noalloc(128, 128, 128, 0.3, 4, 0, 1, buf, buf, ctypes.c_void_p(32), None) == EINVAL
    assert b"at most" in lib.tdks_last_error()


def test_sweep_shape_table(lib):
    n = ctypes.c_int()
    assert lib.tdks_sweep_shape_info(0, ctypes.byref(n), None, None, None, None) == 0
    assert n.value >= 1
    for shape in range(n.value):
        tx, ty, r, w = (ctypes.c_int() for _ in range(4))
        assert lib.tdks_sweep_shape_info(shape, None, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(r),
                                         ctypes.byref(w)) == 0
        assert ty.value % r.value == 0
        # 16-byte thread vectors (4 per point); shape 5 runs complex64 systems with 8-byte ones
        vectors = 8 if shape == 5 else 4
        assert w.value * 32 == vectors * tx.value * ty.value // r.value
    assert lib.tdks_sweep_shape_info(n.value, None, None, None, None, None) == EINVAL
    assert lib.tdks_sweep_shape_info(-1, None, None, None, None, None) == EINVAL
