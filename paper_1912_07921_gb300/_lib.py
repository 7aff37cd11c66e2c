"""ctypes binding of ``libtdks.so`` (the C interface declared in ``include/tdks.h``).

Argument marshalling only: every step of the propagation runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtdks.so")

# Every exported symbol with (argtypes, restype); the header declares the same set.
P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
PI, PD, PLL = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)
SIGNATURES = {
    "tdks_create_grid": ([I, I, I, D, I, I, I, I, I, P, P, P, ctypes.POINTER(P)], I),
    "tdks_destroy": ([P], I),
    "tdks_set_local_potential": ([P, P], I),
    "tdks_set_orbitals": ([P, P], I),
    "tdks_set_upload_buffers": ([P, I], I),
    "tdks_get_orbitals": ([P, P], I),
    "tdks_set_atoms_projectors": ([P, I, P, P, D, D], I),
    "tdks_set_field": ([P, I, P, D, D, I, D], I),
    "tdks_set_xc": ([P, I, D], I),
    "tdks_layout": ([P, PI, PI, PI, PLL], I),
    "tdks_apply_H": ([P, D, P, P], I),
    "tdks_propagate_n": ([P, D, D, I, I], I),
    "tdks_set_propagator": ([P, I], I),
    "tdks_set_exchange": ([P, P, P], I),
    "tdks_save": ([P, ctypes.c_char_p], I),
    "tdks_load": ([ctypes.c_char_p, P, ctypes.POINTER(P)], I),
    "tdks_auto_substeps": ([P, D, PI], I),
    "tdks_reductions": ([P, LL, I, P], I),
    "tdks_step_count": ([P, PLL], I),
    "tdks_observe": ([P, D, D, P], I),
    "tdks_set_profiling": ([P, I], I),
    "tdks_kernel_time": ([P, I, PD, PLL], I),
    "tdks_launch_count": ([P, PLL], I),
    "tdks_set_tile": ([P, I, I, I], I),
    "tdks_set_sweep_path": ([P, I], I),
    "tdks_set_failure_injection": ([P, I], I),
    "tdks_sweep_shape_info": ([I, PI, PI, PI, PI, PI], I),
    "tdks_set_sweep_shape": ([P, I, I], I),
    "tdks_get_sweep_shape": ([P, I, PI], I),
    "tdks_autotune": ([P, I, PD], I),
    "tdks_set_clock": ([P, D, D, I], I),
    "tdks_get_clock": ([P, PD, PLL], I),
    "tdks_batch_create": ([P, I, P, ctypes.POINTER(P)], I),
    "tdks_batch_propagate": ([P, I, I], I),
    "tdks_batch_launch_count": ([P, PLL], I),
    "tdks_batch_destroy": ([P], I),
    "tdks_batch_set_shape": ([P, I, I], I),
    "tdks_batch_get_shape": ([P, I, PI], I),
    "tdks_batch_autotune": ([P, I, PD], I),
    "tdks_apply_H_noalloc": ([I, I, I, D, I, I, I, P, P, P, P], I),
    "tdks_fma_rate": ([I, PD], I),
    "tdks_set_tsurff": ([P, P, I, P], I),
    "tdks_heat_current": ([P, D, PD], I),
    "tdks_get_tsurff": ([P, P, PD], I),
    "tdks_last_error": ([], ctypes.c_char_p),
}

# C type of the exchange hook of tdks_set_exchange: (dev_buf, n, stream, ctx) -> status
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


class TdksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tdks error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build() or paper_1912_07921_gb300/build.py)")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def check(code: int):
    if code != 0:
        raise TdksError(code, load().tdks_last_error().decode())
