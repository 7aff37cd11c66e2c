"""State-parallel propagation of one system over several GPUs, one process per GPU.

The orbitals of a Kohn-Sham system couple only through the density n(r) = sum_i f_i
|phi_i(r)|^2 that enters v_x[n] (Sec. "New propagators for real-time TDDFT": H[n(t), t]);
given H, every orbital advances alone.  The paper's multi-GPU runs distribute the states
only and keep the grid whole on every GPU (Sec. "GPUs"), because a distributed grid needs
far more frequent communication.  Here each rank holds a contiguous slice of the orbitals
(``state_slice``) in its own library system, and the library calls an exchange hook
(``tdks_set_exchange``) where the whole system's density is needed: once per density a
sub-step builds a potential from (one per Taylor-4 sub-step; two for ETRS; four for RK4)
with this rank's density (N doubles), and once per observable record with this rank's band
energy and current sums (4 doubles).  ``allreduce_exchange`` is that hook over
``torch.distributed`` (NCCL on GPUs), enqueued on the library's own CUDA stream.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import numpy as np


def state_slice(n_orb: int, rank: int, world: int, block: int = 1) -> Tuple[int, int]:
    """Orbitals [lo, hi) of `rank` out of `world`: whole blocks of `block` orbitals (the
    library's batch width keeps every rank's batches full), spread as evenly as possible,
    lower ranks taking the extra block; the last block may be partial."""
    if world < 1 or not 0 <= rank < world or block < 1 or n_orb < 0:
        raise ValueError("bad slice request")
    n_blocks = -(-n_orb // block)
    q, r = divmod(n_blocks, world)
    b0 = rank * q + min(rank, r)
    b1 = b0 + q + (1 if rank < r else 0)
    return min(b0 * block, n_orb), min(b1 * block, n_orb)


class DeviceDoubles:
    """A device buffer of n doubles at address ptr, seen through the CUDA array interface
    (``torch.as_tensor(DeviceDoubles(ptr, n), device="cuda")`` makes a view, no copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "stream": None}


def _host_doubles(ptr: int, n: int) -> np.ndarray:
    return np.ctypeslib.as_array((ctypes.c_double * n).from_address(ptr))


def allreduce_exchange(group=None, device: str = "cuda"):
    """Exchange hook for ``System.set_exchange``: the sum over the ranks of ``group``
    (torch.distributed; default group if None), in place.

    device: "cuda" (the library's buffers, which are device memory): the allreduce is issued
    with the library's stream as the current stream, so it starts after the kernels that wrote
    the buffer and the library's later kernels wait for it.  "cpu": buffers in host memory, for
    a hook driven from host code (e.g. over gloo); never for the library's own buffers.
    """
    import torch
    import torch.distributed as dist

    if device not in ("cuda", "cpu"):
        raise ValueError("device must be 'cuda' or 'cpu'")

    def fn(ptr: int, n: int, stream: Optional[int]) -> None:
        if device == "cpu":
            dist.all_reduce(torch.from_numpy(_host_doubles(ptr, n)), op=dist.ReduceOp.SUM, group=group)
            return
        dev = torch.cuda.current_device()
        buf = torch.as_tensor(DeviceDoubles(ptr, n), device=f"cuda:{dev}")
        st = torch.cuda.ExternalStream(stream, device=dev) if stream else torch.cuda.default_stream(dev)
        with torch.cuda.stream(st):
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)

    return fn


def shard_system(spec, inputs, rank: int, world: int, *, stream: Optional[int] = None, group=None,
                 block: Optional[int] = None, **kw):
    """One rank's library system: the slice of `spec`'s orbitals that `state_slice` gives
    this rank, with the exchange hook set.  Returns (system, (lo, hi))."""
    import dataclasses

    from .inputs import PREC_C64
    from .system import System

    bs = block or (8 if spec.prec == PREC_C64 else 4)
    lo, hi = state_slice(spec.n_orb, rank, world, bs)
    if hi <= lo:
        raise ValueError(f"rank {rank} of {world} gets no orbitals of {spec.n_orb}")
    sub = dataclasses.replace(spec, n_orb=hi - lo)
    psi = inputs.psi0[..., lo:hi] if inputs.psi0 is not None else None
    sys_ = System(sub, inputs, stream=stream, orbitals=psi, **kw)
    sys_.set_exchange(allreduce_exchange(group))
    return sys_, (lo, hi)
