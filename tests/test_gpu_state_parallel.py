"""State-parallel propagation on the GPU, through the C interface's exchange hook.

Two ranks are emulated inside one process: two library systems, each with its slice of the
orbitals on its own CUDA stream, driven from two host threads.  Their exchange hook sums
the ranks' buffers on the host side of the stream order (stream synchronise, a host
barrier, the sum in rank order, a second barrier, the write-back); no kernel waits on
another.  The orbitals and records of the sharded run must match one system holding every
orbital (complex128: to 1e-12; the only difference is the order of the density sum over
batches) and the FP64 oracle.  A second test runs the torch.distributed hook over a
one-rank NCCL group: the same arithmetic as the unsharded system, so bit-identical
complex128 results.
"""
import dataclasses
import os
import socket
import threading

import numpy as np
import pytest

import oracle
from paper_1912_07921_gb300 import inputs as I
from tests._util import ragged_molecule, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


class ThreadGroup:
    """Host-side sum over `world` threads, each the rank of one system."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.bufs = [None] * world
        self.calls = [0] * world

    def hook(self, rank):
        from paper_1912_07921_gb300.sharding import DeviceDoubles

        def fn(ptr, n, stream):
            st = torch.cuda.ExternalStream(stream)
            buf = torch.as_tensor(DeviceDoubles(ptr, n), device="cuda")
            st.synchronize()  # the kernels that wrote this rank's buffer are done
            self.bufs[rank] = buf
            self.bar.wait()
            with torch.cuda.stream(st):
                acc = self.bufs[0].clone()
                for r in range(1, self.world):
                    acc += self.bufs[r]
            st.synchronize()
            self.bar.wait()  # every rank has read every buffer
            with torch.cuda.stream(st):
                buf.copy_(acc)
            self.calls[rank] += 1

        return fn


def _rec_err(rec, rec_o):
    """Per-column error relative to each column's scale (the dipole crosses zero)."""
    return max(float(np.max(np.abs(rec[:, c] - rec_o[:, c])) / np.max(np.abs(rec_o[:, c])))
               for c in range(rec.shape[1]) if np.max(np.abs(rec_o[:, c])) > 0)


def _run_sharded(spec, inp, world, steps, substeps, block, prop=0):
    from paper_1912_07921_gb300.sharding import state_slice
    from paper_1912_07921_gb300.system import System

    grp = ThreadGroup(world)
    systems, slices, streams = [], [], []
    for r in range(world):
        lo, hi = state_slice(spec.n_orb, r, world, block)
        st = torch.cuda.Stream()
        s = System(dataclasses.replace(spec, n_orb=hi - lo), inp, stream=st.cuda_stream,
                   orbitals=inp.psi0[..., lo:hi])
        s.set_exchange(grp.hook(r))
        s.set_propagator(prop)
        systems.append(s)
        slices.append((lo, hi))
        streams.append(st)
    errors = [None] * world

    def drive(r):
        try:
            systems[r].propagate(0.0, spec.dt, steps, substeps)
            streams[r].synchronize()
        except BaseException as exc:  # reported below
            errors[r] = exc
            grp.bar.abort()

    threads = [threading.Thread(target=drive, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in errors:
        if e is not None:
            raise e
    psi = np.concatenate([s.get_orbitals() for s in systems], axis=-1)
    recs = [s.reductions(0, steps) for s in systems]
    for s in systems:
        s.close()
    return psi, recs, grp.calls


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_two_thread_ranks_match_one_system_and_the_oracle(prec):
    from paper_1912_07921_gb300.system import System

    spec = ragged_molecule(prec, n_orb=11)
    inp = I.make_inputs(spec)
    steps, substeps = 3, 2
    block = 8 if prec == I.PREC_C64 else 4
    psi_sh, recs, calls = _run_sharded(spec, inp, 2, steps, substeps, block)
    # one density exchange per sub-step and one record exchange per step, on both ranks
    assert calls == [steps * substeps + steps] * 2
    whole = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    whole.propagate(0.0, spec.dt, steps, substeps)
    psi_w = whole.get_orbitals()
    rec_w = whole.reductions(0, steps)
    whole.close()
    ref_psi, ref_rec = oracle.System(spec, inp).propagate(inp.psi0, 0.0, spec.dt, steps, substeps)
    # complex128: the sharded run differs from one system only in the order of the density
    # sum over batches; complex64: also in the FP32 rounding of that sum's parts
    tol_w, tol_o = (1e-12, 1e-12) if prec == I.PREC_C128 else (1e-6, 2e-5)
    for rec in recs:  # every rank's record is the whole system's
        assert _rec_err(rec, rec_w) < tol_w
        assert _rec_err(rec, ref_rec) < tol_o
    assert rel_err(psi_sh, psi_w) < tol_w
    assert rel_err(psi_sh, ref_psi) < tol_o


def test_two_thread_ranks_periodic_cell_currents():
    """A periodic cell in the velocity gauge with k-points: the record's current is the sum of
    the ranks' current partials (exchanged with the band energy), so a sharded run must give
    the whole system's current and energy.  complex128 against one system and the oracle."""
    from tests._util import bloch_cell, bloch_inputs
    from paper_1912_07921_gb300.system import System

    spec = bloch_cell(I.PREC_C128, n_orb=7)
    inp = bloch_inputs(spec)
    steps, substeps = 3, 2
    psi_sh, recs, calls = _run_sharded(spec, inp, 2, steps, substeps, 4)
    assert calls == [steps * substeps + steps] * 2
    whole = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    whole.propagate(0.0, spec.dt, steps, substeps)
    psi_w, rec_w = whole.get_orbitals(), whole.reductions(0, steps)
    whole.close()
    ref_psi, ref_rec = oracle.System(spec, inp).propagate(inp.psi0, 0.0, spec.dt, steps, substeps)
    assert np.max(np.abs(rec_w[:, 4:7])) > 0  # the current is recorded
    for rec in recs:
        assert _rec_err(rec, rec_w) < 1e-12
        assert _rec_err(rec, ref_rec) < 1e-12
    assert rel_err(psi_sh, psi_w) < 1e-12
    assert rel_err(psi_sh, ref_psi) < 1e-12


@pytest.mark.parametrize("prop,name,per_sub", [(1, "cfm4", 1), (2, "emr", 1), (3, "aetrs", 1), (5, "etrs", 2),
                                               (4, "rk4", 4)])
def test_two_thread_ranks_with_every_propagator(prop, name, per_sub):
    """Every propagator state-parallel: the density each one builds its potential from (the
    pushed v_x of CFM4, EMR and AETRS, ETRS's state and trial, every RK4 stage) is summed over
    the ranks first.  complex128 against one system and the oracle."""
    from paper_1912_07921_gb300.system import System

    spec = ragged_molecule(I.PREC_C128, n_orb=7)
    inp = I.make_inputs(spec)
    steps, substeps = 2, 2
    psi_sh, recs, calls = _run_sharded(spec, inp, 2, steps, substeps, 4, prop=prop)
    # per sub-step: the densities of its potentials; per step: the record's density and sums
    assert calls == [steps * (per_sub * substeps + 2)] * 2
    whole = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    whole.set_propagator(prop)
    whole.propagate(0.0, spec.dt, steps, substeps)
    psi_w, rec_w = whole.get_orbitals(), whole.reductions(0, steps)
    whole.close()
    ref_psi, ref_rec = getattr(oracle.System(spec, inp), "propagate_" + name)(inp.psi0, 0.0, spec.dt, steps,
                                                                                substeps)
    for rec in recs:
        assert _rec_err(rec, rec_w) < 1e-12
        assert _rec_err(rec, ref_rec) < 1e-12
    assert rel_err(psi_sh, psi_w) < 1e-12
    assert rel_err(psi_sh, ref_psi) < 1e-12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_nccl_hook_on_one_rank_is_bit_identical_to_one_system():
    import torch.distributed as dist
    from paper_1912_07921_gb300.sharding import shard_system
    from paper_1912_07921_gb300.system import System

    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0, world_size=1)
    try:
        spec = ragged_molecule(I.PREC_C128, n_orb=6)
        inp = I.make_inputs(spec)
        st = torch.cuda.current_stream().cuda_stream
        sh, (lo, hi) = shard_system(spec, inp, 0, 1, stream=st)
        assert (lo, hi) == (0, 6)
        sh.propagate(0.0, spec.dt, 2, 2)
        obs = sh.observe(2 * spec.dt, 2 * spec.dt)
        psi_sh, rec_sh = sh.get_orbitals(), sh.reductions(0, 2)
        sh.close()
    finally:
        dist.destroy_process_group()
    whole = System(spec, inp, stream=st)
    whole.propagate(0.0, spec.dt, 2, 2)
    obs_w = whole.observe(2 * spec.dt, 2 * spec.dt)
    assert np.array_equal(psi_sh, whole.get_orbitals())
    assert np.array_equal(rec_sh, whole.reductions(0, 2))
    assert np.array_equal(obs, obs_w)
    whole.close()


def test_exchange_hook_refusals_and_errors():
    from paper_1912_07921_gb300 import _lib
    from paper_1912_07921_gb300.system import System

    spec = ragged_molecule(I.PREC_C128, n_orb=3)
    inp = I.make_inputs(spec)
    s = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    def broken(ptr, n, stream):
        raise RuntimeError("peer lost")

    s.set_exchange(broken)
    with pytest.raises(_lib.TdksError) as ei:
        s.propagate(0.0, spec.dt, 1, 1)
    assert isinstance(ei.value.__cause__, RuntimeError)
    s.set_exchange(None)  # detached: a plain system again
    s.propagate(0.0, spec.dt, 1, 1)
    s.close()
