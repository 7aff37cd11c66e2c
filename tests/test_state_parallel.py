"""State-parallel propagation on CPU ranks: two gloo processes stand in for two GPUs.

The method couples the orbitals only through the density in v_x[n] (Sec. "New propagators
for real-time TDDFT": H[n(t), t]); the paper's multi-GPU runs distribute the states only
(Sec. "GPUs").  Each rank takes its `state_slice` of the orbitals; the exchange hook
(`sharding.allreduce_exchange`, called through the same C function-pointer type the library
calls) sums the ranks' densities and band sums.  Checked against the oracle of the whole
system: the summed density, the band energy, and one Taylor sub-step of each slice with
the exchanged v_x, which must equal the oracle's sub-step of all orbitals restricted to the
slice.
"""
import ctypes
import dataclasses
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1912_07921_gb300.sharding import state_slice  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_orb,world,block", [(64, 2, 8), (64, 8, 8), (9, 2, 4), (5, 4, 1), (3, 4, 1),
                                               (13, 3, 4), (0, 2, 4), (7, 1, 8)])
def test_state_slices_partition_the_orbitals(n_orb, world, block):
    got = [state_slice(n_orb, r, world, block) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == n_orb
    for (a0, a1), (b0, b1) in zip(got, got[1:]):
        assert a1 == b0 and a0 <= a1
    sizes = [hi - lo for lo, hi in got]
    # whole blocks (the slice ending at n_orb may hold a partial one), block counts within one
    for lo, hi in got:
        assert lo % block == 0 and (hi % block == 0 or hi == n_orb)
    blocks = [-(-sz // block) for sz in sizes]
    assert max(blocks) - min(blocks) <= 1 and sum(sizes) == n_orb


def test_state_slice_rejects_bad_requests():
    for args in [(4, 2, 2, 1), (4, -1, 2, 1), (4, 0, 0, 1), (4, 0, 2, 0), (-1, 0, 1, 1)]:
        with pytest.raises(ValueError):
            state_slice(*args)


def _spec():
    from paper_1912_07921_gb300 import inputs as I
    return I.SystemSpec(nx=11, ny=10, nz=9, h=0.35, fd_order=4, prec=I.PREC_C128, n_orb=5, n_atoms=2,
                        projectors=True, gauge=I.GAUGE_LENGTH, amp=0.05, omega=0.3, envelope=I.ENV_NONE,
                        dt=0.02, seed=44)


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1912_07921_gb300 import _lib, inputs as I
    from paper_1912_07921_gb300.sharding import allreduce_exchange

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = _spec()
        inp = I.make_inputs(spec)
        lo, hi = state_slice(spec.n_orb, rank, world, 2)
        mine = oracle.System(dataclasses.replace(spec, n_orb=hi - lo), inp)
        psi = np.ascontiguousarray(inp.psi0[..., lo:hi])
        # the hook as the library sees it: a C function pointer over host buffers
        fn = allreduce_exchange(device="cpu")
        cb = _lib.EXCHANGE_FN(lambda ptr, n, stream, ctx: (fn(ptr, n, stream), 0)[1])
        call = ctypes.cast(cb, _lib.EXCHANGE_FN)

        n = np.ascontiguousarray(mine.density(psi).ravel())
        assert call(n.ctypes.data, n.size, None, None) == 0
        ex, vx = mine.lda_x(n)
        t, dt = 0.3, spec.dt
        # this rank's band sum sum_i f <phi_i | H[v_x of all orbitals] | phi_i> h^3
        hpsi = mine.apply_H(psi, t, vx)
        band = np.array([spec.occ * np.vdot(psi, hpsi).real * spec.h ** 3, 0.0, 0.0, 0.0])
        assert call(band.ctypes.data, 4, None, None) == 0
        # one Taylor-4 sub-step of the slice with the exchanged v_x, H taken at the midpoint
        acc, term = psi.copy(), psi.copy()
        for k in range(1, 5):
            term = (-1j * dt / k) * mine.apply_H(term, t + 0.5 * dt, vx)
            acc = acc + term
        out[rank] = dict(lo=lo, hi=hi, n=n.copy(), band=band[0], psi=acc, ex=ex)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_whole_system(world):
    """Two ranks (slices of 4 and 1 orbitals), or three (2, 2 and 1: an uneven last slice)."""
    import oracle
    from paper_1912_07921_gb300 import inputs as I

    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = {r: dict(v) for r, v in out.items()}
    spec = _spec()
    inp = I.make_inputs(spec)
    full = oracle.System(spec, inp)
    n_full = full.density(inp.psi0).ravel()
    ex_full, vx_full = full.lda_x(n_full)
    hpsi = full.apply_H(inp.psi0, 0.3, vx_full)
    band_full = spec.occ * np.vdot(inp.psi0, hpsi).real * spec.h ** 3
    stepped = full.taylor_substep(inp.psi0, 0.3, spec.dt)
    slices = [(got[r]["lo"], got[r]["hi"]) for r in range(world)]
    assert slices == ([(0, 4), (4, 5)] if world == 2 else [(0, 2), (2, 4), (4, 5)])
    for r in range(world):
        g = got[r]
        # every rank holds the whole system's density and band energy after the exchange
        assert np.max(np.abs(g["n"] - n_full)) <= 1e-13 * np.max(n_full)
        assert g["ex"] == pytest.approx(ex_full, rel=1e-12)
        assert g["band"] == pytest.approx(band_full, rel=1e-12)
        ref = stepped[..., g["lo"]:g["hi"]]
        assert np.max(np.abs(g["psi"] - ref)) <= 1e-12 * np.max(np.abs(ref))


def _leaving_rank_main(rank, world, port, out):
    """Rank 1 leaves between two exchanges (no collective in flight); rank 0 keeps going."""
    import datetime
    import time
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1912_07921_gb300 import _lib, inputs as I
    from paper_1912_07921_gb300.sharding import allreduce_exchange

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    spec = _spec()
    inp = I.make_inputs(spec)
    lo, hi = state_slice(spec.n_orb, rank, world, 2)
    mine = oracle.System(dataclasses.replace(spec, n_orb=hi - lo), inp)
    psi = np.ascontiguousarray(inp.psi0[..., lo:hi])
    fn = allreduce_exchange(device="cpu")

    def hook(ptr, n, stream, ctx):  # as System.set_exchange wraps it: an exception is a status
        try:
            fn(ptr, n, stream)
            return 0
        except Exception:
            return 1

    cb = _lib.EXCHANGE_FN(hook)
    call = ctypes.cast(cb, _lib.EXCHANGE_FN)
    log = []
    for step in range(3):
        if rank == 1 and step == 1:
            os._exit(0)  # leaves between steps
        n = np.ascontiguousarray(mine.density(psi).ravel())
        t0 = time.time()
        st = call(n.ctypes.data, n.size, None, None)
        log.append((st, time.time() - t0))
    out[rank] = log
    try:
        dist.destroy_process_group()
    except Exception:
        pass


def test_rank_that_leaves_makes_the_survivor_fail_not_hang():
    """The exchange of the survivor's next step fails (status 1, which the library turns into
    TDKS_EDEVICE) within the process group's timeout, and so does every later one."""
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_leaving_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert set(got) == {0}
    statuses = [st for st, _ in got[0]]
    assert statuses == [0, 1, 1], got[0]
    assert all(sec < 30.0 for _, sec in got[0])
