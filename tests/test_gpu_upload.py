"""Orbital uploads through the C interface while a propagation is in flight.

With two upload buffers, each upload packs into the spare state buffer on a stream of its own
and the system then switches buffers: work enqueued before the upload must still see the
old state, work enqueued after it the new one, and the spare may only be overwritten once the
work that used it is done.  Each case compares with systems that never overlap anything (one
upload each, propagated alone): complex128 bit for bit."""
import numpy as np
import pytest

from paper_1912_07921_gb300 import inputs as I
from tests._util import ragged_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _orbitals(spec, seed):
    psi = I.random_orbitals(spec, seed)
    norm = np.sqrt(np.sum(np.abs(psi) ** 2, axis=(1, 2, 3), keepdims=True) * spec.h ** 3)
    return psi / norm


def _alone(spec, inp, psi, t0, n):
    from paper_1912_07921_gb300.system import System
    s = System(spec, inp, stream=_stream(), orbitals=psi)
    s.propagate(t0, spec.dt, n, 2)
    out = s.get_orbitals(), s.reductions(0, n)
    s.close()
    return out


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_uploads_overlapping_propagations_keep_stream_order(prec):
    from paper_1912_07921_gb300.system import System
    spec = ragged_molecule(prec, n_orb=6)
    inp = I.make_inputs(spec)
    states = [inp.psi0, _orbitals(spec, 3), _orbitals(spec, 4), _orbitals(spec, 5)]
    n = 2
    want = [_alone(spec, inp, psi, 0.0, n) for psi in states]
    s = System(spec, inp, stream=_stream(), orbitals=states[0])
    s.set_upload_buffers(2)
    try:
        for i in range(len(states)):
            s.propagate(0.0, spec.dt, n, 2)  # enqueued; the next upload overlaps it
            if i + 1 < len(states):
                s.set_orbitals(states[i + 1])
            rec = s.reductions(s.step_count() - n, n)
            np.testing.assert_array_equal(rec, want[i][1])  # the in-flight run saw the old state
        np.testing.assert_array_equal(s.get_orbitals(), want[-1][0])
        s.set_orbitals(states[1])  # and an upload with nothing in flight
        got = s.get_orbitals()
        tol = 0.0 if prec == I.PREC_C128 else 1e-13
        assert np.max(np.abs(got - states[1])) <= tol * np.max(np.abs(states[1]))
        s.set_upload_buffers(1)  # back to one buffer: the current state stays
        assert np.array_equal(s.get_orbitals(), got)
        s.propagate(0.0, spec.dt, n, 2)
        np.testing.assert_array_equal(s.get_orbitals(), want[1][0])
    finally:
        s.close()


def test_batched_system_uploads_in_place():
    """A system in a batch has one upload buffer: an upload packs in place, and the batch
    propagates the uploaded state.  A system with two buffers is refused by a batch."""
    from paper_1912_07921_gb300._lib import TdksError
    from paper_1912_07921_gb300.system import Batch, System
    spec = ragged_molecule(I.PREC_C64, n_orb=4)
    inp = I.make_inputs(spec)
    psi1 = _orbitals(spec, 7)
    a = System(spec, inp, stream=_stream())
    a.set_clock(0.0, spec.dt, 1)
    a.set_upload_buffers(2)
    with pytest.raises(TdksError):
        Batch([a], stream=_stream())
    a.set_upload_buffers(1)
    b = Batch([a], stream=_stream())
    try:
        a.set_orbitals(psi1)
        b.propagate(2)
        got = a.get_orbitals()
    finally:
        b.close()
        a.close()
    ref = System(spec, inp, stream=_stream(), orbitals=psi1)
    ref.set_clock(0.0, spec.dt, 1)
    rb = Batch([ref], stream=_stream())
    try:
        rb.propagate(2)
        want = ref.get_orbitals()
    finally:
        rb.close()
        ref.close()
    np.testing.assert_array_equal(got, want)
