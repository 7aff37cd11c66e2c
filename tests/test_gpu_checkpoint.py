"""Checkpoint and resume through the C interface (tdks_save / tdks_load): a system saved
mid-run and loaded continues bit for bit as the original, with the same records, step count
and clock; a damaged file is refused."""
import numpy as np
import pytest

from paper_1912_07921_gb300 import inputs as I
from tests._util import bloch_cell, bloch_inputs, ragged_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _resume_case(spec, inp, tmp_path, prop=0, shapes=None, n1=3, n2=2, subs=2, dt=0.03):
    from paper_1912_07921_gb300.system import System
    a = System(spec, inp, stream=_stream())
    a.set_propagator(prop)
    if shapes is not None:
        for sweep, sh in enumerate(shapes):
            a.set_sweep_shape(sweep, sh)
    a.propagate(0.0, dt, n1, subs)
    path = str(tmp_path / "run.ckpt")
    a.save(path)
    a.propagate(n1 * dt, dt, n2, subs)
    b = System.load(path, stream=_stream())
    assert b.step_count() == n1 and b.spec.n_orb == spec.n_orb
    if shapes is not None:
        assert b.sweep_shapes() == shapes
    b.propagate(n1 * dt, dt, n2, subs)
    try:
        assert b.step_count() == a.step_count() == n1 + n2
        assert np.array_equal(b.get_orbitals(), a.get_orbitals())
        assert np.array_equal(b.reductions(0, n1 + n2), a.reductions(0, n1 + n2))
        assert np.array_equal(b.observe((n1 + n2) * dt, (n1 + n2) * dt), a.observe((n1 + n2) * dt, (n1 + n2) * dt))
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_resume_is_bit_identical_molecule(prec, tmp_path):
    spec = ragged_molecule(prec)
    _resume_case(spec, I.make_inputs(spec), tmp_path)


@pytest.mark.parametrize("prop", [1, 2, 3, 5])
def test_resume_keeps_the_exchange_history(prop, tmp_path):
    """CFM4, EMR and AETRS extrapolate v_x from the last sub-steps: the history is saved.
    (ETRS keeps none across sub-steps; it resumes as well.)"""
    spec = ragged_molecule(I.PREC_C64)
    _resume_case(spec, I.make_inputs(spec), tmp_path, prop=prop, n1=2, n2=3, subs=2)


def test_resume_periodic_cell_with_chosen_shapes(tmp_path):
    from paper_1912_07921_gb300.system import shape_count
    spec = bloch_cell(I.PREC_C64)
    n = shape_count()
    _resume_case(spec, bloch_inputs(spec), tmp_path, shapes=[1 % n, 2 % n, 3 % n, 0], dt=0.01)


def test_damaged_or_partial_checkpoints_are_refused(tmp_path):
    from paper_1912_07921_gb300 import _lib
    from paper_1912_07921_gb300.system import System
    spec = ragged_molecule(I.PREC_C128, n_orb=3)
    a = System(spec, I.make_inputs(spec), stream=_stream())
    a.propagate(0.0, 0.03, 1, 2)
    path = tmp_path / "a.ckpt"
    a.save(str(path))
    data = bytearray(path.read_bytes())
    a.close()
    flipped = tmp_path / "flipped.ckpt"
    data2 = bytearray(data)
    data2[len(data2) // 2] ^= 0x40
    flipped.write_bytes(bytes(data2))
    with pytest.raises(_lib.TdksError, match="checksum"):
        System.load(str(flipped))
    cut = tmp_path / "cut.ckpt"
    cut.write_bytes(bytes(data[: len(data) - 100]))
    with pytest.raises(_lib.TdksError, match="truncated"):
        System.load(str(cut))
    assert not (tmp_path / "a.ckpt.tmp").exists()


def test_save_before_orbitals_then_resume(tmp_path):
    from paper_1912_07921_gb300.system import System
    spec = ragged_molecule(I.PREC_C128, n_orb=3)
    inp = I.make_inputs(spec)
    a = System(spec, None, stream=_stream())
    a.set_local_potential(inp.vloc)
    a.set_projectors(inp.pos, inp.D, spec.r_c, spec.r_cut)
    a.set_field(spec.gauge, spec.pol, spec.amp, spec.omega, spec.envelope, spec.t_total)
    path = str(tmp_path / "empty.ckpt")
    a.save(path)
    b = System.load(path, stream=_stream())
    for s in (a, b):
        s.set_orbitals(inp.psi0)
        s.propagate(0.0, 0.03, 2, 2)
    assert np.array_equal(a.get_orbitals(), b.get_orbitals())
    a.close()
    b.close()
