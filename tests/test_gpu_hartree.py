"""The Hartree potential on the GPU (xc = TDKS_XC_LDA_X_HARTREE) against the oracle's exchange-
plus-Hartree mode: the box's Coulomb cell sum computed by the library's own zero-padded FFTs,
and the periodic cell's plane-wave Poisson solve, inside H applications, records (E_H in the
energy) and propagations with every propagator.  complex128 to 1e-12, complex64 to the FP32
tolerances."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1912_07921_gb300 import inputs as I
from tests._util import bloch_cell, bloch_inputs, ragged_molecule, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _case(kind, prec):
    if kind == "box":
        spec = dataclasses.replace(ragged_molecule(prec, n_orb=5 if prec == I.PREC_C128 else 9),
                                   xc=I.XC_LDA_X_HARTREE)
        return spec, I.make_inputs(spec)
    spec = dataclasses.replace(bloch_cell(prec), xc=I.XC_LDA_X_HARTREE)
    return spec, bloch_inputs(spec)


def _system(spec, inp):
    from paper_1912_07921_gb300.system import System
    return System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("kind", ["box", "cell"])
def test_apply_H_with_hartree_matches_oracle(kind):
    spec, inp = _case(kind, I.PREC_C128)
    s = _system(spec, inp)
    psi = I.random_orbitals(spec, 41)
    packed = s.pack(psi)
    din = torch.from_numpy(packed.view(np.float64)).cuda()
    dout = torch.empty_like(din)
    s.apply_H(0.3, din.data_ptr(), dout.data_ptr())
    torch.cuda.synchronize()
    got = s.unpack(dout.cpu().numpy().view(packed.dtype).reshape(packed.shape))
    s.close()
    o = oracle.System(spec, inp)
    ref = o.apply_H(psi, 0.3, o.vx_of(inp.psi0))
    assert rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("kind,prec", [("box", I.PREC_C128), ("cell", I.PREC_C128), ("box", I.PREC_C64)])
def test_propagation_with_hartree_matches_oracle(kind, prec):
    spec, inp = _case(kind, prec)
    s = _system(spec, inp)
    n, dt, subs = 5, 0.02 if kind == "box" else 0.01, 2
    s.propagate(0.0, dt, n, subs)
    rec = s.reductions(0, n)
    psi = s.get_orbitals()
    s.close()
    psi_o, rec_o = oracle.System(spec, inp).propagate(inp.psi0, 0.0, dt, n, subs)
    tol = 1e-12 if prec == I.PREC_C128 else 1e-5
    assert rel_err(psi, psi_o) < tol
    for c in range(1, 8):
        scale = np.abs(rec_o[:, c]).max()
        if scale > 0:
            assert np.abs(rec[:, c] - rec_o[:, c]).max() <= tol * scale, c
    # the Hartree energy is in the record: without it the energy differs
    no_h = oracle.System(dataclasses.replace(spec, xc=I.XC_LDA_X), inp).observables(inp.psi0, 0.0, 0.5 * dt / subs)
    assert abs(no_h[2] - rec_o[0, 2]) > 1e3 * tol * abs(rec_o[0, 2])


@pytest.mark.parametrize("prop,name", [(1, "cfm4"), (2, "emr"), (3, "aetrs"), (5, "etrs"), (4, "rk4")])
@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_other_propagators_with_hartree_match_oracle(prop, name, prec):
    """v_x + v_H together: pushed into the extrapolation history (CFM4, EMR, AETRS), taken from
    the trial's density (ETRS), or rebuilt at every stage (RK4, complex128 only)."""
    if prop == 4 and prec != I.PREC_C128:
        pytest.skip("RK4 runs on complex128 systems")
    spec, inp = _case("box", prec)
    s = _system(spec, inp)
    s.set_propagator(prop)
    n, dt, subs = 4, 0.02, 2
    s.propagate(0.0, dt, n, subs)
    rec = s.reductions(0, n)
    psi = s.get_orbitals()
    s.close()
    psi_o, rec_o = getattr(oracle.System(spec, inp), "propagate_" + name)(inp.psi0, 0.0, dt, n, subs)
    tol = 1e-12 if prec == I.PREC_C128 else 2e-5
    assert rel_err(psi, psi_o) < tol
    for c in range(1, 8):
        scale = np.abs(rec_o[:, c]).max()
        if scale > 0:
            assert np.abs(rec[:, c] - rec_o[:, c]).max() <= tol * scale, c


def test_hartree_refuses_batches():
    from paper_1912_07921_gb300._lib import TdksError
    from paper_1912_07921_gb300.system import Batch
    spec, inp = _case("box", I.PREC_C128)
    s = _system(spec, inp)
    s.set_clock(0.0, spec.dt, 1)
    with pytest.raises(TdksError) as e:
        Batch([s], stream=torch.cuda.current_stream().cuda_stream)
    assert e.value.code == 1
    s.close()
