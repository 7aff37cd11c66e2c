"""t-SURFF amplitudes on the GPU against the oracle (Sec. "t-SURFF": the time integral of the
Volkov-state current through a surface).

The molecule carries the whole Hamiltonian (wells, Kleinman-Bylander projectors, LDA
exchange, a sin^2 length-gauge pulse) and one orbital is given an outgoing momentum, so
that flux crosses the surface; the surface is a box of grid planes crossing the projector
spheres' neighbourhood.  complex128 matches the oracle to 1e-12 of the largest amplitude,
complex64 (FP32 terms, double-float state) to 1e-5; two calls in a row equal one call over
the same steps; bad surfaces and discontinuous times are refused.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1912_07921_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOX = (6, 25, 5, 22, 6, 19)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _case(prec):
    spec = I.SystemSpec(nx=32, ny=28, nz=26, h=0.3, fd_order=8, prec=prec, n_orb=3, n_atoms=3, projectors=True,
                        gauge=I.GAUGE_LENGTH, amp=0.2, omega=0.7, pol=(0.3, -0.2, 0.9), envelope=I.ENV_SIN2,
                        t_total=2.0, dt=0.02, seed=17)
    inp = I.make_inputs(spec)
    x, y, z = ((np.arange(n) - (n - 1) / 2.0) * spec.h for n in (spec.nx, spec.ny, spec.nz))
    # orbital 0 leaves with momentum 1.8 along z
    inp.psi0[..., 0] *= np.exp(1.8j * z)[None, :, None, None]
    p = np.array([[px, py, pz] for px in (0.0, 0.6) for py in (-0.4, 0.3) for pz in (1.2, 1.8, 2.4)])
    return spec, inp, p


def _gpu(spec, inp, p, calls):
    from paper_1912_07921_gb300.system import System
    s = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    s.set_tsurff(BOX, p)
    t = 0.0
    for n in calls:
        s.propagate(t, spec.dt, n, 1)
        t += n * spec.dt
    b, t_rel = s.tsurff()
    rec = s.reductions(0, sum(calls))
    s.close()
    return b, t_rel, rec


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_tsurff_amplitudes_match_the_oracle(prec):
    spec, inp, p = _case(prec)
    n = 30
    b, t_rel, rec = _gpu(spec, inp, p, [n])
    o = oracle.System(spec, inp)
    _, rec_o, b_o, vol, tr = o.propagate_tsurff(inp.psi0, 0.0, spec.dt, n, 1, BOX, p)
    assert t_rel == pytest.approx(tr, abs=1e-12)
    assert np.max(np.abs(b_o)) > 0.0
    tol = 1e-12 if prec == I.PREC_C128 else 1e-5
    assert np.max(np.abs(b - b_o)) <= tol * np.max(np.abs(b_o)), np.max(np.abs(b - b_o)) / np.max(np.abs(b_o))
    assert np.max(np.abs(rec[:, 4:7] - rec_o[:, 4:7])) <= max(tol, 1e-12) * np.max(np.abs(rec_o[:, 4:7]))


def test_tsurff_accumulation_continues_across_calls():
    spec, inp, p = _case(I.PREC_C128)
    b1, t1, _ = _gpu(spec, inp, p, [12])
    b2, t2, _ = _gpu(spec, inp, p, [5, 7])
    assert t1 == pytest.approx(t2, abs=1e-12)
    assert np.max(np.abs(b1 - b2)) <= 1e-13 * np.max(np.abs(b1))


def test_tsurff_refuses_bad_surfaces_and_time_jumps():
    from paper_1912_07921_gb300._lib import TdksError
    from paper_1912_07921_gb300.system import System
    spec, inp, p = _case(I.PREC_C128)
    s = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    for box in ((3, 25, 5, 22, 6, 19), (6, 28, 5, 22, 6, 19), (10, 10, 5, 22, 6, 19)):
        with pytest.raises(TdksError) as e:
            s.set_tsurff(box, p)
        assert e.value.code == 1
    s.set_tsurff(BOX, p)
    s.propagate(0.0, spec.dt, 2, 1)
    with pytest.raises(TdksError) as e:
        s.propagate(1.0, spec.dt, 2, 1)
    assert e.value.code == 1
    s.close()
    cell = dataclasses.replace(spec, bc=I.BC_BLOCH, gauge=I.GAUGE_VELOCITY, projectors=False, n_atoms=0)
    c = System(cell, I.make_inputs(cell), stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(TdksError) as e:
        c.set_tsurff(BOX, p)
    assert e.value.code == 1
    c.close()
