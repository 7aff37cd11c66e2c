"""complex64 H psi over 1000 configured steps against the FP64 oracle.

The precision plan runs H psi and the Taylor terms in complex64 while the state, the
density and every reduction stay in FP64 (or double-float); its bar is the dipole (the
current, in a periodic cell) within 1e-4 of its peak after 1000 steps.  These tests run
the physics of the two large workloads at a grid size the oracle finishes in minutes:
- the medium molecule's: order-8 FD, 16 atoms with projectors, LDA exchange, the sin^2
  pulse, dt = 0.05 as 4 sub-steps, on 32^3 with 8 orbitals;
- the periodic cell's: order-4 FD in a 10.2-bohr cell with 8 diamond atoms, Bloch states
  of 2 k-points x 8 bands, the velocity gauge, dt = 0.04 as 2 sub-steps, on 32^3.
The oracle's records of the same runs are stored under tests/golden/ (written by
tests/golden/make_fp32_horizon.py, which calls only the oracle).  The error of the
observable o(t) is max_t |o32(t) - o64(t)| / max_t |o64(t)|; the induced part
o(t) - o(0), norm and energy are checked too.
"""
import os

import numpy as np
import pytest

from paper_1912_07921_gb300 import inputs as I
from tests._util import HORIZON_CASES, read_horizon_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _run(spec):
    from paper_1912_07921_gb300.system import System
    inp = I.make_inputs(spec)
    s = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    assert s.auto_substeps(spec.dt) == spec.substeps
    s.propagate(0.0, spec.dt, spec.n_steps, spec.substeps)
    rec = s.reductions(0, spec.n_steps)
    s.close()
    return rec


def _err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("name", sorted(HORIZON_CASES))
def test_complex64_observable_after_1000_steps(name):
    ref = read_horizon_golden(os.path.join(GOLDEN, f"fp32_horizon_{name}.txt"))
    spec = HORIZON_CASES[name](I.PREC_C64)
    assert ref.shape == (spec.n_steps, 8)
    rec = _run(spec)
    np.testing.assert_allclose(rec[:, 0], ref[:, 0], rtol=0, atol=1e-12)  # the same times
    o, o_ref = rec[:, 4:7], ref[:, 4:7]
    assert _err(o, o_ref) <= 1e-4, _err(o, o_ref)
    ind, ind_ref = o - o[0], o_ref - o_ref[0]
    assert _err(ind, ind_ref) <= 1e-3, _err(ind, ind_ref)
    assert np.max(np.abs(rec[:, 1] - ref[:, 1])) <= 1e-5 * ref[0, 1]
    assert np.max(np.abs(rec[:, 2] - ref[:, 2])) <= 1e-4 * np.max(np.abs(ref[:, 2]))


@pytest.mark.parametrize("name", sorted(HORIZON_CASES))
def test_complex128_stays_on_the_oracle_over_1000_steps(name):
    """The FP64 path over the same 1000 steps: the records agree with the oracle's to the
    rounding that 1000 steps of two different summation orders accumulate."""
    ref = read_horizon_golden(os.path.join(GOLDEN, f"fp32_horizon_{name}.txt"))
    rec = _run(HORIZON_CASES[name](I.PREC_C128))
    for c in range(1, 8):
        scale = np.max(np.abs(ref[:, c]))
        if scale > 0:
            assert np.max(np.abs(rec[:, c] - ref[:, c])) <= 1e-10 * scale, c
