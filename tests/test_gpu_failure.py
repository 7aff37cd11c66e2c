"""Failure detection of the TMA sweeps, without a GPU fault.

Every wait in the warp-specialised sweep is bounded; a wait that runs out makes the CTA
give up, the producer drains its copies in flight, and the host reports TDKS_ETIMEOUT at
the next synchronising call.  tdks_set_failure_injection(1) injects the failure: the
sweeps' producer warps claim no work item and issue no copy, so every consumer warp's first
wait (for a claim that nothing makes) runs out after its bound (~2 s).  Nothing is read or
written by that sweep and no copy is in flight.  The test checks the status, and that the
same system then propagates exactly like the oracle once the injection is off and the
orbitals are set again.
"""
import time

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


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_wait_that_runs_out_is_reported_and_the_system_recovers(prec):
    from paper_1912_07921_gb300._lib import TdksError
    from paper_1912_07921_gb300.system import System
    spec = ragged_molecule(prec)
    inp = I.make_inputs(spec)
    s = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    s.set_failure_injection(True)
    packed = s.pack(I.random_orbitals(spec, 3))
    view = np.float32 if packed.dtype == np.complex64 else np.float64
    din = torch.from_numpy(packed.view(view)).cuda()
    dout = torch.empty_like(din)
    t0 = time.perf_counter()
    s.apply_H(0.0, din.data_ptr(), dout.data_ptr())  # one sweep, which gives up after ~2 s
    with pytest.raises(TdksError) as e:
        s.reductions(0, 0)
    assert e.value.code == 4 and "gave up" in str(e.value)
    assert time.perf_counter() - t0 < 30.0
    # the error word was cleared: injection off, the state set again, then a normal run
    s.set_failure_injection(False)
    s.set_orbitals(inp.psi0)
    n0 = s.step_count()
    s.propagate(0.0, 0.02, 3, 1)
    rec = s.reductions(n0, 3)
    psi = s.get_orbitals()
    s.close()
    psi_o, rec_o = oracle.System(spec, inp).propagate(inp.psi0, 0.0, 0.02, 3, 1)
    tol = 1e-12 if prec == I.PREC_C128 else 1e-5
    assert rel_err(psi, psi_o) < tol
    assert np.max(np.abs(rec[:, 4:7] - rec_o[:, 4:7])) < tol * np.max(np.abs(rec_o[:, 4:7]))
