"""Batched propagation (one persistent sweep launch per Taylor term over many uneven
systems, replayed as a CUDA graph) gives each system the same result as propagating it
alone, and matches the oracle."""
import numpy as np
import pytest

import oracle
from paper_1912_07921_gb300 import inputs as I
from tests._util import rel_err, small_uneven_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _run(specs, inps, n_steps, batched, use_graph=True):
    from paper_1912_07921_gb300.system import Batch, System
    stream = torch.cuda.current_stream().cuda_stream
    systems = [System(s, i, stream=stream) for s, i in zip(specs, inps)]
    if batched:
        for s in systems:
            s.set_clock(0.0, s.spec.dt, s.spec.substeps)
        b = Batch(systems, stream=stream)
        b.propagate(n_steps, use_graph=use_graph)
        launches = b.launch_count()
    else:
        for s in systems:
            s.propagate(0.0, s.spec.dt, n_steps, s.spec.substeps)
        launches = None
    torch.cuda.synchronize()
    out = [(s.get_orbitals(), s.reductions(0, n_steps)) for s in systems]
    if batched:
        b.close()
    for s in systems:
        s.close()
    return out, launches


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_batch_equals_alone(prec):
    specs = small_uneven_batch(prec)
    inps = [I.make_inputs(s) for s in specs]
    alone, _ = _run(specs, inps, 3, batched=False)
    mixed, launches = _run(specs, inps, 3, batched=True)
    assert launches == (1 + 4 * (3 + 1) + 2) * 3  # LDA, 4 x (gather 1+2, non-local, sweep), record, clock
    tol = 1e-13 if prec == I.PREC_C128 else 1e-6
    for (pa, ra), (pb, rb) in zip(alone, mixed):
        assert rel_err(pb, pa) < tol
        assert rel_err(rb, ra) < tol


def test_batch_graph_and_direct_launches_agree():
    specs = small_uneven_batch(I.PREC_C64, n=3, seed=11)
    inps = [I.make_inputs(s) for s in specs]
    g, _ = _run(specs, inps, 2, batched=True, use_graph=True)
    d, _ = _run(specs, inps, 2, batched=True, use_graph=False)
    for (pa, ra), (pb, rb) in zip(g, d):
        assert np.array_equal(pa, pb) and np.array_equal(ra, rb)


def test_batch_matches_oracle_c128():
    specs = small_uneven_batch(I.PREC_C128, n=3, seed=5)
    inps = [I.make_inputs(s) for s in specs]
    mixed, _ = _run(specs, inps, 3, batched=True)
    for spec, inp, (psi, rec) in zip(specs, inps, mixed):
        psi_o, rec_o = oracle.System(spec, inp).propagate(inp.psi0, 0.0, spec.dt, 3, 1)
        assert rel_err(psi, psi_o) < 1e-12
        np.testing.assert_allclose(rec, rec_o, rtol=1e-12, atol=1e-12 * np.abs(rec_o).max())


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_batch_autotune_and_shapes_keep_results(prec):
    """The batched autotuner times every tile shape on each Taylor term without touching
    any state; a batch with tuned (or mixed) shapes gives each system its alone result."""
    from paper_1912_07921_gb300.system import Batch, System, shape_count
    specs = small_uneven_batch(prec, n=4, seed=13)
    inps = [I.make_inputs(s) for s in specs]
    alone, _ = _run(specs, inps, 2, batched=False)
    stream = torch.cuda.current_stream().cuda_stream
    for mode in ("tuned", "mixed"):
        systems = [System(s, i, stream=stream) for s, i in zip(specs, inps)]
        for s in systems:
            s.set_clock(0.0, s.spec.dt, s.spec.substeps)
        b = Batch(systems, stream=stream)
        before = [s.get_orbitals() for s in systems]
        if mode == "tuned":
            ms = b.autotune(reps=2)
            assert ms.shape == (shape_count(), 4) and np.all(ms > 0)
            assert b.shapes() == [int(i) for i in np.argmin(ms, axis=0)]
            for s, p0 in zip(systems, before):
                assert np.array_equal(s.get_orbitals(), p0)
        else:
            for k in range(4):
                b.set_shape(k, (k + 2) % shape_count())
        b.propagate(2)
        torch.cuda.synchronize()
        tol = 1e-13 if prec == I.PREC_C128 else 1e-6
        for s, (pa, ra) in zip(systems, alone):
            assert rel_err(s.get_orbitals(), pa) < tol
            assert rel_err(s.reductions(0, 2), ra) < tol
        b.close()
        for s in systems:
            s.close()
