"""Continuous batching: jobs admitted by slots and HBM budget while others run give the
same results as each job propagated alone."""
import numpy as np
import pytest

from paper_1912_07921_gb300 import inputs as I
from paper_1912_07921_gb300 import serving
from tests._util import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()


def _trace():
    jobs = serving.serving_trace(8, rate=400.0, seed=9, edge=(17, 29), orbitals=(3, 12), steps=(4, 13),
                                 atoms=(0, 3))
    return jobs


def test_each_job_same_alone_and_in_the_mix():
    from paper_1912_07921_gb300.system import System
    stream = torch.cuda.current_stream().cuda_stream
    jobs = _trace()
    budget = 3 * max(serving.job_bytes(j.spec) for j in jobs)
    srv = serving.Server(hbm_budget=budget, max_slots=3, quantum=3, stream=stream,
                         sync=torch.cuda.synchronize)
    done = srv.run(jobs, keep_orbitals=True)
    rep = srv.report()
    assert rep["jobs"] == len(jobs)
    assert srv.peak_used <= budget
    assert srv.max_concurrent >= 2
    # at least one job joined while another was on the device
    by_id = {j.jid: j for j in done}
    joined = [j for j in done if any(o.jid != j.jid and o.admitted < j.admitted < o.finished for o in done)]
    assert joined
    assert rep["p99_s"] >= rep["p50_s"] > 0
    for j in done:
        s = System(j.spec, I.make_inputs(j.spec), stream=stream)
        s.propagate(0.0, j.spec.dt, j.n_steps, j.spec.substeps)
        rec = s.reductions(0, j.n_steps)
        psi = s.get_orbitals()
        s.close()
        tol = 1e-13 if j.spec.prec == I.PREC_C128 else 1e-6
        assert rel_err(by_id[j.jid].orbitals, psi) < tol
        assert rel_err(by_id[j.jid].records, rec) < tol


def test_served_jobs_match_the_oracle():
    """The complex128 jobs of a served mix against the FP64 oracle (same seeded inputs)."""
    import oracle
    stream = torch.cuda.current_stream().cuda_stream
    jobs = _trace()
    budget = 3 * max(serving.job_bytes(j.spec) for j in jobs)
    srv = serving.Server(hbm_budget=budget, max_slots=3, quantum=3, stream=stream, sync=torch.cuda.synchronize)
    done = srv.run(jobs, keep_orbitals=True)
    c128 = [j for j in done if j.spec.prec == I.PREC_C128]
    assert c128 and all(j.status == "done" for j in done)
    for j in c128:
        inp = I.make_inputs(j.spec)
        psi_o, rec_o = oracle.System(j.spec, inp).propagate(inp.psi0, 0.0, j.spec.dt, j.n_steps, j.spec.substeps)
        assert rel_err(j.orbitals, psi_o) < 1e-12
        assert rel_err(j.records, rec_o) < 1e-12


@pytest.mark.parametrize("prec", [I.PREC_C128, I.PREC_C64])
def test_job_bytes_covers_the_library_allocation(prec):
    """The admission estimate against the device memory a system actually takes (free memory
    before and after creating it, with torch's caching allocator untouched in between)."""
    from paper_1912_07921_gb300.system import System
    spec = I.SystemSpec(nx=64, ny=60, nz=56, h=0.25, fd_order=4, prec=prec, n_orb=24, n_atoms=6, projectors=True,
                        gauge=I.GAUGE_LENGTH, amp=0.005, omega=0.057, dt=0.015, seed=3)
    inp = I.make_inputs(spec)
    # a first system loads the library's kernels (module memory is not the job's)
    w = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    w.propagate(0.0, spec.dt, 1, 1)
    w.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    s = System(spec, inp, stream=torch.cuda.current_stream().cuda_stream)
    s.propagate(0.0, spec.dt, 1, 1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    s.close()
    used = free0 - free1
    est = serving.job_bytes(spec)
    assert used <= est, (used, est)
    assert est <= 1.3 * used + (32 << 20), (used, est)
