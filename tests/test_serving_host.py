"""Host logic of the continuous-batching server on CPU: the library's System and Batch are
replaced by fakes that count steps, so admission by HBM budget and slot count, grouping by
(precision, FD order, sub-steps), batch rebuilds on join and leave, the step quantum and the
report are checked without a GPU."""
import dataclasses

import numpy as np
import pytest

from paper_1912_07921_gb300 import inputs as I
from paper_1912_07921_gb300 import serving


class FakeSystem:
    live = 0

    def __init__(self, spec, inputs, stream=None):
        self.spec, self.steps, self.closed = spec, 0, False
        FakeSystem.live += 1

    def set_clock(self, t, dt, substeps):
        self.clock = (t, dt, substeps)

    def reductions(self, step_from, n):
        assert step_from == 0 and n == self.steps
        return np.zeros((n, 8))

    def get_orbitals(self):
        return np.zeros((1,))

    def close(self):
        assert not self.closed
        self.closed = True
        FakeSystem.live -= 1


class FakeBatch:
    built = []

    def __init__(self, systems, stream=None):
        keys = {(s.spec.prec, s.spec.fd_order, s.spec.substeps) for s in systems}
        assert len(keys) == 1, "a batch mixes precisions, orders or sub-step counts"
        assert not any(s.closed for s in systems)
        self.systems, self.closed = list(systems), False
        FakeBatch.built.append(self)

    def propagate(self, q, use_graph=True):
        assert not self.closed and q >= 1
        for s in self.systems:
            s.steps += q

    def close(self):
        self.closed = True


@pytest.fixture(autouse=True)
def fakes(monkeypatch):
    monkeypatch.setattr(serving, "System", FakeSystem)
    monkeypatch.setattr(serving, "Batch", FakeBatch)
    FakeSystem.live = 0
    FakeBatch.built = []
    yield


def _jobs(n=24, seed=5):
    return serving.serving_trace(n, rate=200.0, seed=seed, edge=(8, 20), orbitals=(1, 12), steps=(3, 40),
                                 atoms=(0, 3))


def _serve(jobs, budget, slots=64, quantum=7):
    srv = serving.Server(budget, max_slots=slots, quantum=quantum, make_inputs=lambda spec: None)
    used = []
    tick = srv._tick

    def watched_tick():
        used.append(srv.used)
        assert srv.used <= budget and len(srv.active) <= slots
        tick()

    srv._tick = watched_tick
    done = srv.run(jobs, time_scale=1e-6)  # arrivals replayed a million times faster
    return srv, done, used


def test_every_job_finishes_with_exactly_its_steps():
    jobs = _jobs()
    srv, done, _ = _serve(jobs, budget=10 ** 12)
    assert sorted(j.jid for j in done) == list(range(len(jobs)))
    for j in done:
        assert j.steps_done == j.n_steps and j.records.shape == (j.n_steps, 8)
        assert j.finished >= j.admitted >= j.arrival
    assert FakeSystem.live == 0 and all(b.closed for b in FakeBatch.built)
    rep = srv.report()
    assert rep["jobs"] == len(jobs) and rep["updates"] == sum(j.updates for j in jobs)
    assert rep["p50_s"] <= rep["p99_s"]


def test_budget_and_slots_bound_the_resident_jobs():
    jobs = _jobs(seed=9)
    sizes = [serving.job_bytes(j.spec) for j in jobs]
    budget = 2 * max(sizes) + min(sizes)
    srv, done, used = _serve(jobs, budget=budget, slots=3)
    assert len(done) == len(jobs)
    assert max(used) <= budget and srv.peak_used <= budget and srv.max_concurrent <= 3


def test_batches_are_grouped_and_rebuilt_when_membership_changes():
    jobs = _jobs(seed=13)
    _serve(jobs, budget=10 ** 12, quantum=5)
    precisions = {j.spec.prec for j in jobs}
    assert len(precisions) == 2  # the trace mixes complex64 and complex128
    # each batch holds one group; a new batch appears whenever a job joins or leaves
    assert len(FakeBatch.built) > len(precisions)


def test_quantum_never_overshoots_a_job():
    spec = dataclasses.replace(_jobs(1)[0].spec, prec=I.PREC_C64)
    jobs = [serving.Job(jid=i, spec=spec, n_steps=n, arrival=0.0) for i, n in enumerate((5, 12, 3))]
    _, done, _ = _serve(jobs, budget=10 ** 12, quantum=50)
    assert {j.jid: j.steps_done for j in done} == {0: 5, 1: 12, 2: 3}


def test_a_job_larger_than_the_budget_is_refused():
    jobs = _jobs(2)
    with pytest.raises(ValueError, match="more than the whole budget"):
        _serve(jobs, budget=16)


def test_job_bytes_grows_with_the_job():
    base = I.SystemSpec(nx=20, ny=20, nz=20, h=0.25, n_orb=8, prec=I.PREC_C64)
    b = serving.job_bytes(base)
    assert serving.job_bytes(dataclasses.replace(base, prec=I.PREC_C128)) > b
    assert serving.job_bytes(dataclasses.replace(base, n_orb=16)) > b
    assert serving.job_bytes(dataclasses.replace(base, nx=40)) > b
    # at least the state, the three Taylor terms and the host-layout staging buffer
    assert b >= base.n_points * 8 * (16 + 3 * 8) + base.n_points * 8 * 16
