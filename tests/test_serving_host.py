"""Host logic of the continuous-batching server on CPU: the library's System and Batch are
replaced by fakes that count steps, so admission by HBM budget and slot count, grouping by
(precision, FD order, sub-steps), batch rebuilds on join and leave, the step quantum and the
report are checked without a GPU."""
import dataclasses
import math

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

    def watched_tick(now=0.0):
        used.append(srv.used)
        assert srv.used <= budget and len(srv.active) <= slots
        tick(now)

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


def test_a_job_larger_than_the_budget_is_rejected_alone():
    jobs = _jobs(6, seed=21)
    sizes = sorted(serving.job_bytes(j.spec) for j in jobs)
    budget = sizes[-2]  # the largest job alone does not fit
    big = max(jobs, key=lambda j: serving.job_bytes(j.spec))
    srv, done, _ = _serve(jobs, budget=budget)
    status = {j.jid: j.status for j in done}
    assert status.pop(big.jid) == "rejected" and set(status.values()) == {"done"}
    assert "more than the whole budget" in big.error
    assert srv.report()["status"] == {"done": len(jobs) - 1, "rejected": 1}


class RefusingSystem(FakeSystem):
    """The library refusing one job at creation (an allocation that does not fit)."""
    refuse = set()

    def __init__(self, spec, inputs, stream=None):
        if spec.seed in RefusingSystem.refuse:
            from paper_1912_07921_gb300._lib import TdksError
            raise TdksError(2, "cudaMalloc: out of memory")
        super().__init__(spec, inputs, stream)


def test_an_allocation_refusal_fails_that_job_alone(monkeypatch):
    jobs = _jobs(8, seed=23)
    RefusingSystem.refuse = {jobs[3].spec.seed}
    monkeypatch.setattr(serving, "System", RefusingSystem)
    srv, done, used = _serve(jobs, budget=10 ** 12)
    status = {j.jid: j.status for j in done}
    assert status[3] == "failed" and "out of memory" in jobs[3].error
    assert all(v == "done" for k, v in status.items() if k != 3)
    assert srv.used == 0 and FakeSystem.live == 0  # nothing was charged or left for the refused job


def test_a_non_finite_input_is_found_before_any_allocation():
    jobs = _jobs(5, seed=25)
    inp = I.Inputs(vloc=np.zeros(4), psi0=np.array([1.0, np.nan]), pos=np.zeros((0, 3)), D=np.zeros((0, 4)),
                   kpts=np.zeros((1, 3)), kw=np.ones(1))
    jobs[2].inputs = inp
    srv = serving.Server(10 ** 12, quantum=7, make_inputs=lambda spec: None)
    done = srv.run(jobs, time_scale=1e-6)
    status = {j.jid: j.status for j in done}
    assert status[2] == "invalid" and jobs[2].system is None
    assert sum(v == "done" for v in status.values()) == 4
    assert FakeSystem.live == 0


def test_cancelled_jobs_leave_the_queue_or_release_their_memory():
    jobs = _jobs(6, seed=27)
    for j in jobs:
        j.arrival = 0.0
    jobs[5].n_steps = 10 ** 6  # long enough to be cancelled while active
    srv = serving.Server(10 ** 12, max_slots=5, quantum=3, make_inputs=lambda spec: None)
    tick = srv._tick
    calls = []

    def ticking(now=0.0):
        calls.append(1)
        if len(calls) == 2:
            srv.cancel(5)   # active by now
            srv.cancel(4)   # maybe active, maybe finished
        tick(now)

    srv._tick = ticking
    srv.cancel(0)  # cancelled while queued, never admitted
    done = srv.run(jobs, time_scale=1e-6)
    status = {j.jid: j.status for j in done}
    assert status[0] == "cancelled" and jobs[0].system is None and math.isnan(jobs[0].admitted)
    assert status[5] == "cancelled" and jobs[5].steps_done < jobs[5].n_steps
    assert status[4] in ("cancelled", "done")
    assert srv.used == 0 and FakeSystem.live == 0


class FailingBatch(FakeBatch):
    """A batch whose propagation reports an error when it holds a poisoned job."""
    poison = set()

    def propagate(self, q, use_graph=True):
        if any(s.spec.seed in FailingBatch.poison for s in self.systems):
            from paper_1912_07921_gb300._lib import TdksError
            raise TdksError(4, "a sweep kernel gave up waiting for its TMA copies")
        super().propagate(q, use_graph)


def test_a_batch_error_fails_its_group_and_the_others_go_on(monkeypatch):
    jobs = _jobs(10, seed=29)
    c64 = [j for j in jobs if j.spec.prec == I.PREC_C64]
    c128 = [j for j in jobs if j.spec.prec == I.PREC_C128]
    assert c64 and c128
    for j in jobs:
        j.arrival = 0.0
    FailingBatch.poison = {c64[0].spec.seed}
    monkeypatch.setattr(serving, "Batch", FailingBatch)
    srv, done, _ = _serve(jobs, budget=10 ** 12)
    status = {j.jid: j.status for j in done}
    assert status[c64[0].jid] == "failed"
    assert all(status[j.jid] == "done" for j in c128)
    assert srv.used == 0 and FakeSystem.live == 0


def test_job_bytes_grows_with_the_job():
    base = I.SystemSpec(nx=48, ny=48, nz=48, h=0.25, n_orb=16, prec=I.PREC_C64)
    b = serving.job_bytes(base)
    assert serving.job_bytes(dataclasses.replace(base, prec=I.PREC_C128)) > b
    assert serving.job_bytes(dataclasses.replace(base, n_orb=32)) > b
    assert serving.job_bytes(dataclasses.replace(base, nx=96)) > b
    assert serving.job_bytes(dataclasses.replace(base, n_atoms=4, projectors=True)) > b
    # at least the state, the three Taylor terms and the host-layout staging buffer
    assert b >= base.n_points * 16 * (16 + 3 * 8) + base.n_points * 16 * 16
