"""Continuous-batching server for propagation jobs (host-side scheduling only).

Jobs (a seeded system, a number of steps, an arrival time) are admitted while device
slots and an HBM budget allow; each admitted job's orbitals, potentials and projector
tables stay resident on the device until it finishes.  Every scheduler tick advances all
active jobs together: jobs sharing precision, FD order and sub-step count form one batch,
advanced with one persistent sweep launch per Taylor term (``Batch``, replayed as a CUDA
graph), and the batch is rebuilt whenever a job joins or leaves.  A job that arrives
while others are on the GPU joins at the next tick; a finished job releases its memory
and slot at once.  Latency is measured from arrival to the moment the job's results
(its observable records and final orbitals' norm) are on the host.

A bad request fails alone.  Every job ends with a status: "done"; "rejected" (its footprint
exceeds the whole HBM budget); "invalid" (a non-finite number in its inputs, found on the
host before any device allocation); "failed" (the library refused it, e.g. an allocation
that did not fit, or its batch reported an error; the job's memory is released and the
others go on); "cancelled" (``Server.cancel``, while queued or active).  Percentiles are
taken over the jobs that finished.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

from . import inputs as I
from .system import Batch, System


@dataclasses.dataclass
class Job:
    jid: int
    spec: I.SystemSpec
    n_steps: int
    arrival: float
    # filled by the server
    admitted: float = math.nan
    finished: float = math.nan
    steps_done: int = 0
    records: Optional[np.ndarray] = None
    orbitals: Optional[np.ndarray] = None
    inputs: Optional[I.Inputs] = None  # the request's payload (built at admission when absent)
    system: Optional[System] = None
    nbytes: int = 0
    status: str = "queued"  # queued, active, done, rejected, invalid, failed, cancelled
    error: str = ""

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def updates(self) -> int:
        return self.spec.n_points * self.spec.n_orb * self.n_steps


_PAGE = 2 << 20  # device allocations are made in 2 MiB pages


def _pages(nbytes: float) -> int:
    return int(-(-int(math.ceil(nbytes)) // _PAGE)) * _PAGE if nbytes > 0 else 0


def job_bytes(spec: I.SystemSpec) -> int:
    """Device memory a job holds while resident: the library's buffers for it, each rounded
    up to the 2 MiB pages it occupies (state and Taylor terms, potentials and per-point
    records, density partials, observable partials, record ring, upload staging, projector
    tables).  A GPU test checks it against the device's free memory around a system."""
    bs = 8 if spec.prec == I.PREC_C64 else 4
    nb = -(-spec.n_orb // bs)
    n_kb = nb * spec.n_k
    N = spec.n_points
    packed = n_kb * N * 64  # one packed array: 64 bytes per (point, batch)
    total = _pages(packed) * (5 if spec.prec == I.PREC_C64 else 4)  # state (hi, lo) and 3 terms
    total += _pages(N * 8) + _pages(N * 16) + _pages(n_kb * N * 8)  # V_loc, records, density
    # observable partials: the most records a first sweep can write over the tile shapes
    items_gen = -(-spec.nx // 8) * -(-spec.ny // 4) * n_kb * spec.nz
    shapes = ((16, 8, 8), (16, 12, 6), (16, 12, 12), (16, 8, 16), (14, 8, 7), (16, 12, 12))
    items_ws = max(-(-spec.nx // tx) * -(-spec.ny // ty) * n_kb * spec.nz * w for tx, ty, w in shapes)
    total += _pages(max(items_gen, items_ws) * 32)
    total += _pages(65536 * 8 * 8) + 6 * _PAGE  # record ring; error word, LDA/finalise partials, k-points
    total += _pages(spec.n_k * N * spec.n_orb * 16)  # upload staging
    if spec.projectors and spec.n_atoms > 0:
        pts = 1.15 * 4.0 / 3.0 * math.pi * (spec.r_cut / spec.h + 1.0) ** 3  # points in a sphere (bound)
        ent = spec.n_atoms * pts * (8 if spec.bc == I.BC_BLOCH else 1)     # periodic: the images
        total += _pages(ent * 120) + _pages(ent * 16) + _pages(ent * 8) + _pages(ent * 4) + _pages(ent * 8)
        total += _pages(n_kb * (ent + 1) * 64)  # non-local term per sphere point
        total += _pages(n_kb * spec.n_atoms * 4 * 64) + _pages(n_kb * spec.n_atoms * 64 * 4 * 4 * 32)
        total += 3 * _PAGE  # atom ranges, strengths, sphere-point ranges
    return total


def serving_trace(n_jobs: int, rate: float, seed: int, edge=(32, 128), orbitals=(4, 128),
                  steps=(200, 5000), atoms=(0, 32)) -> List[Job]:
    """Poisson arrivals of propagation requests (grid edge, orbitals, steps, atoms drawn
    uniformly; half complex64, half complex128; h = 0.25, 4th-order FD, dt = 0.015)."""
    rng = I.SplitMix64(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += rng.exponential(rate)
        e = rng.randint(*edge)
        n_orb = rng.randint(*orbitals)
        n_steps = rng.randint(*steps)
        n_atoms = rng.randint(*atoms)
        prec = I.PREC_C64 if rng.uniform() < 0.5 else I.PREC_C128
        spec = I.SystemSpec(nx=e, ny=e, nz=e, h=0.25, fd_order=4, prec=prec, n_orb=n_orb, n_atoms=n_atoms,
                            projectors=n_atoms > 0, gauge=I.GAUGE_LENGTH, amp=0.005, omega=0.057, dt=0.015,
                            n_steps=n_steps, substeps=1, seed=(seed << 24) + j)
        jobs.append(Job(jid=j, spec=spec, n_steps=n_steps, arrival=t))
    return jobs


class Server:
    """Admission by HBM budget and slot count; continuous batching of the active jobs."""

    def __init__(self, hbm_budget: int, max_slots: int = 64, quantum: int = 50, stream: Optional[int] = None,
                 use_graph: bool = True, sync: Optional[Callable[[], None]] = None,
                 make_inputs: Callable[[I.SystemSpec], I.Inputs] = I.make_inputs):
        self.budget = hbm_budget
        self.max_slots = max_slots
        self.quantum = quantum
        self.stream = stream
        self.use_graph = use_graph
        self.sync = sync or (lambda: None)
        self.make_inputs = make_inputs
        self.used = 0
        self.peak_used = 0
        self.active: List[Job] = []
        self.done: List[Job] = []
        self.batches: Dict[Tuple, Tuple[Tuple[int, ...], Batch]] = {}
        self.ticks = 0
        self.max_concurrent = 0
        self._cancel: set = set()

    # -- admission / eviction -----------------------------------------------------------
    def cancel(self, jid: int):
        """Cancel a job: dropped from the queue, or released at the next tick if active."""
        self._cancel.add(jid)

    def _end(self, job: Job, status: str, now: float, error: str = ""):
        """A job that leaves without results (rejected, invalid, failed, cancelled)."""
        job.status, job.error, job.finished = status, error, now
        job.inputs = None
        self.done.append(job)

    @staticmethod
    def _finite_inputs(inp: Optional[I.Inputs]) -> bool:
        if inp is None:
            return True
        return all(a is None or bool(np.all(np.isfinite(a))) for a in (inp.vloc, inp.psi0, inp.pos, inp.D))

    def _admit(self, job: Job, now: float):
        job.nbytes = job_bytes(job.spec)
        inp = job.inputs if job.inputs is not None else self.make_inputs(job.spec)
        if not self._finite_inputs(inp):
            self._end(job, "invalid", now, "non-finite input")
            return
        try:
            job.system = System(job.spec, inp, stream=self.stream)
            job.system.set_clock(0.0, job.spec.dt, job.spec.substeps)
        except Exception as exc:  # the library refused this job (e.g. out of memory): it fails alone
            if job.system is not None:
                job.system.close()
                job.system = None
            self._end(job, "failed", now, str(exc))
            return
        job.admitted = now
        job.status = "active"
        self.used += job.nbytes
        self.peak_used = max(self.peak_used, self.used)
        self.active.append(job)
        self.max_concurrent = max(self.max_concurrent, len(self.active))

    def _release(self, job: Job):
        if job.system is not None:
            job.system.close()
            job.system = None
        job.inputs = None
        self.used -= job.nbytes
        self.active.remove(job)

    def _finish(self, job: Job, now_fn):
        try:
            job.records = job.system.reductions(0, job.n_steps)
            job.orbitals = job.system.get_orbitals() if self.keep_orbitals else None
        except Exception as exc:
            self._release(job)
            self._end(job, "failed", now_fn(), str(exc))
            return
        job.finished = now_fn()
        job.status = "done"
        self._release(job)
        self.done.append(job)

    def _fail_group(self, jobs: List[Job], key, exc: Exception, now: float):
        """A batch that reported an error: its jobs fail, the others are untouched."""
        if key in self.batches:
            self.batches.pop(key)[1].close()
        for j in jobs:
            self._release(j)
            self._end(j, "failed", now, str(exc))

    # -- one tick: every active job advances ---------------------------------------------
    def _tick(self, now: float = 0.0):
        groups: Dict[Tuple, List[Job]] = {}
        for j in self.active:
            key = (j.spec.prec, j.spec.fd_order, j.spec.substeps)
            groups.setdefault(key, []).append(j)
        for key in list(self.batches):
            if key not in groups:
                self.batches.pop(key)[1].close()
        advanced = []
        for key, jobs in groups.items():
            ids = tuple(j.jid for j in jobs)
            try:
                if key not in self.batches or self.batches[key][0] != ids:
                    if key in self.batches:
                        self.batches.pop(key)[1].close()
                    self.batches[key] = (ids, Batch([j.system for j in jobs], stream=self.stream))
                q = min(self.quantum, min(j.n_steps - j.steps_done for j in jobs))
                self.batches[key][1].propagate(q, use_graph=self.use_graph)
            except Exception as exc:
                self._fail_group(jobs, key, exc, now)
                continue
            advanced.append((jobs, q))
        self.sync()
        for jobs, q in advanced:
            for j in jobs:
                j.steps_done += q
        self.ticks += 1

    def run(self, jobs: List[Job], keep_orbitals: bool = False, time_scale: float = 1.0) -> List[Job]:
        """Serve the trace in real time (arrival times scaled by time_scale)."""
        self.keep_orbitals = keep_orbitals
        pending = sorted(jobs, key=lambda j: j.arrival)
        queue: List[Job] = []
        t0 = time.perf_counter()
        now = lambda: (time.perf_counter() - t0) / time_scale
        while pending or queue or self.active:
            t = now()
            while pending and pending[0].arrival <= t:
                queue.append(pending.pop(0))
            for j in [j for j in queue if j.jid in self._cancel]:
                queue.remove(j)
                self._end(j, "cancelled", t)
            for j in [j for j in self.active if j.jid in self._cancel]:
                self._release(j)
                self._end(j, "cancelled", t)
            while queue and len(self.active) < self.max_slots:
                nb = job_bytes(queue[0].spec)
                if nb > self.budget:
                    self._end(queue.pop(0), "rejected", t, f"needs {nb} bytes, more than the whole budget")
                    continue
                if self.used + nb > self.budget:
                    break
                self._admit(queue.pop(0), t)
            if not self.active:
                if pending:
                    time.sleep(max(0.0, (pending[0].arrival - now()) * time_scale))
                continue
            self._tick(t)
            for j in [j for j in self.active if j.steps_done >= j.n_steps]:
                self._finish(j, now)
        for _, b in self.batches.values():
            b.close()
        self.batches.clear()
        self.wall = now()
        return self.done

    def report(self) -> dict:
        ok = [j for j in self.done if j.status == "done"]
        lat = np.array([j.latency for j in ok]) if ok else np.array([math.nan])
        upd = sum(j.updates for j in ok)
        status: Dict[str, int] = {}
        for j in self.done:
            status[j.status] = status.get(j.status, 0) + 1
        return {"jobs": len(ok), "wall_s": self.wall, "updates": upd,
                "throughput": upd / self.wall if self.wall > 0 else math.nan,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "ticks": self.ticks, "peak_hbm_bytes": self.peak_used, "max_concurrent": self.max_concurrent,
                "status": status}
