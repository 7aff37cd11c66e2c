"""Benchmark: orbital-gridpoint updates per second of the real-time TDDFT step.

Workload (one "step" = one configured time step of the whole hot path): the medium
molecule, 96^3 grid, h = 0.25 bohr, 8th-order FD (25-point star), 64 orbitals, 16 atoms
with Gaussian wells and 4 Kleinman-Bylander projectors each, sin^2 laser pulse, LDA
exchange rebuilt from the density every sub-step, dt = 0.05 split into 4 Taylor-4
sub-steps, FP64 density/norm/energy/dipole record every step.  Default precision is the
mixed path (complex64 H psi and Taylor terms, complex128 state and FP64 reductions); the
same step in complex128 is measured alongside.  An update is one orbital at one grid
point advanced by one configured step.

Timing: W warm-up steps, then K steps between CUDA events on the system's stream, with
a device synchronise (and a barrier across ranks) on both sides; the working set
(~2.3 GB) is far larger than L2, so no flush is needed.  Multi-GPU runs split the
molecule's orbitals over the ranks with an FP64 density allreduce per sub-step (strong
scaling; --shard replicas runs independent copies instead); the time is the maximum over
ranks.

``--impl reference`` times the FP64 CPU oracle on the host cores on a bounded sample of
the same workload (a subset of the orbitals) and reports the same metric.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H.psi orbital-gridpoint updates/s (medium molecule, Taylor-4 step)"
UNIT = "updates/s"


SWEEP_SOURCES = ["tdks_sweep_tma.cu", "tdks_tma.cuh", "tdks_sweep_ws1.cu", "tdks_sweep_ws2.cu", "tdks_sweep_ws3.cu", "tdks_sweep_ws5.cu",
                 "tdks_sweep_ws4.cu", "tdks_sweep_common.cuh", "tdks_vec.cuh", "tdks_internal.cuh"]
WORKLOAD = ("medium molecule 96^3 h=0.25 order-8 FD, 64 orbitals, 16 atoms x 4 KB projectors, sin^2 pulse, "
            "LDA exchange, dt=0.05 as 4 Taylor-4 sub-steps")
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e data-sheet bandwidth, for context beside the measured peak
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "tma_sweep_medium_molecule.md")


def sweep_source_hash() -> str:
    """Hash of the stencil-sweep sources: a DRAM traffic figure taken with ncu is used only
    while the kernel it was measured on is unchanged."""
    import hashlib
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1912_07921_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_per_launch():
    """DRAM bytes (read + write) per sweep launch at 64 orbitals from the committed ncu
    summary, or None when the summary is absent or was taken on other kernel sources."""
    import re
    if not os.path.exists(TRAFFIC_PROFILE):
        return None
    m = re.search(r"traffic_bytes_per_launch_64_orbitals:\s*([0-9.eE+]+)\s*\(sweep source hash ([0-9a-f]+)\)",
                  open(TRAFFIC_PROFILE).read())
    if not m or m.group(2) != sweep_source_hash():
        return None
    return float(m.group(1))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _sweep_bytes(spec, sysm) -> float:
    """Algorithmic HBM bytes of the 4 stencil sweeps of one Taylor sub-step.

    Per (point, padded orbital): sweep 1 reads the state and writes t1; sweeps 2-3 read
    t_(k-1) and write t_k; sweep 4 reads t3, the state, t1, t2 and writes the state; plus
    per point V_eff (each sweep) and one density word per batch.  complex128: every array
    is 16 B per value.  complex64: terms 8 B; the state is hi + lo (8 B + 8 B), of which
    sweep 1 reads only hi (the FP32 stencil input).
    """
    bs, nb, eb, _ = sysm.layout()
    vals = spec.n_points * nb * bs * sysm.n_k
    st_first, st = (8.0, 16.0) if eb == 8 else (16.0, 16.0)
    per_val = (st_first + eb) + 2 * (eb + eb) + (eb + st + eb + eb + st)
    veff = 4 * spec.n_points * (4 if eb == 8 else 8)
    dens = spec.n_points * nb * sysm.n_k * 8
    return vals * per_val + veff + dens


def _sweep_bytes_by_term(spec, sysm):
    """_sweep_bytes split over the four Taylor-term sweeps (each reads the per-point V_eff
    record; the last writes the density words)."""
    bs, nb, eb, _ = sysm.layout()
    vals = spec.n_points * nb * bs * sysm.n_k
    st_first, st = (8.0, 16.0) if eb == 8 else (16.0, 16.0)
    veff = spec.n_points * (4 if eb == 8 else 8)
    dens = spec.n_points * nb * sysm.n_k * 8
    return [vals * (st_first + eb) + veff, vals * 2 * eb + veff, vals * 2 * eb + veff,
            vals * (eb + st + eb + eb + st) + veff + dens]


def _by_term(term_bytes, term_ms, peak):
    """Per Taylor-term sweep: average launch time (CUDA events in the timed region), the
    algorithmic bytes of one launch, and the achieved GB/s and its fraction of the peak."""
    out = []
    for b, (ms, n) in zip(term_bytes, term_ms):
        us = 1e3 * ms / max(n, 1)
        gbs = b / (us * 1e-6) / 1e9 if n else 0.0
        out.append({"avg_launch_us": us, "launches": n, "bytes_per_launch": b, "achieved": gbs,
                    "frac": gbs / peak})
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's); x itself at N = 1."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _free_port() -> int:
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Replicas: every rank advances its own copy of the workload, so the job's rate is the
    units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1912_07921_gb300 import inputs as I
    from paper_1912_07921_gb300.system import System, shape_count, shape_info
    import __graft_entry__

    torch.cuda.set_device(local_rank)
    dist = None
    shard = args.shard == "states"
    if world > 1 or shard:
        import torch.distributed as dist
        if world > 1:
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        else:  # one-rank group: the state-parallel path with its exchange on one GPU
            dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{_free_port()}", rank=0,
                                    world_size=1, device_id=torch.device("cuda", local_rank))
    prec = I.PREC_C64 if args.prec == "c64" else I.PREC_C128
    spec = I.medium_molecule(prec=prec)
    if args.n_orb:
        spec = dataclasses.replace(spec, n_orb=args.n_orb)
    inp = I.make_inputs(spec)
    stream = torch.cuda.Stream()
    if shard:
        # one molecule over the ranks: each holds its slice of the orbitals; the density and
        # the record's band sums are allreduced (NCCL) on the library's stream
        from paper_1912_07921_gb300.sharding import shard_system
        sysm, (o_lo, o_hi) = shard_system(spec, inp, rank, world, stream=stream.cuda_stream)
    else:
        sysm = System(spec, inp, stream=stream.cuda_stream)
        o_lo, o_hi = 0, spec.n_orb
    if args.sweep_path:
        sysm.set_sweep_path(args.sweep_path)
    tune = None
    if args.shape >= 0:
        sysm.set_sweep_shape(-1, args.shape)
    elif not args.no_tune:
        # the autotuner times every tile shape on each Taylor-term sweep of this system
        # (outside the timed region) and keeps the fastest per sweep
        tune = sysm.autotune(reps=5)
    subs = spec.substeps
    dt = spec.dt
    upd_per_step = spec.n_points * (o_hi - o_lo)  # this rank's orbital updates per step
    # the whole job's units per step: every replica's, or the one sharded molecule's
    job_per_step = spec.n_points * spec.n_orb if shard else upd_per_step * world

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    t = 0.0
    sysm.propagate(t, dt, args.warmup, subs)
    t += args.warmup * dt
    barrier()
    sysm.set_profiling(True)
    sysm.kernel_time(0), sysm.kernel_time(1), sysm.kernel_time(2)
    l0 = sysm.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        barrier()
        ev0.record(stream)
        sysm.propagate(t, dt, args.steps, subs)
        ev1.record(stream)
        barrier()
    t += args.steps * dt
    ms = ev0.elapsed_time(ev1)
    launches = sysm.launch_count() - l0
    sweep_ms, sweep_n = sysm.kernel_time(0)
    gath_ms, gath_n = sysm.kernel_time(1)
    aux_ms, aux_n = sysm.kernel_time(2)
    term_ms = [sysm.kernel_time(3 + k) for k in range(4)]
    sysm.set_profiling(False)
    rec = sysm.reductions(sysm.step_count() - 1, 1)[0]
    ms = max_over_ranks(ms, dist, "cuda")

    # end to end through the C interface with host buffers: every step uploads its input
    # orbitals from pinned memory, advances one configured step and reads the step's
    # observable record back.  The upload of step i+1's inputs is issued right after step i
    # is enqueued, so its copy and its packing (into the system's second upload buffer)
    # overlap step i on the GPU; step 0's upload is not overlapped.
    psi_host = torch.from_numpy(np.ascontiguousarray(inp.psi0[..., o_lo:o_hi]).view(np.float64)
                                .reshape(-1)).pin_memory()
    h2d = psi_host.numel() * 8
    e2e_steps = max(3, min(args.steps, 20))
    sysm.set_upload_buffers(2)  # a stream of uploads: each one packs while the step before it runs
    # the host link's upload rate on this machine, for context (one upload with its packing)
    barrier()
    u0 = time.perf_counter()
    sysm.set_orbitals_ptr(psi_host.data_ptr())
    barrier()
    upload_gbs = h2d / (time.perf_counter() - u0) / 1e9
    barrier()
    w0 = time.perf_counter()
    sysm.set_orbitals_ptr(psi_host.data_ptr())
    for i in range(e2e_steps):
        sysm.propagate(t, dt, 1, subs)
        if i + 1 < e2e_steps:
            sysm.set_orbitals_ptr(psi_host.data_ptr())
        r = sysm.reductions(sysm.step_count() - 1, 1)
        t += dt
    barrier()
    e2e_s = time.perf_counter() - w0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")

    out = None
    if rank == 0:
        peak, peak_kind = _peaks()
        bytes_sub = _sweep_bytes(sysm.spec, sysm)
        per_launch_bytes = bytes_sub / 4.0
        avg_launch_s = (sweep_ms / 1e3) / max(sweep_n, 1)
        achieved = per_launch_bytes / avg_launch_s / 1e9
        value = (job_per_step * args.steps / (ms / 1e3) if shard
                 else whole_job_rate(upd_per_step * args.steps, world, ms / 1e3))
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None,
            "dtype": "c64 terms + f64 state/reductions" if prec == I.PREC_C64 else "c128 (f64)",
            "data": "synthetic (seeded molecule: Gaussian orbitals, wells, KB projectors)",
            "config": {"workload": WORKLOAD,
                       "grid": [spec.nx, spec.ny, spec.nz], "n_orb": spec.n_orb, "substeps": subs,
                       "precision": args.prec, "l2": "working set > L2 (state 906 MB + terms), no flush",
                       "parallelism": f"states x{world} (density allreduce per sub-step)" if shard
                       else f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": "taylor stencil sweep (4 per sub-step)",
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak,
                         "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                         "traffic": _traffic_per_launch() if sysm.spec.n_orb == 64 and prec == I.PREC_C64
                         else None,
                         "sweep_source_hash": sweep_source_hash(),
                         "bytes_per_launch": per_launch_bytes, "avg_launch_us": avg_launch_s * 1e6,
                         "by_taylor_term": _by_term(_sweep_bytes_by_term(sysm.spec, sysm), term_ms, peak)},
            "kernel_ms": {"sweep": sweep_ms, "sweep_launches": sweep_n, "projector": gath_ms,
                          "projector_steps": gath_n, "density_lda_finalize": aux_ms, "aux_launches": aux_n},
            "sweep_shapes": {"chosen": sysm.sweep_shapes(),
                             "autotune_ms_per_launch": None if tune is None else
                             [[round(float(x), 4) for x in r] for r in tune],
                             "shapes": [list(shape_info(i)) for i in range(shape_count())],
                             "legend": "shape = (tile tx, ty, points per thread, consumer warps); "
                                       "ms[shape][sweep], sweeps t1..t4"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": {"value": (job_per_step * e2e_steps / e2e_s if shard
                              else whole_job_rate(upd_per_step * e2e_steps, world, e2e_s)), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * 8, "bytes_scope": "per rank",
                    "upload_gbs": upload_gbs,
                    "how": "per step: host orbitals (complex128, pinned) uploaded through tdks_set_orbitals, "
                           "one configured step, its record read back; step i+1's upload overlaps step i"},
            "last_record": {"t": rec[0], "norm": rec[1], "energy": rec[2], "dipole": list(rec[4:7])},
        }
    sysm.close()
    if dist is not None:
        dist.destroy_process_group()
    return out


# FP64 instructions (thread level: DADD, DMUL, DFMA) per orbital value of one complex128
# Taylor sub-step in the stencil sweeps, counted from the sweep source: per sweep the diagonal
# term (1 add, 2 mul), M = 4 stencil distances of 5 complex adds and 1 complex FMA (12 each),
# the Taylor coefficient (4); the last sweep adds the series combine (8 adds) and the density
# (|psi|^2: 2, the lane sum and weight: ~2).  3 x 55 + 67 = 232.
C128_FP64_INSTR_PER_VALUE_SUBSTEP = 232.0


def fp64_peak():
    """The FP64 FMA rate of this GPU from the library's probe kernel (thread-level FMA
    instructions per second), with the nominal rate of 2 per clock per SM beside it."""
    import ctypes
    import torch
    from paper_1912_07921_gb300 import _lib
    lib = _lib.load()
    r = ctypes.c_double(0.0)
    _lib.check(lib.tdks_fma_rate(0, ctypes.byref(r)))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return r.value, props.multi_processor_count


def run_c128_side(args):
    """The same step fully in complex128 (the FP64 path), fewer steps, with its roofline:
    the sweeps' FP64 instruction rate against the probe's FP64 FMA rate, and their
    algorithmic bytes against the HBM peak (the path is bound by the nearer of the two)."""
    import torch
    from paper_1912_07921_gb300 import inputs as I
    from paper_1912_07921_gb300.system import System
    spec = I.medium_molecule(prec=I.PREC_C128)
    inp = I.make_inputs(spec)
    stream = torch.cuda.Stream()
    sysm = System(spec, inp, stream=stream.cuda_stream)
    sysm.propagate(0.0, spec.dt, 2, spec.substeps)
    torch.cuda.synchronize()
    k = max(2, args.steps // 20)
    sysm.set_profiling(True)
    sysm.kernel_time(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sysm.propagate(0.1, spec.dt, k, spec.substeps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sweep_ms, sweep_n = sysm.kernel_time(0)
    sysm.set_profiling(False)
    bs, nb, eb, _ = sysm.layout()
    sub_bytes = _sweep_bytes(spec, sysm)
    sysm.close()
    values = spec.n_points * nb * bs  # padded orbital values per sweep
    substeps = sweep_n / 4.0
    sweep_s = sweep_ms / 1e3
    fma_rate, sms = fp64_peak()
    instr_rate = values * substeps * C128_FP64_INSTR_PER_VALUE_SUBSTEP / sweep_s
    peak, peak_kind = _peaks()
    hbm = sub_bytes * substeps / sweep_s / 1e9
    return {"value": spec.n_points * spec.n_orb * k / (ms / 1e3), "unit": UNIT, "steps": k,
            "ms_per_step": ms / k,
            "roofline": {"bound": "alu", "kernel": "taylor stencil sweeps, complex128",
                         "achieved": instr_rate / 1e9, "peak": fma_rate / 1e9, "unit": "G FP64 instr/s",
                         "frac": instr_rate / fma_rate,
                         "peak_kind": "measured (tdks_fma_rate probe: DFMA, thread level)",
                         "nominal_peak": 2.0 * sms * 2.07e9 / 1e9,
                         "fp64_instr_per_value_substep": C128_FP64_INSTR_PER_VALUE_SUBSTEP,
                         "hbm_achieved_gbs": hbm, "hbm_frac": hbm / peak, "hbm_peak": peak,
                         "avg_sweep_us": sweep_ms * 1e3 / max(sweep_n, 1)}}


def _batched_sweep_roofline(specs, systems, tune, shapes):
    """The four batched sweeps of a sub-step: the algorithmic bytes of every system over the
    autotuner's CUDA-event time of each Taylor term's chosen shape."""
    sub_bytes = sum(_sweep_bytes(sp, s) for sp, s in zip(specs, systems))
    sweep_s = sum(float(tune[sh][term]) for term, sh in enumerate(shapes)) / 1e3
    peak, peak_kind = _peaks()
    achieved = sub_bytes / sweep_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": achieved / peak, "bytes_per_substep": sub_bytes,
            "basis": "autotuner CUDA-event times of the chosen shape per Taylor term"}


def run_batched(args, n_sample=16, full_horizon=True):
    """The batched workload: n independent molecules (edges U[32,80], 4..32 orbitals,
    0..12 atoms with projectors, complex64, 4th-order FD, h = 0.25, dt = 0.015), advanced
    by one persistent sweep launch per Taylor term over all of them, replayed as a CUDA
    graph.  Also returns the first n_sample systems' records over the workload's 500 steps
    (full_horizon; else over the steps run) for the precision check."""
    import torch
    from paper_1912_07921_gb300 import inputs as I
    from paper_1912_07921_gb300.system import Batch, System
    specs = I.batched_systems(args.batched)
    stream = torch.cuda.Stream()
    systems = []
    for sp in specs:
        s = System(sp, I.make_inputs(sp), stream=stream.cuda_stream)
        s.set_clock(0.0, sp.dt, sp.substeps)
        systems.append(s)
    b = Batch(systems, stream=stream.cuda_stream)
    # the autotuner times every tile shape on each Taylor term's batched sweep (outside the
    # timed region) and keeps the fastest per term
    tune = None if args.no_tune else b.autotune(reps=2)
    b.propagate(2)
    torch.cuda.synchronize()
    k = max(2, args.steps // 10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.launch_count()
    e0.record(stream)
    b.propagate(k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    upd = sum(sp.n_points * sp.n_orb for sp in specs)
    out = {"systems": len(specs), "value": upd * k / (ms / 1e3), "unit": UNIT, "steps": k,
           "ms_per_step": ms / k, "values_per_step": upd, "launches": b.launch_count() - l0,
           "graph": True, "sweep_shapes": b.shapes(),
           "autotune_ms_per_launch": None if tune is None else [[round(float(x), 4) for x in r] for r in tune]}
    if tune is not None:
        out["sweep_roofline"] = _batched_sweep_roofline(specs, systems, tune, b.shapes())
    # the rest of the workload's steps (untimed), so that the precision check covers the
    # configured horizon
    horizon = max(sp.n_steps for sp in specs) if full_horizon else 2 + k
    if horizon > 2 + k:
        b.propagate(horizon - 2 - k)
        torch.cuda.synchronize()
    records = [systems[i].reductions(0, horizon) for i in range(min(n_sample, len(systems)))]
    b.close()
    for s in systems:
        s.close()
    return out, specs[:len(records)], records


def run_fp64_reference_path(specs, records32):
    """The plain FP64 single-system path on a sample of the batched systems: each system
    alone in complex128 (FP64 H psi, FP64 state), propagated over the same steps as the
    batched complex64 run.  Returns its throughput and the complex64 batch's dipole error
    against it: max over systems of max_t |d32(t) - d64(t)| / max_t |d64(t)|, and the same
    for the induced dipole d(t) - d(0)."""
    import dataclasses as dc
    import torch
    from paper_1912_07921_gb300 import inputs as I
    from paper_1912_07921_gb300.system import System
    stream = torch.cuda.Stream()
    tot_ms, tot_upd, err, err_ind = 0.0, 0, 0.0, 0.0
    for sp, r32 in zip(specs, records32):
        n = r32.shape[0]
        sp64 = dc.replace(sp, prec=I.PREC_C128)
        s = System(sp64, I.make_inputs(sp64), stream=stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.propagate(0.0, sp.dt, n, sp.substeps)
        e1.record(stream)
        torch.cuda.synchronize()
        tot_ms += e0.elapsed_time(e1)
        tot_upd += sp.n_points * sp.n_orb * n
        r64 = s.reductions(0, n)
        s.close()
        d32, d64 = r32[:, 4:7], r64[:, 4:7]
        err = max(err, float(np.max(np.abs(d32 - d64)) / np.max(np.abs(d64))))
        i32, i64 = d32 - d32[0], d64 - d64[0]
        if np.max(np.abs(i64)) > 0:
            err_ind = max(err_ind, float(np.max(np.abs(i32 - i64)) / np.max(np.abs(i64))))
    return {"value": tot_upd / (tot_ms / 1e3), "unit": UNIT, "systems": len(specs),
            "steps": int(records32[0].shape[0]), "dipole_err": err, "induced_dipole_err": err_ind}


def run_tiny_dipole_check():
    """Dipole of the tiny molecule over 1000 steps: complex64 H psi (double-float state,
    FP64 reductions) against complex128, both on the GPU."""
    import dataclasses as dc
    import torch
    from paper_1912_07921_gb300 import inputs as I
    from paper_1912_07921_gb300.system import System
    stream = torch.cuda.Stream()
    recs = []
    for prec in (I.PREC_C64, I.PREC_C128):
        spec = I.tiny_molecule(prec=prec, n_steps=1000)
        s = System(spec, I.make_inputs(spec), stream=stream.cuda_stream)
        s.propagate(0.0, spec.dt, spec.n_steps, spec.substeps)
        torch.cuda.synchronize()
        recs.append(s.reductions(0, spec.n_steps))
        s.close()
    d32, d64 = recs[0][:, 4:7], recs[1][:, 4:7]
    return float(np.max(np.abs(d32 - d64)) / np.max(np.abs(d64)))


def run_periodic_side(args):
    """The periodic cell (64^3 Bloch cell, 32 k-points x 16 bands in complex64, velocity
    gauge, 6 sub-steps per step) through the TMA sweep with autotuned tile shapes, a few
    steps."""
    import torch
    from paper_1912_07921_gb300 import inputs as I
    from paper_1912_07921_gb300.system import System
    spec = I.periodic_cell(n_k=args.periodic_k)
    inp = I.make_inputs(spec)
    stream = torch.cuda.Stream()
    sysm = System(spec, inp, stream=stream.cuda_stream)
    tune = None
    if args.shape >= 0:
        sysm.set_sweep_shape(-1, args.shape)
    elif not args.no_tune:
        tune = sysm.autotune(reps=3)
    sysm.propagate(0.0, spec.dt, 2, spec.substeps)
    torch.cuda.synchronize()
    k = max(2, args.steps // 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sysm.set_profiling(True)
    sysm.kernel_time(0)
    e0.record(stream)
    sysm.propagate(2 * spec.dt, spec.dt, k, spec.substeps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sweep_ms, sweep_n = sysm.kernel_time(0)
    sysm.set_profiling(False)
    shapes = sysm.sweep_shapes()
    sysm.close()
    states = spec.n_orb * spec.n_k
    # algorithmic bytes per sweep launch: 104 B per value per sub-step (as the medium molecule's
    # complex64 path) over four sweeps, plus the 16-byte point records per orbital block
    per_launch = (spec.n_points * states * 104 + spec.n_points * 16 * 4 * (states // 8)) / 4
    sweep_gbs = per_launch / ((sweep_ms / 1e3) / max(sweep_n, 1)) / 1e9
    peak, peak_kind = _peaks()
    return {"workload": f"periodic cell 64^3 L=10.2 order-4 FD, {spec.n_k} k x 16 bands c64, 8 atoms x 4 KB, "
                        "velocity gauge A0=0.2, dt=0.04 as 6 Taylor-4 sub-steps",
            "value": spec.n_points * states * k / (ms / 1e3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
            "sweep_gbs": sweep_gbs, "sweep_shapes": shapes,
            "roofline": {"bound": "hbm", "achieved": sweep_gbs, "peak": peak, "unit": "GB/s",
                         "frac": sweep_gbs / peak, "frac_of_nominal_7900": sweep_gbs / 7900.0,
                         "peak_kind": peak_kind, "traffic": None,
                         "bytes_per_launch": per_launch, "launches": sweep_n,
                         "avg_launch_us": 1e3 * sweep_ms / max(sweep_n, 1)},
            "autotune_ms_per_launch": None if tune is None else [[round(float(x), 4) for x in r] for r in tune]}


def run_propagator_study(args):
    """Cost against error of the propagators (the comparison of the paper's EMR/CFM4 figure,
    on a synthetic molecule): a 48^3 molecule (h = 0.25, order 8, 16 orbitals in complex128,
    6 atoms with projectors, LDA exchange, laser E0 = 0.02, omega = 0.5) over T = 1 (20 steps
    of dt = 0.05), with Taylor-4 and EMR (one exponential per sub-step) and RK4 (four stages)
    and ETRS (a trial exponential of the sub-step and two halves) at 4, 8, 16, AETRS and CFM4
    (two half exponentials) at 2, 4, 8 sub-steps per step;
    error = ||psi - psi_ref|| / ||psi_ref||, psi_ref from RK4 at 64 sub-steps per step (the
    density rebuilt at every stage, fourth order in the whole non-linear problem); time from
    CUDA events around each propagation."""
    import dataclasses as dc
    import torch
    from paper_1912_07921_gb300 import inputs as I
    from paper_1912_07921_gb300.system import System
    spec = dc.replace(I.medium_molecule(prec=I.PREC_C128), nx=48, ny=48, nz=48, n_orb=16, n_atoms=6, amp=0.02,
                      omega=0.5, envelope=I.ENV_NONE)
    inp = I.make_inputs(spec)
    stream = torch.cuda.Stream()
    T, n_steps = 1.0, 20
    dt = T / n_steps

    def run(prop, subs):
        s = System(spec, inp, stream=stream.cuda_stream)
        s.set_propagator(prop)
        s.propagate(0.0, dt, 1, subs)  # warm-up (then restart from the same state)
        s.set_orbitals(inp.psi0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.propagate(0.0, dt, n_steps, subs)
        e1.record(stream)
        torch.cuda.synchronize()
        psi = s.get_orbitals()
        s.close()
        return psi, e0.elapsed_time(e1)

    ref, _ = run(4, 64)
    nref = np.linalg.norm(ref)
    pts = []
    for prop, name, subs_list in ((0, "taylor4", (4, 8, 16)), (2, "emr", (4, 8, 16)), (3, "aetrs", (2, 4, 8)),
                                  (5, "etrs", (4, 8, 16)), (1, "cfm4", (2, 4, 8)), (4, "rk4", (4, 8, 16))):
        for subs in subs_list:
            psi, ms = run(prop, subs)
            pts.append({"propagator": name, "substeps": subs, "ms": round(ms, 2),
                        "err": float(np.linalg.norm(psi - ref) / nref)})
    return {"workload": "48^3 molecule h=0.25 order-8, 16 orbitals c128, 6 atoms x 4 KB, LDA exchange, "
                        "laser E0=0.02 omega=0.5, T=1 as 20 steps of dt=0.05",
            "reference": "RK4 at 64 sub-steps per step", "points": pts}


def run_serving(args):
    """A scaled serving trace (Poisson arrivals) through the continuous-batching server.
    Each request carries its inputs (built before the server starts, as a client would
    send them); latency runs from arrival to results on the host."""
    import torch
    from paper_1912_07921_gb300 import inputs as I, serving
    jobs = serving.serving_trace(args.serving, rate=20.0, seed=5, edge=(32, 64), orbitals=(4, 32),
                                 steps=(50, 400), atoms=(0, 16))
    for j in jobs:
        j.inputs = I.make_inputs(j.spec)
    stream = torch.cuda.Stream()
    srv = serving.Server(hbm_budget=150 * 10 ** 9, max_slots=64, quantum=50, stream=stream.cuda_stream,
                         sync=torch.cuda.synchronize)
    srv.run(jobs)
    r = srv.report()
    r["trace"] = (f"{args.serving} jobs, Poisson 20/s, edges U[32,64], orbitals U[4,32], steps U[50,400], "
                  f"atoms U[0,16], half complex64 / half complex128, 150 GB budget, 64 slots, quantum 50")
    return r


def run_serving_full(args):
    """The serving workload's size distribution: grid edges U[32,128], 4..128 orbitals,
    0..32 atoms with projectors, half complex64 and half complex128, a 150 GB HBM budget,
    Poisson arrivals; each job's step count drawn from U[200,5000] and divided by
    --serving-steps-scale (the whole distribution at full length offers ~1e11 updates per job,
    hours of GPU time for a few hundred jobs).  Two traces of the same jobs: the configured
    20 jobs/s (far above the GPU's capacity, so latency is queueing), then arrivals at 70% of
    the capacity measured on the first trace."""
    import torch
    from paper_1912_07921_gb300 import inputs as I, serving
    scale = max(1, args.serving_steps_scale)
    stream = torch.cuda.Stream()

    def trace(rate):
        jobs = serving.serving_trace(args.serving_full, rate=rate, seed=5, edge=(32, 128), orbitals=(4, 128),
                                     steps=(200, 5000), atoms=(0, 32))
        for j in jobs:
            j.n_steps = max(1, j.n_steps // scale)
            j.spec = dataclasses.replace(j.spec, n_steps=j.n_steps)
        return jobs

    def serve(jobs):
        srv = serving.Server(hbm_budget=150 * 10 ** 9, max_slots=64, quantum=50, stream=stream.cuda_stream,
                             sync=torch.cuda.synchronize)
        srv.run(jobs)
        return srv.report()

    sat = serve(trace(20.0))
    capacity = sat["jobs"] / sat["wall_s"]  # jobs per second the GPU completed under saturation
    relaxed = serve(trace(0.7 * capacity))
    desc = (f"{args.serving_full} jobs: edges U[32,128], orbitals U[4,128], atoms U[0,32], steps U[200,5000]/{scale}, "
            "half complex64 / half complex128, 150 GB budget, 64 slots, quantum 50")
    return {"trace": desc, "as_specified_20_per_s": sat,
            "at_0.7_utilisation": dict(relaxed, arrival_rate_per_s=0.7 * capacity)}


def cpu_baseline(n_orb_sample: int):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample: one
    configured step (4 sub-steps plus the observable record) of the medium molecule with
    n_orb_sample of its 64 orbitals."""
    import oracle
    from paper_1912_07921_gb300 import inputs as I
    spec = I.medium_molecule(prec=I.PREC_C128)
    inp = I.make_inputs(spec)
    inp.psi0 = np.ascontiguousarray(inp.psi0[..., :n_orb_sample])
    import dataclasses
    sspec = dataclasses.replace(spec, n_orb=n_orb_sample)
    o = oracle.System(sspec, inp)
    cores = len(os.sched_getaffinity(0))
    prev = oracle.set_threads(cores)
    t0 = time.perf_counter()
    o.propagate(inp.psi0, 0.0, spec.dt, 1, spec.substeps)
    s = time.perf_counter() - t0
    # the same oracle on one host thread, on a smaller sample of the same step
    n1 = 2
    inp1 = I.make_inputs(spec)
    inp1.psi0 = np.ascontiguousarray(inp1.psi0[..., :n1])
    o1 = oracle.System(dataclasses.replace(spec, n_orb=n1), inp1)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    o1.propagate(inp1.psi0, 0.0, spec.dt, 1, spec.substeps)
    s1 = time.perf_counter() - t1
    oracle.set_threads(prev)
    return {"value": spec.n_points * n_orb_sample / s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"1 configured step (4 sub-steps + record) of the medium molecule with "
                      f"{n_orb_sample} of 64 orbitals, {s:.1f} s",
            "single_thread": {"value": spec.n_points * n1 / s1, "unit": UNIT, "cores": 1,
                              "sample": f"the same step with {n1} of 64 orbitals, {s1:.1f} s"}}


def run_reference(args, rank):
    """The FP64 oracle on the host cores, on bounded samples of the medium molecule's step.

    Each step advances a sample of the 64 orbitals; the oracle's per-point work (density,
    exchange potential, record) does not shrink with the sample, so two sample sizes are
    timed (2 orbitals for the K timed steps, 4 orbitals for K/5 of them) and the step time
    is fitted as a + b n_orb; `value` is the rate that fit gives for all 64 orbitals, and the
    2-orbital rate is reported beside it."""
    if rank != 0:
        return None
    import oracle
    oracle.build()  # the CPU oracle only: this arm loads no CUDA code
    from paper_1912_07921_gb300 import inputs as I
    import dataclasses
    spec = I.medium_molecule(prec=I.PREC_C128)
    inp = I.make_inputs(spec)

    def timed(n_s, steps, warmup):
        psi = np.ascontiguousarray(inp.psi0[..., :n_s])
        o = oracle.System(dataclasses.replace(spec, n_orb=n_s), inp)
        for _ in range(warmup):
            psi, _ = o.propagate(psi, 0.0, spec.dt, 1, spec.substeps)
        t0 = time.perf_counter()
        for i in range(steps):
            psi, _ = o.propagate(psi, i * spec.dt, spec.dt, 1, spec.substeps)
        return (time.perf_counter() - t0) / steps

    n1, n2 = 2, 4
    k2 = max(2, args.steps // 5)
    s1 = timed(n1, args.steps, args.warmup)
    s2 = timed(n2, k2, 1)
    b = max((s2 - s1) / (n2 - n1), 1e-12)  # seconds per orbital per step
    a = max(s1 - b * n1, 0.0)              # seconds per step that do not scale with the orbitals
    s64 = a + b * spec.n_orb
    v = spec.n_points * spec.n_orb / s64
    v_sample = spec.n_points * n1 / s1
    cores = len(os.sched_getaffinity(0))
    sample = (f"{args.steps} steps with {n1} and {k2} with {n2} of the 64 orbitals; step time fitted as "
              f"a + b n_orb (a = {a:.3f} s, b = {b:.3f} s) and taken at 64 orbitals")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": s64 * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded molecule)",
            "config": {"workload": WORKLOAD, "grid": [spec.nx, spec.ny, spec.nz], "n_orb": spec.n_orb,
                       "substeps": spec.substeps, "precision": "c128 oracle", "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "sampled_value": v_sample,
                             "sampled": f"{n1} of 64 orbitals per step, {args.steps} steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-c128", action="store_true", help="skip the complex128 side measurement")
    ap.add_argument("--batched", type=int, default=256,
                    help="also measure the batched workload with this many systems (0: skip)")
    ap.add_argument("--no-periodic", action="store_true", help="skip the periodic-cell side measurement")
    ap.add_argument("--periodic-k", type=int, default=32,
                    help="k-points of the periodic cell (profiling on a smaller case); 32 = the workload")
    ap.add_argument("--serving", type=int, default=48,
                    help="also run a serving trace with this many jobs")
    ap.add_argument("--serving-full", type=int, default=0,
                    help="also serve this many jobs of the serving workload's full size distribution (0: skip)")
    ap.add_argument("--serving-steps-scale", type=int, default=25,
                    help="divide each full-distribution job's step count by this")
    ap.add_argument("--n-orb", type=int, default=0,
                    help="orbital count override (profiling on a smaller case); 0 = the workload's 64")
    ap.add_argument("--no-tune", action="store_true", help="keep the default sweep tile shape (no autotuner)")
    ap.add_argument("--no-study", action="store_true", help="skip the propagator cost-against-error study")
    ap.add_argument("--shape", type=int, default=-1, help="force one sweep tile shape for all Taylor terms")
    ap.add_argument("--shard", default="auto", choices=["auto", "replicas", "states"],
                    help="states: split one molecule's orbitals over the ranks with a density allreduce per "
                         "sub-step (strong scaling; also at --gpus 1); replicas: every rank runs its own copy; "
                         "auto (default): states on several GPUs, the single system on one")
    ap.add_argument("--sweep-path", type=int, default=0,
                    help="stencil sweep variant: 0 warp-specialised TMA (default), 1 general, 2 lockstep TMA")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    # NCCL's own log lines (its version banner, when NCCL_DEBUG asks for it) go to stderr, so
    # that rank 0's stdout holds the one JSON line
    os.environ.setdefault("NCCL_DEBUG_FILE", "/dev/stderr")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.shard == "auto":
        # one molecule over several GPUs is the paper's multi-GPU mode (states distributed)
        args.shard = "states" if world > 1 else "replicas"
    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out))
        return
    import __graft_entry__
    __graft_entry__.build()
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_c128 and args.prec == "c64" and world == 1:
            out["c128_path"] = run_c128_side(args)
        if args.batched and world == 1:
            out["batched"], sample, rec32 = run_batched(args)
            ref = run_fp64_reference_path(sample, rec32)
            out["fp32_vs_fp64"] = {
                "factor": out["batched"]["value"] / ref["value"],
                "fp32": "batched complex64 H psi (double-float state, FP64 reductions), all systems, graph",
                "fp64": f"each of the first {ref['systems']} batched systems alone in complex128",
                "fp64_value": ref["value"], "unit": UNIT,
                "dipole_err": ref["dipole_err"], "induced_dipole_err": ref["induced_dipole_err"],
                "dipole_err_over": f"{ref['steps']} steps of those systems (the workload's horizon)",
                "tiny_molecule_dipole_err_1000_steps": run_tiny_dipole_check(),
                "err_definition": "max_t |d32 - d64| / max_t |d64| (induced: d(t) - d(0))"}
        if not args.no_periodic and world == 1:
            out["periodic"] = run_periodic_side(args)
        if args.serving and world == 1:
            out["serving"] = run_serving(args)
        if args.serving_full and world == 1:
            out["serving_full"] = run_serving_full(args)
        if not args.no_study and world == 1:
            out["propagators"] = run_propagator_study(args)
        if not args.no_cpu and world == 1:
            out["cpu_baseline"] = cpu_baseline(32)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
