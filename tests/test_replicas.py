"""The replica (N > 1) logic of bench.py on CPU ranks: two gloo processes stand in for two
GPUs.  Each rank reports its own time; the job's time is the slowest rank's and the job's rate
counts every rank's units (weak scaling, no data-path collective).  The reference arm runs on
rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.0 + 0.5 * rank              # ranks finish at different times
        slowest = bench.max_over_ranks(mine, dist, "cpu")
        rate = bench.whole_job_rate(1000.0, world, slowest)
        dist.barrier()
        out[rank] = (slowest, rate)
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_rate_counts_all_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert got[0] == got[1]
    slowest, rate = got[0]
    assert slowest == 1.5
    assert rate == pytest.approx(1000.0 * 2 / 1.5)


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(gpus=2, steps=1, warmup=3)
    assert bench.run_reference(args, rank=1) is None


def test_batched_sweep_roofline_uses_the_chosen_shape_of_each_term():
    """The batched roofline divides the systems' algorithmic sweep bytes by the sum of the
    autotuner's times of the shape chosen for each Taylor term."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_1912_07921_gb300 import inputs as I

    class Layout:  # what System.layout reports for a complex64 system
        def __init__(self, sp):
            self.sp, self.n_k = sp, 1

        def layout(self):
            return 8, -(-self.sp.n_orb // 8), 8, 0

    specs = I.batched_systems(4)
    systems = [Layout(sp) for sp in specs]
    tune = np.full((5, 4), 9.0)
    tune[2] = [0.5, 9.0, 9.0, 0.9]
    tune[1] = [9.0, 0.3, 0.3, 9.0]
    r = bench._batched_sweep_roofline(specs, systems, tune, [2, 1, 1, 2])
    want = sum(bench._sweep_bytes(sp, s) for sp, s in zip(specs, systems)) / 2.0e-3 / 1e9
    assert r["achieved"] == pytest.approx(want) and r["frac"] == pytest.approx(want / r["peak"])
