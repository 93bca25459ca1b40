"""The multi-GPU host logic on CPU: two gloo ranks (world size 2, 127.0.0.1)
run bench.py's rank helpers and a sharded campaign with a stand-in runner.
Ranks share no field data; only the timing maximum and the R/T scalars of a
campaign cross ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_runner(log):
    def run(specs, steps):
        log.extend(s.name for s in specs)
        R = np.array([s.lambda0 * 1e6 + 0.01 * s.nx + 0.5 * s.polarization for s in specs])
        return R, 1.0 - 2.0 * R
    return run


def _worker(rank, world, port):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        import bench
        from fdtd_inputs import config_c1b
        from paper_2512_17132_gb300 import campaign
        # timing: the slowest rank sets the job time; value aggregates all ranks
        assert bench._max_over_ranks(world, 1.5 + rank) == 1.5 + world - 1
        orders = [bench.rank_order(r, 5, 3) for r in range(world)]
        assert orders[0] != orders[1] and len(orders[rank]) == 8
        assert bench.aggregate_rate(world, 5, 1e9, 2.0) == world * 5 * 1e9 / 2.0 / 1e9
        # sharded campaign: every rank gets the whole result, runs only its share
        make = lambda lam: config_c1b(nx=100, steps=7).with_(lambda0=lam, name=f"s{lam:.0e}")
        wl = [500e-9, 600e-9, 700e-9]
        log_local, log_ref = [], []
        got = campaign.run_campaign(make, wl, n_slices=3, runner=_fake_runner(log_local),
                                    rank=rank, world=world)
        ref = campaign.run_campaign(make, wl, n_slices=3, runner=_fake_runner(log_ref))
        n_runs = len(wl) * 3 * 2
        assert len(log_ref) == n_runs
        assert len(log_local) == len(campaign.shard(n_runs, rank, world))
        for k in ("R_runs", "T_runs", "R", "T", "A"):
            np.testing.assert_array_equal(got[k], ref[k])
        assert sorted(sum((campaign.shard(n_runs, r, world) for r in range(world)), [])) == \
            list(range(n_runs))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_bench_helpers_and_sharded_campaign():
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)
