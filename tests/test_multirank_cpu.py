"""The multi-rank bench logic as two gloo ranks on the CPU: each rank reads its
rank from the launcher's environment, processes its own pairs (distinct
seeds), the job's time is the slowest rank's (MAX over ranks) and its value
the units of all ranks over that time; the reference arm runs on rank 0 only
(the other ranks exit at once)."""
import argparse
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench._dist_env()
        seeds = [bench.pair_seed(r, i) for i in range(2)]
        gathered = [None] * w
        dist.all_gather_object(gathered, seeds)
        t_max = bench.max_over_ranks(1.5 + r, dist, "cpu")          # rank 1 is the slow one
        args = argparse.Namespace(warmup=3, steps=3)
        ref_rc = bench.run_reference(args) if r != 0 else None      # rank 0 would run the oracle
        out.put((r, w, local, gathered, t_max, bench.job_rate(w, 200, t_max), ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_pairs_and_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, gathered, t_max, rate, ref_rc) in enumerate(res):
        assert (rank, w, local) == (r, world, r)
        all_seeds = [s for seeds in gathered for s in seeds]
        assert len(set(all_seeds)) == len(all_seeds)            # no pair processed twice
        assert t_max == 2.5                                      # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 200 / 2.5)              # all ranks' units over that time
    assert res[1][6] == 0                                        # reference arm: rank 1 exits at once


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    saved = {k: os.environ.pop(k, None) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    try:
        assert bench._dist_env() == (0, 1, 0)
        assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
        assert bench.job_rate(1, 20, 0.5) == 40
    finally:
        for k, v in saved.items():
            if v is not None:
                os.environ[k] = v
