"""The multi-rank path of bench.py, on CPU with two gloo ranks.

Rays are independent, so under torchrun every rank renders a shard of its
own (replicas of the tree, no data exchange); the only collectives are the
timing reductions.  These tests run those host-side pieces as two real
processes over a gloo process group: the job's time is the slowest rank's,
the whole-job rate counts every rank's rays, and the ranks' shards differ.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    import plogen
    assert bench.dist_env() == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's own timing; the job's is the largest
        t = bench.max_over_ranks(10.0 + 7.5 * rank, dist, "cpu")
        # each rank's shard of rays
        rays = plogen.rays_room(256, seed=bench.shard_seed(rank))
        np.save(os.path.join(out_dir, f"rays{rank}.npy"), rays)
        with open(os.path.join(out_dir, f"t{rank}.txt"), "w") as f:
            f.write(repr(t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    # both ranks agree on the slowest rank's time
    for r in range(world):
        assert float((tmp_path / f"t{r}.txt").read_text()) == 17.5
    # the shards differ, and each is the single-process stream for its seed
    sys.path.insert(0, ROOT)
    import bench
    import plogen
    a, b = np.load(tmp_path / "rays0.npy"), np.load(tmp_path / "rays1.npy")
    assert not np.any(np.all(a == b, axis=1))
    np.testing.assert_array_equal(a, plogen.rays_room(256, seed=bench.shard_seed(0)))
    np.testing.assert_array_equal(b, plogen.rays_room(256, seed=bench.shard_seed(1)))


def test_job_rate_and_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    # whole-job throughput: every rank's rays over the slowest rank's time
    assert bench.job_rate(2, 1000, 5, 2.0) == pytest.approx(0.005)
    assert bench.job_rate(8, 1 << 24, 20, 1.1) == pytest.approx(8 * (1 << 24) * 20 / 1.1 / 1e6)
    # without a process group the value passes through
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
