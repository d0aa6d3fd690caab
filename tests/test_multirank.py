"""The benchmark's multi-GPU path on CPU: two gloo ranks.

Poses shard with no data-path collective (weak scaling: each rank draws its own poses of
the same distribution); the only collectives are the timing reductions -- the slowest
rank's time -- and the whole-job rate divides all ranks' units by it.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 37.0 * rank
        m = bench.max_over_ranks(local_ms, "cpu")
        rate = bench.whole_job_rate(2 * 1000 * 5, world, m)
        _, _, H = synth.heightfield(64, 4.0, seed=1002)
        P = bench.rank_poses(64, rank, H)
        np.save(os.path.join(out, f"poses{rank}.npy"), P)
        with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
            f.write(f"{m} {rate}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    vals = [tuple(map(float, open(tmp_path / f"r{r}.txt").read().split())) for r in range(2)]
    assert vals[0] == vals[1] == (137.0, 2 * 1000 * 5 * 2 / 0.137)
    p0, p1 = np.load(tmp_path / "poses0.npy"), np.load(tmp_path / "poses1.npy")
    assert p0.shape == p1.shape == (64, 12) and not np.allclose(p0, p1)
    import bench
    import synth
    _, _, H = synth.heightfield(64, 4.0, seed=1002)
    assert np.array_equal(bench.rank_poses(64, 1, H), p1)  # deterministic per rank
    assert np.array_equal(bench.rank_poses(64, 0, H), synth.poses_terrain(64, seed=2002, height_fn=H))


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
    assert bench.whole_job_rate(1000, 1, 500.0) == 2000.0
