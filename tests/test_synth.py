"""Input generators: checks of the pose arithmetic the workloads are built from (no part of
the method; the oracle and the engine consume the same generated inputs)."""
import numpy as np

import synth


def test_relative_poses_compose_to_the_world_pose():
    """synth.relative_poses: applying link j's pose in link i's frame and then link i's
    world pose equals link j's world pose (checked on points, in FP64)."""
    q = np.random.default_rng(3).uniform(-np.pi, np.pi, size=(20, 6))
    LP = synth.dh_link_poses(q).astype(np.float64)
    x = np.random.default_rng(4).normal(size=(5, 3))
    for i, j in synth.self_pairs(6):
        rel = synth.relative_poses(LP, i, j).astype(np.float64)
        for n in range(20):
            Rr, tr = rel[n, :9].reshape(3, 3), rel[n, 9:]
            Ri, ti = LP[n, i, :9].reshape(3, 3), LP[n, i, 9:]
            Rj, tj = LP[n, j, :9].reshape(3, 3), LP[n, j, 9:]
            world_via_i = (Ri @ (Rr @ x.T + tr[:, None])).T + ti
            assert np.allclose(world_via_i, (Rj @ x.T).T + tj, atol=1e-5)
    assert len(synth.self_pairs(6)) == 10
