"""The allocation-free proximity query against the ordinary one.

cbvh_distance_noalloc serves callers that cannot give the library device memory while they
run (a planner loop that must not block on the allocator, a plug-in whose host owns all
device memory): its scratch is a fixed array inside the library.  It must return what
cbvh_distance returns, and keep doing so on the next call, when the array still holds the
previous call's contents.  This file is collected last and also runs on its own.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL_PQ = 1e-5  # fraction of the scene diameter, as in the parity tests


@pytest.fixture(scope="module")
def cb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


def _noalloc(cb, A, B, P):
    import torch
    n = int(P.shape[0])
    dist = torch.full((n,), -1.0, dtype=torch.float32, device=P.device)
    status = torch.full((1,), 12345, dtype=torch.int32, device=P.device)
    rc = cb.lib.cbvh_distance_noalloc(A.handle, B.handle, C.c_void_p(P.data_ptr()), n, C.c_void_p(dist.data_ptr()),
                                      C.c_void_p(status.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0, cb.lib.cbvh_last_error().decode()
    assert int(status.item()) == 0
    return dist.cpu().numpy()


def test_distance_noalloc_matches_the_oracle_on_two_calls(cb):
    """The small sphere pair (1,280 triangles each, 256 poses away from contact) against the
    FP64 oracle: within 1e-5 of the scene diameter, zero exactly where the oracle's is."""
    import torch
    import oracle
    c = synth.C1(4)
    (va, ta), (vb, tb) = c["A"], c["B"]
    Ao = oracle.BVH(va, ta, 18, 4, 16, 4096)
    Bo = oracle.BVH(vb, tb, 18, 4, 16, 4096)
    D = synth.scene_diameter(va, vb)
    P = oracle.filtered_poses(Ao, Bo, lambda cnt, r: synth.poses_box(cnt, seed=2001 + 7919 * r), 256, 1e-6 * D)
    o_d, _ = oracle.distance(Ao, Bo, P)
    A = cb.BVH(va, ta, 18, 4, 16, 4096)
    B = cb.BVH(vb, tb, 18, 4, 16, 4096)
    Pd = torch.as_tensor(P, device="cuda")
    for _ in range(2):
        got = _noalloc(cb, A, B, Pd).astype(np.float64)
        assert np.abs(got - o_d).max() <= TOL_PQ * D
        assert ((got == 0) == (o_d == 0)).all()
    assert (o_d == 0).sum() > 20 and (o_d > 0).sum() > 20


def test_distance_noalloc_sequence_of_different_pairs(cb):
    """Spheres, then the terrain at the full 10,000 poses (about half a million tasks handed
    on between rounds, half the fixed task buffers), then the spheres again: each call
    equals cbvh_distance, whatever the previous call left in the shared array."""
    import torch
    s = synth.C1(300)
    t = synth.C2(10000)
    cases = []
    for c, cfg in ((s, (18, 4, 16, 4096)), (t, (24, 8, 8, 16384))):
        (va, ta), (vb, tb) = c["A"], c["B"]
        A, B = cb.BVH(va, ta, *cfg), cb.BVH(vb, tb, *cfg)
        P = torch.as_tensor(c["poses"], device="cuda")
        cases.append((A, B, P, synth.scene_diameter(va, vb), cb.distance(A, B, P).cpu().numpy()))
    for k in (0, 1, 0):
        A, B, P, D, ref = cases[k]
        got = _noalloc(cb, A, B, P)
        assert np.abs(got - ref).max() <= TOL_PQ * D
        assert ((got == 0) == (ref == 0)).all()


@pytest.mark.parametrize("case", ["spheres", "terrain"])
def test_distance_noalloc_matches_distance_on_two_calls(cb, case):
    import torch
    if case == "spheres":
        c = synth.C1(300)
        (va, ta), (vb, tb) = c["A"], c["B"]
        cfg = (18, 4, 16, 4096)
    else:
        c = synth.C2(600, cells=256)
        (va, ta), (vb, tb) = c["A"], c["B"]
        cfg = (24, 8, 8, 16384)
    A = cb.BVH(va, ta, *cfg)
    B = cb.BVH(vb, tb, *cfg)
    P = torch.as_tensor(c["poses"], device="cuda")
    D = synth.scene_diameter(va, vb)
    ref = cb.distance(A, B, P).cpu().numpy()
    first = _noalloc(cb, A, B, P)
    second = _noalloc(cb, A, B, P)
    for got in (first, second):
        assert np.abs(got - ref).max() <= TOL_PQ * D
    assert (ref == 0).sum() > 0 and (ref > 0).sum() > 0
