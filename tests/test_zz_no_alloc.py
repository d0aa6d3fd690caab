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
