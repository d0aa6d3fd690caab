"""Bounded device waits: a wait that runs out reports CBVH_ERR_TIMEOUT and the kernel returns.

The waits are those of an idle warp for donated work in a work-queue launch and of a block
for its staged treelets.  CBVH_OPT_WAIT_CAP shrinks them to a few polls, so that a small
query makes them run out on purpose: no fault, trap or endless loop is involved, the query
returns with the status word set, and the next query with the default cap is exact.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

EPS_NEAR = 1e-6
TOL_PQ = 1e-5
ERR_TIMEOUT = -6


@pytest.fixture(scope="module")
def cb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


@pytest.fixture(scope="module")
def c1(cb):
    c = synth.C1(4)
    (va, ta), (vb, tb) = c["A"], c["B"]
    Ao = oracle.BVH(va, ta, 18, 4, 16, 4096)
    Bo = oracle.BVH(vb, tb, 18, 4, 16, 4096)
    D = synth.scene_diameter(va, vb)
    P = oracle.filtered_poses(Ao, Bo, lambda cnt, r: synth.poses_box(cnt, seed=2001 + 7919 * r), 256, EPS_NEAR * D)
    return dict(A=cb.BVH(va, ta, 18, 4, 16, 4096), B=cb.BVH(vb, tb, 18, 4, 16, 4096), Ao=Ao, Bo=Bo, P=P, D=D)


@pytest.fixture
def restore(cb):
    yield
    cb.set_option(cb.OPT_WAIT_CAP, cb.WAIT_CAP_DEFAULT)
    cb.set_option(cb.OPT_SPLIT, cb.SPLIT_DEFAULT)
    cb.set_option(cb.OPT_STAGE_BYTES, 0)


def _distance_status(cb, A, B, P):
    import torch
    n = int(P.shape[0])
    dist = torch.empty(n, dtype=torch.float32, device=P.device)
    status = torch.zeros(1, dtype=torch.int32, device=P.device)
    wsb = cb.workspace_bytes(A, B, n, 1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=P.device)
    rc = cb.lib.cbvh_distance(A.handle, B.handle, C.c_void_p(P.data_ptr()), n, C.c_void_p(dist.data_ptr()),
                              C.c_void_p(ws.data_ptr()), wsb, C.c_void_p(status.data_ptr()),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0, cb.lib.cbvh_last_error().decode()
    return dist.cpu().numpy(), int(status.item())


def _exact(cb, c1, P):
    o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], c1["P"])
    o_d, _ = oracle.distance(c1["Ao"], c1["Bo"], c1["P"])
    res = cb.collide(c1["A"], c1["B"], P)
    assert res.status == 0
    assert (res.hit.cpu().numpy() == o_hit).all()
    assert (res.offsets.cpu().numpy() == o_off).all() and (res.pairs.cpu().numpy() == o_ij).all()
    d, st = _distance_status(cb, c1["A"], c1["B"], P)
    assert st == 0 and np.abs(d - o_d).max() <= TOL_PQ * c1["D"]


@pytest.mark.parametrize("split", ["queue", "rounds_queue"])
def test_work_queue_wait_runs_out_and_reports_timeout(cb, c1, restore, split):
    """Idle warps of a work-queue launch wait for donated tasks; with a one-poll cap every
    warp that finds no pose left gives up at once (256 poses, thousands of warps), so the
    query must come back with CBVH_ERR_TIMEOUT -- and the next one, with the default cap, is
    exact against the oracle."""
    import torch
    P = torch.as_tensor(c1["P"], device="cuda")
    cb.set_option(cb.OPT_SPLIT, cb.SPLIT_QUEUE if split == "queue" else cb.SPLIT_ROUNDS_QUEUE)
    cb.set_option(cb.OPT_WAIT_CAP, 1)
    res = cb.collide(c1["A"], c1["B"], P, check=False)
    torch.cuda.synchronize()
    assert res.status == ERR_TIMEOUT
    _, st = _distance_status(cb, c1["A"], c1["B"], P)
    assert st == ERR_TIMEOUT
    cb.set_option(cb.OPT_WAIT_CAP, cb.WAIT_CAP_DEFAULT)
    _exact(cb, c1, P)


def test_staging_wait_is_bounded(cb, c1, restore):
    """Blocks wait for their staged treelets (TMA bulk copies) on an mbarrier.  With a
    one-poll cap the first wait may run out before the copy lands: then the block reports
    CBVH_ERR_TIMEOUT, lets its copies land (the full default wait) and reads every treelet
    from global memory.  Either way the call returns, and the next query is exact."""
    import torch
    P = torch.as_tensor(c1["P"], device="cuda")
    cb.set_option(cb.OPT_SPLIT, cb.SPLIT_POSE)  # no work queue: only the staging wait is capped
    cb.set_option(cb.OPT_STAGE_BYTES, 4096)
    cb.set_option(cb.OPT_WAIT_CAP, 1)
    res = cb.collide(c1["A"], c1["B"], P, check=False)
    torch.cuda.synchronize()
    assert res.status in (0, ERR_TIMEOUT)
    if res.status == 0:  # the copies won the race: the result is the ordinary one
        o_hit, *_ = oracle.collide(c1["Ao"], c1["Bo"], c1["P"])
        assert (res.hit.cpu().numpy() == o_hit).all()
    cb.set_option(cb.OPT_WAIT_CAP, cb.WAIT_CAP_DEFAULT)
    _exact(cb, c1, P)
