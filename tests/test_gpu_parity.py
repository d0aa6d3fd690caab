"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Bars: decoded bounds bit-exact (lattice integers and FP32 bits); CD hit flags and
intersecting-pair sets bit-exact on poses that the oracle's near-contact filter keeps
(no triangle pair within 1e-6 D of contact, D = scene diameter); PQ within 1e-5 D per pose.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

EPS_NEAR = 1e-6   # near-contact band, fraction of the scene diameter
TOL_PQ = 1e-5     # PQ tolerance, fraction of the scene diameter


@pytest.fixture(scope="module")
def cb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


def _pairs_by_pose(off, ij):
    off = np.asarray(off)
    ij = np.asarray(ij)
    return [ij[off[p]:off[p + 1]] for p in range(len(off) - 1)]


def _gpu(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _check_cd(res, o_hit, o_off, o_ij):
    hit = res.hit.cpu().numpy()
    off = res.offsets.cpu().numpy()
    ij = res.pairs.cpu().numpy()
    assert (hit == o_hit).all(), np.nonzero(hit != o_hit)[0][:10]
    assert (off == o_off).all()
    assert ij.shape == o_ij.shape and (ij == o_ij).all()


def _filtered(Ao, Bo, draw, n, D):
    return oracle.filtered_poses(Ao, Bo, draw, n, EPS_NEAR * D)


# ------------------------------------------------------------------ decode
@pytest.fixture
def bottom_up(cb):
    cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_BOTTOM_UP)
    yield
    cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)


@pytest.mark.parametrize("packing", [0, 1])
@pytest.mark.parametrize("k,m,bits,tb", [(18, 4, 16, 4096), (24, 8, 8, 16384), (6, 2, 8, 4096),
                                         (26, 16, 16, 8192), (18, 4, 0, 4096), (24, 8, 16, 65536),
                                         (18, 4, 1, 4096), (24, 8, 1, 16384), (18, 4, 2, 4096), (24, 8, 2, 16384),
                                         (26, 16, 2, 8192), (6, 2, 2, 65536)])
def test_decode_bit_exact(cb, k, m, bits, tb, packing):
    v, t = synth.icosphere(4, 1.0, 0.15, seed=40 + k)
    cb.set_option(cb.OPT_TREELET_PACKING, packing)
    try:
        h = cb.BVH(v, t, k, m, bits, tb)
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
    lat, f = h.decode_all()
    o_lat, o_f, _ = oracle.decode_blob(h.blob_host())
    assert (f.cpu().numpy().view(np.uint32) == o_f.view(np.uint32)).all()
    if bits >= 8 or bits == 2:
        assert (lat.cpu().numpy() == o_lat).all()


@pytest.mark.parametrize("bits", [8, 2])
def test_decode_bit_exact_terrain(cb, bits):
    c = synth.C2(1, cells=512)
    h = cb.BVH(*c["A"], 24, 8, bits, 16384)
    lat, f = h.decode_all()
    o_lat, o_f, _ = oracle.decode_blob(h.blob_host())
    assert (lat.cpu().numpy() == o_lat).all()
    assert (f.cpu().numpy().view(np.uint32) == o_f.view(np.uint32)).all()


# ------------------------------------------------------------------ C1: small case, in full
@pytest.fixture(scope="module")
def c1(cb):
    c = synth.C1(4)
    (va, ta), (vb, tb) = c["A"], c["B"]
    Ao = oracle.BVH(va, ta, 18, 4, 16, 4096)
    Bo = oracle.BVH(vb, tb, 18, 4, 16, 4096)
    D = synth.scene_diameter(va, vb)
    P = _filtered(Ao, Bo, lambda cnt, r: synth.poses_box(cnt, seed=2001 + 7919 * r), 256, D)
    A = cb.BVH(va, ta, 18, 4, 16, 4096)
    B = cb.BVH(vb, tb, 18, 4, 16, 4096)
    return dict(A=A, B=B, Ao=Ao, Bo=Bo, P=P, D=D, mesh=(va, ta, vb, tb))


def test_c1_collide_bit_exact(cb, c1):
    o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], c1["P"])
    assert o_hit.sum() > 20 and (o_hit == 0).sum() > 20
    res = cb.collide(c1["A"], c1["B"], _gpu(c1["P"]))
    _check_cd(res, o_hit, o_off, o_ij)


def test_c1_collide_hits_only_and_early_exit(cb, c1):
    o_hit, *_ = oracle.collide(c1["Ao"], c1["Bo"], c1["P"])
    P = _gpu(c1["P"])
    r1 = cb.collide(c1["A"], c1["B"], P, pairs=False)
    r2 = cb.collide(c1["A"], c1["B"], P, pairs=False, early_exit=True)
    assert (r1.hit.cpu().numpy() == o_hit).all()
    assert (r2.hit.cpu().numpy() == o_hit).all()


def test_c1_distance_within_tolerance(cb, c1):
    o_d, _ = oracle.distance(c1["Ao"], c1["Bo"], c1["P"])
    d = cb.distance(c1["A"], c1["B"], _gpu(c1["P"])).cpu().numpy().astype(np.float64)
    tol = TOL_PQ * c1["D"]
    assert np.abs(d - o_d).max() <= tol
    assert ((d == 0) == (o_d == 0)).all()
    assert (o_d > 0).sum() > 20


def test_brute_force_agrees_on_a_c1_subset(cb, c1):
    """The GPU against the plain definition (all triangle pairs), not only Algorithm 1."""
    P = c1["P"][:24]
    b_hit, b_off, b_ij = oracle.brute_collide(c1["Ao"], c1["Bo"], P)
    res = cb.collide(c1["A"], c1["B"], _gpu(P))
    _check_cd(res, b_hit, b_off, b_ij)
    b_d = oracle.brute_distance(c1["Ao"], c1["Bo"], P)
    d = cb.distance(c1["A"], c1["B"], _gpu(P)).cpu().numpy()
    assert np.abs(d - b_d).max() <= TOL_PQ * c1["D"]


@pytest.mark.parametrize("stage", [4096, 16384, 32768])
def test_staged_treelets_against_oracle(cb, c1, stage):
    """Treelet staging (Sec. III-B: treelets sized to a cache, here shared memory filled by
    TMA bulk copies): with the leading treelets of both hierarchies read from shared memory
    (one to eight of the small case's 4 KB treelets), collision is bit-exact and distances
    within 1e-5 D against the oracle."""
    o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], c1["P"])
    o_d, _ = oracle.distance(c1["Ao"], c1["Bo"], c1["P"])
    cb.set_option(cb.OPT_STAGE_BYTES, stage)
    try:
        res = cb.collide(c1["A"], c1["B"], _gpu(c1["P"]))
        d = cb.distance(c1["A"], c1["B"], _gpu(c1["P"])).cpu().numpy().astype(np.float64)
    finally:
        cb.set_option(cb.OPT_STAGE_BYTES, 0)
    _check_cd(res, o_hit, o_off, o_ij)
    assert np.abs(d - o_d).max() <= TOL_PQ * c1["D"]
    assert ((d == 0) == (o_d == 0)).all()


@pytest.mark.parametrize("split,budget0", [(0, 256), (1, 16), (2, 16), (3, 16), (4, 1)])
def test_work_mappings_against_oracle(cb, c1, split, budget0):
    """Every work mapping -- one warp per pose to the end, rounds of handed-on tasks, one
    launch over a work queue with donation, rounds ending in a queue round -- with small
    budgets so that tasks are handed on and donated often: collision bit-exact and
    distances within 1e-5 D against the oracle."""
    o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], c1["P"])
    o_d, _ = oracle.distance(c1["Ao"], c1["Bo"], c1["P"])
    cb.set_option(cb.OPT_SPLIT, split)
    cb.set_option(cb.OPT_BUDGET0, budget0)
    try:
        res = cb.collide(c1["A"], c1["B"], _gpu(c1["P"]))
        flags = cb.collide(c1["A"], c1["B"], _gpu(c1["P"]), pairs=False).hit.cpu().numpy()
        d = cb.distance(c1["A"], c1["B"], _gpu(c1["P"])).cpu().numpy().astype(np.float64)
    finally:
        cb.set_option(cb.OPT_SPLIT, cb.SPLIT_DEFAULT)
        cb.set_option(cb.OPT_BUDGET0, cb.BUDGET0_DEFAULT)
    _check_cd(res, o_hit, o_off, o_ij)
    assert (flags == o_hit).all()
    assert np.abs(d - o_d).max() <= TOL_PQ * c1["D"]
    assert ((d == 0) == (o_d == 0)).all()


@pytest.mark.parametrize("k,m,bits,tb", [(6, 2, 8, 4096), (18, 4, 0, 4096), (18, 4, 8, 4096), (24, 8, 16, 16384),
                                         (26, 16, 16, 8192), (24, 16, 8, 131072), (18, 2, 16, 65536),
                                         (18, 4, 1, 4096), (24, 8, 1, 16384), (18, 4, 2, 4096), (24, 8, 2, 16384),
                                         (26, 16, 2, 8192)])
def test_other_configs_bit_exact(cb, c1, k, m, bits, tb):
    va, ta, vb, tb_ = c1["mesh"]
    A = cb.BVH(va, ta, k, m, bits, tb)
    B = cb.BVH(vb, tb_, k, m, bits, tb)
    P = c1["P"][:96]
    o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], P)
    _check_cd(cb.collide(A, B, _gpu(P)), o_hit, o_off, o_ij)
    o_d, _ = oracle.distance(c1["Ao"], c1["Bo"], P)
    d = cb.distance(A, B, _gpu(P)).cpu().numpy()
    assert np.abs(d - o_d).max() <= TOL_PQ * c1["D"]


@pytest.mark.parametrize("k,m,bits,tb", [(18, 4, 16, 4096), (24, 8, 8, 16384), (18, 4, 8, 131072), (18, 4, 0, 16384),
                                         (24, 8, 2, 16384)])
def test_bottom_up_packing_bit_exact(cb, c1, bottom_up, k, m, bits, tb):
    va, ta, vb, tb_ = c1["mesh"]
    A = cb.BVH(va, ta, k, m, bits, tb)
    B = cb.BVH(vb, tb_, k, m, bits, tb)
    P = c1["P"][:128]
    o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], P)
    _check_cd(cb.collide(A, B, _gpu(P)), o_hit, o_off, o_ij)
    o_d, _ = oracle.distance(c1["Ao"], c1["Bo"], P)
    d = cb.distance(A, B, _gpu(P)).cpu().numpy()
    assert np.abs(d - o_d).max() <= TOL_PQ * c1["D"]


def test_mixed_configs_for_A_and_B(cb, c1):
    va, ta, vb, tb_ = c1["mesh"]
    A = cb.BVH(va, ta, 24, 8, 8, 16384)
    B = cb.BVH(vb, tb_, 6, 2, 16, 4096)
    P = c1["P"][:64]
    o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], P)
    _check_cd(cb.collide(A, B, _gpu(P)), o_hit, o_off, o_ij)


# ------------------------------------------------------------------ edge cases
def test_empty_and_ragged_pose_counts(cb, c1):
    import torch
    for n in (0, 1, 3, 31, 33, 129):
        P = c1["P"][:n]
        res = cb.collide(c1["A"], c1["B"], _gpu(P.reshape(-1, 12)) if n else torch.empty((0, 12), device="cuda"))
        assert res.hit.numel() == n and res.offsets.cpu().numpy()[-1] == res.pairs.shape[0]
        if n:
            o_hit, o_off, o_ij, _ = oracle.collide(c1["Ao"], c1["Bo"], P)
            _check_cd(res, o_hit, o_off, o_ij)
            d = cb.distance(c1["A"], c1["B"], _gpu(P)).cpu().numpy()
            o_d, _ = oracle.distance(c1["Ao"], c1["Bo"], P)
            assert np.abs(d - o_d).max() <= TOL_PQ * c1["D"]


def test_capacity_overflow_reports_and_retries(cb, c1):
    import torch
    P = _gpu(c1["P"][:64])
    full = cb.collide(c1["A"], c1["B"], P)
    total = full.pairs.shape[0]
    assert total > 4
    r = cb.collide(c1["A"], c1["B"], P, capacity=total - 1, check=False)  # retried internally
    assert r.status == 0 and (r.pairs.cpu().numpy() == full.pairs.cpu().numpy()).all()
    # the raw C call reports CAPACITY with the exact requirement
    import ctypes as C
    n = 64
    hit = torch.empty(n, dtype=torch.uint8, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    prs = torch.empty((2, 2), dtype=torch.int32, device="cuda")
    need = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    wsb = cb.workspace_bytes(c1["A"], c1["B"], n, 0, 2)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    rc = cb.lib.cbvh_collide(c1["A"].handle, c1["B"].handle, C.c_void_p(P.data_ptr()), n, C.c_void_p(hit.data_ptr()),
                             C.c_void_p(off.data_ptr()), C.c_void_p(prs.data_ptr()), 2, C.c_void_p(need.data_ptr()),
                             2, C.c_void_p(ws.data_ptr()), wsb, C.c_void_p(st.data_ptr()),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and int(st.item()) == -4 and int(need.item()) == total
    assert (hit.cpu().numpy() == full.hit.cpu().numpy()).all()
    assert (off.cpu().numpy() == full.offsets.cpu().numpy()).all()


def test_single_triangle_meshes(cb):
    va = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    ta = np.array([[0, 1, 2]], np.int32)
    vb = np.array([[0.2, 0.2, -0.5], [0.3, 0.2, 0.5], [0.2, 0.35, 0.5]], np.float32)
    A = cb.BVH(va, ta, 18, 4, 16, 4096)
    B = cb.BVH(vb, ta, 18, 4, 16, 4096)
    Ao = oracle.BVH(va, ta, 18, 4, 16, 4096)
    Bo = oracle.BVH(vb, ta, 18, 4, 16, 4096)
    eye = np.concatenate([np.eye(3).ravel(), [0, 0, 0]])
    P = np.array([eye, eye + np.r_[np.zeros(9), [0, 0, 2.0]], eye + np.r_[np.zeros(9), [0.5, 0.5, 0.0]]], np.float32)
    o_hit, o_off, o_ij, _ = oracle.collide(Ao, Bo, P)
    assert list(o_hit) == [1, 0, 0]
    _check_cd(cb.collide(A, B, _gpu(P)), o_hit, o_off, o_ij)
    o_d, _ = oracle.distance(Ao, Bo, P)
    d = cb.distance(A, B, _gpu(P)).cpu().numpy()
    assert np.abs(d - o_d).max() <= 1e-5 * 3


def test_compressed_and_uncompressed_agree(cb, c1):
    va, ta, vb, tb_ = c1["mesh"]
    P = _gpu(c1["P"])
    res, dists = [], []
    for bits in (0, 1, 8, 16):
        A = cb.BVH(va, ta, 18, 4, bits, 4096)
        B = cb.BVH(vb, tb_, 18, 4, bits, 4096)
        res.append(cb.collide(A, B, P))
        dists.append(cb.distance(A, B, P).cpu().numpy())
    for r in res[1:]:
        assert (r.hit.cpu().numpy() == res[0].hit.cpu().numpy()).all()
        assert (r.pairs.cpu().numpy() == res[0].pairs.cpu().numpy()).all()
    for d in dists[1:]:
        assert np.abs(d - dists[0]).max() <= 1e-6 * c1["D"]


# ------------------------------------------------------------------ C2 at full size
@pytest.fixture(scope="module")
def c2(cb):
    c = synth.C2(10000)
    A = cb.BVH(*c["A"], 24, 8, 8, 16384)
    B = cb.BVH(*c["B"], 24, 8, 8, 16384)
    Ao = oracle.BVH(*c["A"], 24, 8, 8, 16384)
    Bo = oracle.BVH(*c["B"], 24, 8, 8, 16384)
    D = synth.scene_diameter(c["A"][0], c["B"][0])
    return dict(c=c, A=A, B=B, Ao=Ao, Bo=Bo, D=D)


def _keys(off, ij):
    """Pairs of a CSR as one int64 per (pose, i, j): pose << 40 | i << 20 | j."""
    off = np.asarray(off)
    ij = np.asarray(ij, dtype=np.int64).reshape(-1, 2)
    pose = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    assert (ij[:, 0] < (1 << 20)).all() and (ij[:, 1] < (1 << 20)).all()
    return (pose << 40) | (ij[:, 0] << 20) | ij[:, 1]


def test_c2_every_pose_against_oracle(cb, c2):
    """The 10,000-pose terrain workload exactly as the benchmark launches it (its poses are
    not near-contact filtered), every pose checked against the oracle.  Pairs within 1e-6 D
    of a contact decision may go either way; the rest is unique: certain = oracle pairs not
    near contact, and certain <= GPU <= oracle | near.  Poses with no near-contact pair
    must match exactly; every distance within 1e-5 D."""
    P = c2["c"]["poses"]
    n = len(P)
    res = cb.collide(c2["A"], c2["B"], _gpu(P))
    dist = cb.distance(c2["A"], c2["B"], _gpu(P)).cpu().numpy().astype(np.float64)
    hit = res.hit.cpu().numpy()
    off = res.offsets.cpu().numpy()
    ij = res.pairs.cpu().numpy()
    eps = EPS_NEAR * c2["D"]
    o_hit, o_off, o_ij, _ = oracle.collide(c2["Ao"], c2["Bo"], P)
    n_off, n_ij = oracle.near_pairs(c2["Ao"], c2["Bo"], P, eps)
    o_d, _ = oracle.distance(c2["Ao"], c2["Bo"], P)
    G, O, M = _keys(off, ij), _keys(o_off, o_ij), _keys(n_off, n_ij)
    certain = np.setdiff1d(O, M)
    allowed = np.union1d(O, M)
    missing = certain[~np.isin(certain, G)]
    extra = G[~np.isin(G, allowed)]
    assert len(missing) == 0, ("pairs the oracle finds clear of contact are missing", len(missing), missing[:5] >> 40)
    assert len(extra) == 0, ("pairs outside the oracle's and the near-contact set", len(extra), extra[:5] >> 40)
    near_pose = np.zeros(n, bool)
    near_pose[np.unique(M >> 40)] = True
    certain_pose = np.zeros(n, bool)
    certain_pose[np.unique(certain >> 40)] = True
    allowed_pose = np.zeros(n, bool)
    allowed_pose[np.unique(allowed >> 40)] = True
    assert (hit[certain_pose] == 1).all() and (hit[~allowed_pose] == 0).all()
    exact = ~near_pose
    assert (hit[exact] == o_hit[exact]).all()
    assert (np.diff(off)[exact] == np.diff(o_off)[exact]).all()
    # pose by pose on poses clear of contact: same pairs (sets equal, and sorted on both sides)
    G_ex = G[exact[G >> 40]]
    O_ex = np.sort(O[exact[O >> 40]])
    assert len(G_ex) == len(O_ex) and (G_ex == O_ex).all()
    # sorted by (i, j) inside every pose; a hit iff the pose has a pair
    assert (np.diff(G) > 0).all()
    assert ((np.diff(off) > 0) == (hit == 1)).all()
    assert np.abs(dist - o_d).max() <= TOL_PQ * c2["D"]
    # hit iff distance 0, except where CD and PQ may decide a near-contact pair differently
    bad = np.nonzero((dist == 0) != (hit == 1))[0]
    assert near_pose[bad].all() if len(bad) else True
    assert exact.sum() >= n // 4 and o_hit[exact].sum() >= 100 and (o_hit[exact] == 0).sum() >= 100


@pytest.mark.parametrize("stage,split,budget0", [(16384, 1, 16), (32768, 3, 256), (0, 0, 256), (0, 1, 256),
                                                (0, 2, 256), (16384, 2, 64), (0, 3, 16), (0, 4, 1024)])
def test_launch_options_keep_results(cb, c1, c2, stage, split, budget0):
    """Treelet staging in shared memory (TMA bulk copies), the work mapping (warp per pose,
    rounds of handed-on tasks, or one launch over a work queue with donation) and the task
    budget change how the work is scheduled, never the result."""
    import torch
    P1 = _gpu(c1["P"])
    P2 = _gpu(c2["c"]["poses"][:1500])
    ref = (cb.collide(c1["A"], c1["B"], P1), cb.distance(c1["A"], c1["B"], P1).cpu().numpy(),
           cb.collide(c2["A"], c2["B"], P2), cb.distance(c2["A"], c2["B"], P2).cpu().numpy())
    cb.set_option(cb.OPT_STAGE_BYTES, stage)
    cb.set_option(cb.OPT_SPLIT, split)
    cb.set_option(cb.OPT_BUDGET0, budget0)
    try:
        got = (cb.collide(c1["A"], c1["B"], P1), cb.distance(c1["A"], c1["B"], P1).cpu().numpy(),
               cb.collide(c2["A"], c2["B"], P2), cb.distance(c2["A"], c2["B"], P2).cpu().numpy())
    finally:
        cb.set_option(cb.OPT_STAGE_BYTES, 0)
        cb.set_option(cb.OPT_SPLIT, cb.SPLIT_DEFAULT)
        cb.set_option(cb.OPT_BUDGET0, cb.BUDGET0_DEFAULT)
    for r, g in ((ref[0], got[0]), (ref[2], got[2])):
        assert torch.equal(r.hit, g.hit) and torch.equal(r.offsets, g.offsets) and torch.equal(r.pairs, g.pairs)
    assert np.allclose(ref[1], got[1], rtol=0, atol=1e-5 * c1["D"])
    assert np.allclose(ref[3], got[3], rtol=0, atol=1e-5 * c2["D"])


def test_bottom_up_terrain_equals_top_down(cb, c2):
    """The two treelet packings give different blobs of the same tree: every collision
    result is identical and distances agree to rounding."""
    import torch
    cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_BOTTOM_UP)
    try:
        A = cb.BVH(*c2["c"]["A"], 24, 8, 8, 16384)
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
    assert A.info["node_bytes"] < c2["A"].info["node_bytes"]
    P = _gpu(c2["c"]["poses"][:2000])
    r0, r1 = cb.collide(c2["A"], c2["B"], P), cb.collide(A, c2["B"], P)
    assert torch.equal(r0.hit, r1.hit) and torch.equal(r0.offsets, r1.offsets) and torch.equal(r0.pairs, r1.pairs)
    d0, d1 = cb.distance(c2["A"], c2["B"], P).cpu().numpy(), cb.distance(A, c2["B"], P).cpu().numpy()
    assert np.abs(d0 - d1).max() <= 1e-6 * c2["D"]


def test_kernel_launch_counter(cb, c1):
    """cbvh_kernel_launches counts what a query launches: with the default mapping a collide
    with sorted pair lists is one work-queue traversal + scan, scatter and sort; a distance
    is six rounds of early-exit collision and six of branch and bound."""
    P = _gpu(c1["P"])
    n0 = cb.kernel_launches()
    cb.collide(c1["A"], c1["B"], P, capacity=1 << 20)
    n1 = cb.kernel_launches()
    cb.distance(c1["A"], c1["B"], P)
    n2 = cb.kernel_launches()
    assert n1 - n0 == 4 and n2 - n1 == 12


def test_loaded_hierarchy_answers_like_the_original(cb, c1, tmp_path):
    """cbvh_save / cbvh_load: the loaded blob is the saved one, so every query agrees."""
    A = cb.BVH.load(_save_to(c1["A"], tmp_path / "a.cbvh"))
    B = cb.BVH.load(_save_to(c1["B"], tmp_path / "b.cbvh"))
    P = _gpu(c1["P"][:128])
    r0, r1 = cb.collide(c1["A"], c1["B"], P), cb.collide(A, B, P)
    assert (r0.hit.cpu().numpy() == r1.hit.cpu().numpy()).all()
    assert (r0.offsets.cpu().numpy() == r1.offsets.cpu().numpy()).all()
    assert (r0.pairs.cpu().numpy() == r1.pairs.cpu().numpy()).all()
    assert (cb.distance(c1["A"], c1["B"], P).cpu().numpy() == cb.distance(A, B, P).cpu().numpy()).all()


def _save_to(h, path):
    h.save(str(path))
    return str(path)
