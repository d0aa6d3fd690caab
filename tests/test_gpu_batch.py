"""Batched queries (cbvh_batch_*) on the GPU.

- Every item of a mixed batch (different pairs of hierarchies, collision with and without
  early exit, distances) returns exactly what the same query returns on its own.
- The batch launch can be captured in a CUDA graph; replays reproduce the direct results,
  with every scheduler (rounds of handed-on tasks, one launch over a work queue, or
  rounds ending in a work-queue round).
- A reduced arm-against-clutter sweep, and 1,000 configurations against the full clutter,
  agree with the FP64 oracle on poses away from contact.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


@pytest.fixture(scope="module")
def scene(cb):
    import torch
    c1 = synth.C1(300)
    (va, ta), (vb, tb) = c1["A"], c1["B"]
    S1 = cb.BVH(va, ta, 18, 4, 16, 4096)
    S2 = cb.BVH(vb, tb, 18, 4, 16, 4096)
    S3 = cb.BVH(vb, tb, 18, 8, 8, 16384)   # a second B, different branching
    c3 = synth.C3(400, n_boxes=30, n_spheres=30)
    clutter = cb.BVH(*c3["A"], 24, 8, 8, 16384)
    links = [cb.BVH(*l, 24, 8, 8, 16384) for l in c3["links"]]
    P1 = torch.as_tensor(c1["poses"], device="cuda")
    LP = [torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:, i]), device="cuda") for i in range(6)]
    return dict(S1=S1, S2=S2, S3=S3, P1=P1, clutter=clutter, links=links, LP=LP, c3=c3, c1=c1)


def _items(sc):
    it = [dict(A=sc["S1"], B=sc["S2"], kind="collide", poses=sc["P1"]),
          dict(A=sc["S1"], B=sc["S3"], kind="collide", poses=sc["P1"][:137], early_exit=True),
          dict(A=sc["S1"], B=sc["S2"], kind="distance", poses=sc["P1"][:211]),
          dict(A=sc["S1"], B=sc["S3"], kind="distance", poses=sc["P1"][50:90])]
    for i, (L, P) in enumerate(zip(sc["links"], sc["LP"])):
        it.append(dict(A=sc["clutter"], B=L, kind="collide", poses=P, early_exit=True))
    it.append(dict(A=sc["clutter"], B=sc["links"][3], kind="distance", poses=sc["LP"][3][:100]))
    return it


def _alone(cb, it):
    if it["kind"] == "collide":
        return cb.collide(it["A"], it["B"], it["poses"], pairs=False, early_exit=bool(it.get("early_exit"))).hit
    return cb.distance(it["A"], it["B"], it["poses"])


def test_batch_items_equal_single_queries(cb, scene):
    items = _items(scene)
    batch = cb.Batch(items)
    outs = batch.run()
    for it, out in zip(items, outs):
        ref = _alone(cb, it).cpu().numpy()
        got = out.cpu().numpy()
        if it["kind"] == "collide":
            assert (got == ref).all()
        else:
            # the visiting order differs between the two launches, so a pruned pair whose FP32
            # distance lies within rounding of its lower bound may change the last ulps
            assert np.allclose(got, ref, rtol=0, atol=1e-5 * 8.0)
    hits = np.stack([o.cpu().numpy() for o in outs[4:10]])
    assert 0 < hits.any(0).sum() < hits.shape[1]  # some configurations collide, some do not


@pytest.mark.parametrize("split", [1, 2, 3, 4])
def test_batch_graph_capture_and_replay(cb, scene, split):
    cb.set_option(cb.OPT_SPLIT, split)
    try:
        _graph_replay(cb, scene)
    finally:
        cb.set_option(cb.OPT_SPLIT, cb.SPLIT_DEFAULT)


def _graph_replay(cb, scene):
    import torch
    items = _items(scene)
    batch = cb.Batch(items)
    direct = [o.clone() for o in batch.run()]
    for o in batch.outputs:
        o.fill_(77)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        batch.launch(stream)  # warm the launch path outside capture
    torch.cuda.current_stream().wait_stream(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.launch()
    for _ in range(2):
        for o in batch.outputs:
            o.fill_(77)
        g.replay()
        torch.cuda.synchronize()
        assert int(batch.status.item()) == 0
        for it, a, b in zip(items, direct, batch.outputs):
            if it["kind"] == "collide":
                assert torch.equal(a, b)
            else:  # branch-and-bound visiting order may move the last ulps
                assert torch.allclose(a, b, rtol=0, atol=1e-5 * 8.0)


def test_arm_sweep_against_oracle(cb, scene):
    c3 = scene["c3"]
    A = oracle.BVH(*c3["A"], 24, 8, 8, 16384)
    items = [dict(A=scene["clutter"], B=L, kind="collide", poses=P) for L, P in zip(scene["links"], scene["LP"])]
    outs = [o.cpu().numpy() for o in cb.Batch(items).run()]
    va = c3["A"][0]
    checked = 0
    for i, (v, t) in enumerate(c3["links"]):
        B = oracle.BVH(v, t, 24, 8, 8, 16384)
        P = c3["link_poses"][:60, i]
        D = synth.scene_diameter(va, v)
        near, _ = oracle.near_contact(A, B, P, 1e-6 * D)
        hit, *_ = oracle.collide(A, B, P)
        ok = ~near
        assert (outs[i][:60][ok] == hit[ok]).all()
        checked += int(ok.sum())
    assert checked > 200


@pytest.mark.parametrize("m,tb", [(8, 16384), (16, 4096)])
def test_arm_sweep_full_clutter_against_oracle(cb, m, tb):
    """The sweep as the benchmark runs it: the full 1,026,400-triangle clutter, 1,000
    configurations x 6 links in one batch with early-exit collision, at the default
    hierarchy (branching 8, 16 KB treelets) and at the one the autotuner picks on the box
    (branching 16, 4 KB).  Flags equal the oracle's on every link pose away from contact,
    and so does each configuration's answer (any link in collision) where all six are."""
    import torch
    n = 1000
    c3 = synth.C3(n)
    va = c3["A"][0]
    clutter = cb.BVH(*c3["A"], 24, m, 8, tb)
    links = [cb.BVH(*l, 24, m, 8, tb) for l in c3["links"]]
    LP = [torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:, i]), device="cuda") for i in range(6)]
    items = [dict(A=clutter, B=L, kind="collide", poses=P, early_exit=True) for L, P in zip(links, LP)]
    outs = np.stack([o.cpu().numpy() for o in cb.Batch(items).run()])
    A = oracle.BVH(*c3["A"], 24, 8, 8, 16384)
    o_hit = np.zeros((6, n), np.uint8)
    near = np.zeros((6, n), bool)
    for i, (v, t) in enumerate(c3["links"]):
        B = oracle.BVH(v, t, 24, 8, 8, 16384)
        P = c3["link_poses"][:, i]
        near[i], _ = oracle.near_contact(A, B, P, 1e-6 * synth.scene_diameter(va, v))
        o_hit[i], *_ = oracle.collide(A, B, P)
    ok = ~near
    assert (outs[ok] == o_hit[ok]).all(), np.argwhere((outs != o_hit) & ok)[:10]
    all_clear = ok.all(0)
    assert (outs.any(0)[all_clear] == o_hit.any(0)[all_clear]).all()
    assert ok.sum() >= 3000 and o_hit[ok].sum() >= 500 and (o_hit[ok] == 0).sum() >= 1000
    # the links as one configuration set: each configuration stops at its first colliding
    # link, and the set's flag is the configuration's answer
    sets = [dict(it, set="arm") for it in items]
    batch = cb.Batch(sets)
    for _ in range(2):  # the launch clears the set's flags: a second launch answers the same
        souts = np.stack([o.cpu().numpy() for o in batch.run()])
        anyh = batch.any_hit["arm"].cpu().numpy()
        certain = (o_hit.astype(bool) & ok).any(0)
        assert anyh[certain].all()
        assert (anyh[all_clear] == o_hit.any(0)[all_clear]).all()
        assert ((souts == 1) & ok <= (o_hit == 1)).all()  # an item's 1 is a real intersection
        assert ((souts.any(0) == anyh.astype(bool))).all()
        assert souts.sum() < outs.sum()  # configurations stopped at their first colliding link


def test_distance_sets_against_oracle(cb, scene):
    """The arm's clearance: distance items of the six links as one configuration set share
    the configuration's best distance.  The set's minimum equals the smallest of the
    oracle's per-link distances within 1e-5 D, and every item's own output is at least its
    oracle distance (an upper bound, exact where it is the set's minimum); two launches in a
    row give the same minima."""
    import torch
    c3 = scene["c3"]
    n = 60
    LP = [torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:n, i]), device="cuda") for i in range(6)]
    items = [dict(A=scene["clutter"], B=L, kind="distance", poses=P, set="arm") for L, P in zip(scene["links"], LP)]
    batch = cb.Batch(items)
    va = c3["A"][0]
    A = oracle.BVH(*c3["A"], 24, 8, 8, 16384)
    o_d = []
    D = 0.0
    for i, (v, t) in enumerate(c3["links"]):
        B = oracle.BVH(v, t, 24, 8, 8, 16384)
        o_d.append(oracle.distance(A, B, c3["link_poses"][:n, i])[0])
        D = max(D, synth.scene_diameter(va, v))
    o_d = np.stack(o_d)
    for _ in range(2):
        outs = np.stack([o.cpu().numpy() for o in batch.run()]).astype(np.float64)
        mind = batch.min_dist["arm"].cpu().numpy().astype(np.float64)
        assert np.abs(mind - o_d.min(0)).max() <= 1e-5 * D
        assert (outs >= o_d - 1e-5 * D).all()
        assert np.allclose(outs.min(0), mind, rtol=0, atol=1e-5 * D)
    assert (o_d.min(0) > 0).sum() >= 5


def test_arm_self_collision_against_oracle(cb, scene):
    """Self-collision of the arm: every non-adjacent link pair, link j posed in link i's
    frame, all in one batch; flags match the oracle on configurations away from contact."""
    c3 = scene["c3"]
    pairs = synth.self_pairs(6)
    n = 80
    rel = {(i, j): synth.relative_poses(c3["link_poses"][:n], i, j) for i, j in pairs}
    import torch
    items = [dict(A=scene["links"][i], B=scene["links"][j], kind="collide",
                  poses=torch.as_tensor(rel[i, j], device="cuda"), early_exit=True) for i, j in pairs]
    outs = [o.cpu().numpy() for o in cb.Batch(items).run()]
    checked = 0
    for (i, j), got in zip(pairs, outs):
        vi, ti = c3["links"][i]
        vj, tj = c3["links"][j]
        Ao = oracle.BVH(vi, ti, 24, 8, 8, 16384)
        Bo = oracle.BVH(vj, tj, 24, 8, 8, 16384)
        D = synth.scene_diameter(vi, vj)
        near, _ = oracle.near_contact(Ao, Bo, rel[i, j], 1e-6 * D)
        hit, *_ = oracle.collide(Ao, Bo, rel[i, j])
        assert (got[~near] == hit[~near]).all(), (i, j)
        checked += int((~near).sum())
    assert checked > 600
    hits = np.stack(outs).any(0)
    assert 0 < hits.sum() < n  # some configurations fold onto themselves, some do not
    # the ten link pairs as one configuration set: the set's flag is the configuration's
    # answer (some pair of links intersects), equal to the pairs' flags taken one by one
    sb = cb.Batch([dict(it, set="self") for it in items])
    sb.run()
    assert (sb.any_hit["self"].cpu().numpy().astype(bool) == hits).all()
    # validity: the links against the clutter and the link pairs against each other in one
    # set; the answer is the OR of both, each computed on its own
    env = [dict(A=scene["clutter"], B=scene["links"][i], kind="collide", early_exit=True,
                poses=torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:n, i]), device="cuda")) for i in range(6)]
    env_hits = np.stack([o.cpu().numpy() for o in cb.Batch(env).run()]).any(0)
    vb = cb.Batch([dict(it, set="valid") for it in env + items])
    vb.run()
    assert (vb.any_hit["valid"].cpu().numpy().astype(bool) == (env_hits | hits)).all()


def test_batch_refuses_stream_vbyte_hierarchies(cb, scene):
    """Stream VByte records vary in size; the batched kernels are compiled for fixed-size
    records only, so a batch with such a hierarchy is refused before anything launches,
    while the same hierarchy answers single queries."""
    c1 = scene["c1"]
    (va, ta), (vb, tb) = c1["A"], c1["B"]
    A = cb.BVH(va, ta, 18, 4, cb.QUANT_SVB, 4096)
    P = scene["P1"][:64]
    with pytest.raises(cb.CbvhError) as e:
        cb.Batch([dict(A=A, B=scene["S2"], kind="collide", poses=P)])
    assert e.value.code == -1
    want = cb.collide(scene["S1"], scene["S2"], P, pairs=False).hit.cpu().numpy()
    assert (cb.collide(A, scene["S2"], P, pairs=False).hit.cpu().numpy() == want).all()
