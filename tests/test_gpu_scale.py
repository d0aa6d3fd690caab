"""The scale-and-compression workload: a field of fractal-displaced spheres probed by a
displaced sphere, with bottom-up packed treelets at 8 and 16 bits and with FP32 bounds.

- A reduced field (6 level-4 spheres in a 6 m cube, level-3 probe) against the FP64 oracle
  in full: collision bit-exact on poses away from contact, distances within 1e-5 of the
  scene diameter, for every compression setting.
- The full field (32 level-7 spheres, 1,000,000 poses) at the benchmark's launch
  configuration, checked by the oracle on 1,000 flags, 100 pair lists and 200 distances.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_PQ = 1e-5
EPS_NEAR = 1e-6


@pytest.fixture(scope="module")
def cb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    m.set_option(m.OPT_TREELET_PACKING, m.PACK_BOTTOM_UP)
    yield m
    m.set_option(m.OPT_TREELET_PACKING, m.PACK_TOP_DOWN)


@pytest.fixture(scope="module")
def field(cb):
    c = synth.C5(1, n_spheres=6, level=4, probe_level=3, half=3.0)
    (va, ta), (vb, tb) = c["A"], c["B"]
    Ao = oracle.BVH(va, ta, 18, 4, 8, 16384, packing=oracle.PACKING_BOTTOM_UP)
    Bo = oracle.BVH(vb, tb, 18, 4, 8, 16384, packing=oracle.PACKING_BOTTOM_UP)
    D = synth.scene_diameter(va, vb)
    P = oracle.filtered_poses(Ao, Bo, lambda cnt, r: synth.poses_box(cnt, seed=2005 + 7919 * r, lo=-3.0, hi=3.0),
                              384, EPS_NEAR * D)
    return dict(mesh=(va, ta, vb, tb), Ao=Ao, Bo=Bo, D=D, P=P)


@pytest.mark.parametrize("bits,tb", [(8, 16384), (16, 16384), (0, 16384), (1, 16384), (8, 131072), (16, 65536),
                                     (2, 16384)])
def test_reduced_field_against_oracle(cb, field, bits, tb):
    import torch
    va, ta, vb, tb_ = field["mesh"]
    A = cb.BVH(va, ta, 18, 4, bits, tb)
    B = cb.BVH(vb, tb_, 18, 4, bits, tb)
    P = field["P"]
    Pd = torch.as_tensor(P, device="cuda")
    o_hit, o_off, o_ij, _ = oracle.collide(field["Ao"], field["Bo"], P)
    assert o_hit.sum() > 10 and (o_hit == 0).sum() > 10
    r = cb.collide(A, B, Pd)
    assert (r.hit.cpu().numpy() == o_hit).all()
    assert (r.offsets.cpu().numpy() == o_off).all()
    assert (r.pairs.cpu().numpy() == o_ij).all()
    o_d, _ = oracle.distance(field["Ao"], field["Bo"], P)
    d = cb.distance(A, B, Pd).cpu().numpy()
    assert np.abs(d - o_d).max() <= TOL_PQ * field["D"]
    assert ((d == 0) == (o_d == 0)).all()


def _pairs_by_pose(off, ij):
    return [ij[off[p]:off[p + 1]] for p in range(len(off) - 1)]


def test_full_field_sampled_against_oracle(cb):
    """The full 10,485,760-triangle field in the benchmark's launch configuration (8-bit,
    16 KB bottom-up treelets): flags for all 1,000,000 poses, pair lists for the first
    100,000, distances for the first 20,000.  The oracle checks 1,000 flags drawn from all
    1,000,000 poses (poses away from contact), 100 pair lists (near-contact pairs compared as
    a set: certain <= GPU <= certain | ambiguous) and 200 distances one by one."""
    import torch
    c = synth.C5(1_000_000)
    (va, ta), (vb, tb) = c["A"], c["B"]
    A = cb.BVH(va, ta, 18, 4, 8, 16384)
    B = cb.BVH(vb, tb, 18, 4, 8, 16384)
    P = c["poses"]
    Pd = torch.as_tensor(P, device="cuda")
    flags = cb.collide(A, B, Pd, pairs=False).hit.cpu().numpy()
    res = cb.collide(A, B, Pd[:100_000], capacity=250_000_000)
    hit = res.hit.cpu().numpy()
    pairs = _pairs_by_pose(res.offsets.cpu().numpy(), res.pairs.cpu().numpy())
    dist = cb.distance(A, B, Pd[:20_000]).cpu().numpy()
    assert (flags[:100_000] == hit).all()
    # every pose's list sorted by (i, j), strictly: long lists (thousands of pairs) take the
    # sort's merge passes
    off = res.offsets.cpu().numpy()
    ij = res.pairs.cpu().numpy().astype(np.int64)
    keys = (ij[:, 0] << 32) | ij[:, 1]
    inner = np.ones(len(keys) - 1, bool)
    inner[off[1:-1][(off[1:-1] > 0) & (off[1:-1] < len(keys))] - 1] = False
    assert (np.diff(keys)[inner] > 0).all()
    assert np.diff(off).max() > 4 * 4096
    del res
    Ao = oracle.BVH(va, ta, 18, 4, 8, 16384, packing=oracle.PACKING_BOTTOM_UP)
    Bo = oracle.BVH(vb, tb, 18, 4, 8, 16384, packing=oracle.PACKING_BOTTOM_UP)
    D = synth.scene_diameter(va, vb)
    eps = EPS_NEAR * D
    rng = np.random.default_rng(7)
    # pair lists: 100 poses of the first 100,000
    idx = np.sort(rng.choice(100_000, 100, replace=False))
    o_hit, o_off, o_ij, _ = oracle.collide(Ao, Bo, P[idx])
    o_pairs = _pairs_by_pose(o_off, o_ij)
    n_off, n_ij = oracle.near_pairs(Ao, Bo, P[idx], eps)
    amb = _pairs_by_pose(n_off, n_ij)
    key = lambda a: set(map(tuple, np.asarray(a).tolist()))  # noqa: E731
    exact = 0
    for q, p in enumerate(idx):
        gpu, ora, am = key(pairs[p]), key(o_pairs[q]), key(amb[q])
        certain = ora - am
        assert certain <= gpu <= (ora | am), (p, len(certain - gpu), len(gpu - (ora | am)))
        if not am:
            exact += 1
            assert gpu == ora and hit[p] == o_hit[q]
    assert exact >= 50 and o_hit.sum() >= 5
    # distances: 200 poses of the first 20,000
    idd = np.sort(rng.choice(20_000, 200, replace=False))
    o_d, _ = oracle.distance(Ao, Bo, P[idd])
    assert np.abs(dist[idd] - o_d).max() <= TOL_PQ * D
    assert (o_d == 0).sum() >= 5 and (o_d > 0).sum() >= 100
    # flags: 1,000 poses drawn from all 1,000,000.  Almost every intersecting pose of this
    # field has some pair near contact, so flags are judged by the pair sets: a pose with an
    # intersecting pair clear of contact must be flagged, a pose with neither an
    # intersecting nor a near-contact pair must not; poses with no near pair match exactly.
    far = np.sort(rng.choice(1_000_000, 1000, replace=False))
    f_hit, f_off, f_ij, _ = oracle.collide(Ao, Bo, P[far])
    m_off, m_ij = oracle.near_pairs(Ao, Bo, P[far], eps)
    for q in range(len(far)):
        ora, am = key(f_ij[f_off[q]:f_off[q + 1]]), key(m_ij[m_off[q]:m_off[q + 1]])
        if ora - am:
            assert flags[far[q]] == 1, far[q]
        if not (ora | am):
            assert flags[far[q]] == 0, far[q]
        if not am:
            assert flags[far[q]] == f_hit[q], far[q]
    has_near = np.diff(m_off) > 0
    assert (~has_near).sum() >= 700 and f_hit.sum() >= 100 and (f_hit[~has_near] == 0).sum() >= 500
