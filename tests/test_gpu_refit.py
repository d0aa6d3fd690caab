"""Device refit for deforming meshes (cbvh_refit): the tree is kept and every bound is
recomputed on the GPU.  The refitted blob must equal, byte for byte, the FP64 oracle's
refit of the same tree with the same new vertices (or_refit: exact rational lattice bounds,
its own encoder), in every storage mode and treelet packing; queries on the refitted
hierarchy match the oracle; bad vertices are reported, not used.  Hierarchies meant for
refits are built with lattice headroom (CBVH_OPT_LATTICE_HEADROOM) so that a mesh whose
extent grows still fits the build's lattice."""
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


def _deform(v, seed, amp=0.08):
    """A smooth deformation: every vertex moved by a few sine waves of its position."""
    rng = np.random.default_rng(seed)
    k = rng.normal(size=(3, 3)) * 2.0
    ph = rng.uniform(0, 2 * np.pi, size=3)
    w = np.sin(np.asarray(v, np.float64) @ k + ph)
    return (v + amp * w).astype(np.float32)


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


MESHES = {"sphere": lambda: synth.icosphere(3, 1.0, 0.15, seed=9),
          "terrain": lambda: synth.heightfield(48, 4.0, seed=4)[:2]}


@pytest.mark.parametrize("packing", [0, 1])
@pytest.mark.parametrize("k,m,bits,tb", [(18, 4, 8, 4096), (24, 8, 16, 16384), (18, 4, 1, 4096), (24, 8, 0, 8192)])
@pytest.mark.parametrize("mesh", ["sphere", "terrain"])
def test_refit_blob_equals_oracle_refit(cb, mesh, k, m, bits, tb, packing):
    v, t = MESHES[mesh]()
    cb.set_option(cb.OPT_TREELET_PACKING, packing)
    cb.set_option(cb.OPT_LATTICE_HEADROOM, 2)  # room for the deformed mesh's larger extent
    try:
        h = cb.BVH(v, t, k, m, bits, tb)
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
        cb.set_option(cb.OPT_LATTICE_HEADROOM, 0)
    o = oracle.BVH(v, t, k, m, bits, tb, packing=packing, headroom=2)
    assert (h.blob_dev.cpu().numpy() == o.blob()).all()
    T = _dev(t)
    for seed in (1, 2):
        v2 = _deform(v, seed)
        h.refit(_dev(v2), T)
        o.refit(v2)
        got = h.blob_dev.cpu().numpy()
        want = o.blob()
        assert got.shape == want.shape
        assert (got == want).all(), int((got != want).sum())
    h.refit(_dev(v), T)  # back to the build's vertices: the build's blob again
    assert (h.blob_dev.cpu().numpy() == h.blob_host()).all()


def test_queries_after_refit_match_oracle(cb):
    c = synth.C1(4)
    (va, ta), (vb, tb) = c["A"], c["B"]
    cb.set_option(cb.OPT_LATTICE_HEADROOM, 1)
    try:
        A = cb.BVH(va, ta, 18, 4, 16, 4096)
        B = cb.BVH(vb, tb, 18, 4, 16, 4096)
    finally:
        cb.set_option(cb.OPT_LATTICE_HEADROOM, 0)
    va2, vb2 = _deform(va, 3, 0.1), _deform(vb, 4, 0.1)
    A.refit(_dev(va2), _dev(ta))
    B.refit(_dev(vb2), _dev(tb))
    Ao = oracle.BVH(va, ta, 18, 4, 16, 4096, headroom=1)
    Bo = oracle.BVH(vb, tb, 18, 4, 16, 4096, headroom=1)
    Ao.refit(va2)
    Bo.refit(vb2)
    D = synth.scene_diameter(va2, vb2)
    P = oracle.filtered_poses(Ao, Bo, lambda cnt, r: synth.poses_box(cnt, seed=2001 + 31 * r), 128, 1e-6 * D)
    res = cb.collide(A, B, _dev(P))
    o_hit, o_off, o_ij, _ = oracle.collide(Ao, Bo, P)
    assert (res.hit.cpu().numpy() == o_hit).all()
    assert (res.offsets.cpu().numpy() == o_off).all() and (res.pairs.cpu().numpy() == o_ij).all()
    o_d, _ = oracle.distance(Ao, Bo, P)
    d = cb.distance(A, B, _dev(P)).cpu().numpy()
    assert np.abs(d - o_d).max() <= 1e-5 * D
    assert o_hit.sum() > 10 and (o_hit == 0).sum() > 10


def test_refit_reports_bad_vertices(cb):
    v, t = synth.icosphere(2, 1.0, 0.1, seed=2)
    h = cb.BVH(v, t, 18, 4, 8, 4096)
    T = _dev(t)
    bad = v.copy()
    bad[3, 1] = np.nan
    with pytest.raises(cb.CbvhError):
        h.refit(_dev(bad), T)
    with pytest.raises(cb.CbvhError):
        h.refit(_dev(v * 4096.0), T)  # beyond the build's lattice range
    cb.set_option(cb.OPT_LATTICE_HEADROOM, 1)
    try:
        h16 = cb.BVH(v * 30000.0, t, 18, 4, 1, 4096)  # FP16: inside +-65504 at build time ...
    finally:
        cb.set_option(cb.OPT_LATTICE_HEADROOM, 0)
    with pytest.raises(cb.CbvhError):
        h16.refit(_dev(v * 45000.0), T)  # ... not after (the lattice itself has room)
    h.refit(_dev(v), T)  # a good refit afterwards restores the build's blob
    assert (h.blob_dev.cpu().numpy() == h.blob_host()).all()
    hs = cb.BVH(v, t, 18, 4, 2, 4096)  # Stream VByte: record sizes follow the deltas
    with pytest.raises(cb.CbvhError) as e:
        hs.refit(_dev(v), T)
    assert e.value.code == -1
