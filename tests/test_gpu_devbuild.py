"""Device-side build (cbvh_build_plan + cbvh_build_device): the blob built on the GPU from a
device mesh must equal, byte for byte, the FP64 oracle's build of the same mesh (its own
median split, exact rational lattice and encoder) in every storage mode, branching, k,
treelet packing and lattice headroom -- including meshes whose centroids tie (a grid
terrain), signed zeros, a ragged triangle count, one triangle, extreme scales and the
full-size terrain.  A plan rebuilt with another mesh of the same size (a new frame) gives
that mesh's blob; bad meshes are refused with the host build's error, and the handle then
refuses queries until a good build."""
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


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _signed_zero_terrain():
    v, t = synth.heightfield(20, 4.0, seed=6)[:2]
    v = v.copy()
    v[v == 0.0] = -0.0  # the grid's zero coordinates as negative zeros: they tie with +0
    v[::7, 2] = 0.0
    return v, t


def _box_corner(shift):
    """A unit box moved so that its largest |d.v| is a power of two (shift 0.5: every
    coordinate 0 or 1) or just below one (shift 0.5 - 2^-24: the far corner at 1 - 2^-24),
    where the exponent search must decide exactly at the threshold."""
    v, t = synth.box_mesh((1.0, 1.0, 1.0))
    return (v.astype(np.float64) + shift).astype(np.float32), t


MESHES = {
    "sphere": lambda: synth.icosphere(3, 1.0, 0.15, seed=9),
    "box_pow2": lambda: _box_corner(0.5),
    "box_below_pow2": lambda: _box_corner(0.5 - 2.0 ** -24),
    "terrain": lambda: synth.heightfield(32, 4.0, seed=4)[:2],
    "signed_zero": _signed_zero_terrain,
    "ragged_unused": lambda: (synth.icosphere(3, 1.0, 0.15, seed=3)[0], synth.icosphere(3, 1.0, 0.15, seed=3)[1][:1111]),
    "one": lambda: (synth.icosphere(1)[0], synth.icosphere(1)[1][:1]),
    "three": lambda: (synth.icosphere(1)[0], synth.icosphere(1)[1][5:8]),
    "tiny_scale": lambda: ((synth.icosphere(2, 1.0, 0.1, seed=1)[0] * np.float32(1e-25)).astype(np.float32),
                           synth.icosphere(2, 1.0, 0.1, seed=1)[1]),
    "huge_scale": lambda: ((synth.icosphere(2, 1.0, 0.1, seed=1)[0] * np.float32(3e20)).astype(np.float32),
                           synth.icosphere(2, 1.0, 0.1, seed=1)[1]),
}
CONFIGS = [(18, 4, 16, 4096, 0, 0), (24, 8, 8, 16384, 1, 0), (6, 2, 8, 4096, 0, 0), (26, 16, 1, 8192, 0, 0),
           (24, 8, 0, 8192, 1, 2), (18, 4, 8, 4096, 0, 3)]


def _device_build(cb, v, t, k, m, bits, tb, packing, headroom, host_copy=True):
    cb.set_option(cb.OPT_TREELET_PACKING, packing)
    cb.set_option(cb.OPT_LATTICE_HEADROOM, headroom)
    try:
        return cb.BVH.on_device(_dev(v), _dev(t), k, m, bits, tb, host_copy=host_copy)
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
        cb.set_option(cb.OPT_LATTICE_HEADROOM, 0)


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "k%d_m%d_b%d_tb%d_p%d_h%d" % c)
@pytest.mark.parametrize("mesh", list(MESHES))
def test_device_build_equals_oracle(cb, mesh, cfg):
    v, t = MESHES[mesh]()
    k, m, bits, tb, packing, headroom = cfg
    if bits == 1 and mesh == "huge_scale":
        pytest.skip("beyond the half-precision range (covered by the error test)")
    o = oracle.BVH(v, t, k, m, bits, tb, packing=packing, headroom=headroom)
    h = _device_build(cb, v, t, k, m, bits, tb, packing, headroom)
    want = o.blob()
    got = h.blob_dev.cpu().numpy()
    assert got.shape == want.shape
    assert (got == want).all(), int((got != want).sum())
    assert (h.blob_host() == want).all()  # the host copy came back
    assert h.info["lattice_exp"] == o.e


def test_device_build_full_terrain(cb):
    """The 512 x 512 terrain (524,288 triangles, many tied centroids): many tiles in every
    sort pass and prefix sum, 19 split rounds."""
    v, t = synth.heightfield(512, 4.0, seed=1002)[:2]
    o = oracle.BVH(v, t, 24, 8, 8, 16384)
    h = _device_build(cb, v, t, 24, 8, 8, 16384, 0, 0, host_copy=False)
    assert (h.blob_dev.cpu().numpy() == o.blob()).all()
    with pytest.raises(cb.CbvhError) as e:
        h.blob_host()  # not copied back
    assert e.value.code == -9


def test_new_frame_on_the_same_plan(cb):
    """A second mesh of the same counts with another topology and vertex order."""
    v1, t1 = synth.icosphere(3, 1.0, 0.15, seed=9)
    v2, t2 = synth.icosphere(3, 1.7, 0.3, seed=21)
    rng = np.random.default_rng(8)
    pv = rng.permutation(len(v2))
    inv = np.empty_like(pv)
    inv[pv] = np.arange(len(pv))
    v2 = v2[pv]
    t2 = inv[t2][rng.permutation(len(t2))].astype(np.int32)
    h = cb.BVH.plan(len(v1), len(t1), 24, 8, 16, 4096)
    for v, t in ((v1, t1), (v2, t2), (v1, t1)):
        h.build_device(_dev(v), _dev(t))
        assert (h.blob_dev.cpu().numpy() == oracle.BVH(v, t, 24, 8, 16, 4096).blob()).all()


def test_queries_on_device_built_hierarchies(cb):
    c = synth.C1(4)
    (va, ta), (vb, tb) = c["A"], c["B"]
    A = cb.BVH.on_device(_dev(va), _dev(ta), 18, 4, 16, 4096)
    B = cb.BVH.on_device(_dev(vb), _dev(tb), 18, 4, 16, 4096)
    Ao = oracle.BVH(va, ta, 18, 4, 16, 4096)
    Bo = oracle.BVH(vb, tb, 18, 4, 16, 4096)
    D = synth.scene_diameter(va, vb)
    P = oracle.filtered_poses(Ao, Bo, lambda cnt, r: synth.poses_box(cnt, seed=2001 + 31 * r), 128, 1e-6 * D)
    res = cb.collide(A, B, _dev(P))
    o_hit, o_off, o_ij, _ = oracle.collide(Ao, Bo, P)
    assert (res.hit.cpu().numpy() == o_hit).all()
    assert (res.offsets.cpu().numpy() == o_off).all() and (res.pairs.cpu().numpy() == o_ij).all()
    o_d, _ = oracle.distance(Ao, Bo, P)
    assert np.abs(cb.distance(A, B, _dev(P)).cpu().numpy() - o_d).max() <= 1e-5 * D


def test_refit_after_device_build(cb):
    v, t = synth.icosphere(3, 1.0, 0.15, seed=9)
    h = _device_build(cb, v, t, 18, 4, 8, 4096, 0, 2)
    o = oracle.BVH(v, t, 18, 4, 8, 4096, headroom=2)
    rng = np.random.default_rng(2)
    v2 = (v * (1.0 + 0.2 * rng.random((1, 3)))).astype(np.float32)
    h.refit(_dev(v2), _dev(t))  # the build's workspace already holds the refit plan
    o.refit(v2)
    assert (h.blob_dev.cpu().numpy() == o.blob()).all()


def test_device_build_errors(cb):
    v, t = synth.icosphere(2, 1.0, 0.1, seed=2)
    h = cb.BVH.plan(len(v), len(t), 18, 4, 8, 4096)
    probe = cb.BVH(v, t, 18, 4, 8, 4096)
    P = _dev(synth.poses_box(4, seed=3))

    def refused(vv, tt, bits_plan=None):
        hh = h if bits_plan is None else bits_plan
        with pytest.raises(cb.CbvhError) as e:
            hh.build_device(_dev(vv), _dev(tt))
        assert e.value.code == -2
        with pytest.raises(cb.CbvhError) as e:  # no geometry until a good build
            cb.collide(hh, probe, P)
        assert e.value.code == -9

    bad = t.copy()
    bad[5] = (bad[5][0], bad[5][0], bad[5][1])
    refused(v, bad)  # zero-area triangle
    bad = t.copy()
    bad[7, 2] = len(v)
    refused(v, bad)  # index out of range
    bad = v.copy()
    bad[11, 0] = np.nan
    refused(bad, t)  # non-finite vertex
    bad = v.copy()
    bad[3, 1] = np.inf
    refused(bad, t)
    refused((v * np.float32(1e-30)).astype(np.float32), t)  # lattice exponent below its range
    h16 = cb.BVH.plan(len(v), len(t), 18, 4, 1, 4096)
    refused((v * 70000.0).astype(np.float32), t, h16)  # beyond the half range
    h.build_device(_dev(v), _dev(t))  # a good build afterwards
    assert (h.blob_dev.cpu().numpy() == probe.blob_host()).all()
    assert cb.collide(h, probe, P).hit.shape[0] == 4
    with pytest.raises(ValueError):
        h.build_device(_dev(v[:-1]), _dev(t))  # the plan's vertex count


def test_device_build_counts_launches(cb):
    v, t = synth.icosphere(2, 1.0, 0.1, seed=2)
    h = cb.BVH.plan(len(v), len(t), 18, 4, 8, 4096)
    n0 = cb.kernel_launches()
    h.build_device(_dev(v), _dev(t))
    assert cb.kernel_launches() - n0 > 20
