"""Host side of the device build (CPU): cbvh_build_plan lays out the tree's shape from the
triangle count alone.  Its blob must carry exactly the host build's structure -- header,
treelet offsets and every record's topology words -- with zero bounds, a zero triangle
table and lattice exponent 0, for any mesh of that size: the median split (Sec. III)
halves every node's triangles log2(branching) times, so the geometry cannot move a node
boundary.  Argument checks and state errors come before any CUDA call."""
import ctypes as C

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def cb():
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


def _structure(blob):
    """(blob with every bound field, the triangle table and the exponent zeroed, record count)."""
    b = blob.copy()
    hdr = b[:64].view(np.uint32)
    n_treelets, rec, root = int(hdr[6]), int(hdr[7]), int(hdr[8])
    off_tris = int(b[48:56].view(np.uint64)[0])
    toff = b[64:64 + 8 * (n_treelets + 1)].view(np.uint64)
    records = 0
    for t in range(n_treelets):
        o = int(toff[t])
        count = int(b[o:o + 4].view(np.uint32)[0])
        r = o + 16
        for i in range(count):
            size = root if i == 0 else rec
            b[r + 8:r + size] = 0
            r += size
            records += 1
    b[off_tris:] = 0
    b[12:16] = 0
    return b, records


def _host_blob(cb, v, t, k, m, bits, tb):
    return cb.BVH(v, t, k, m, bits, tb, device=None).blob_host()


def _plan_blob(cb, nv, nt, k, m, bits, tb):
    h = cb.BVH.plan(nv, nt, k, m, bits, tb, device=None)
    return h.blob_host(), h


MESHES = {
    "sphere": lambda: synth.icosphere(3, 1.0, 0.15, seed=9),
    "terrain": lambda: synth.heightfield(24, 4.0, seed=4)[:2],
    "ragged": lambda: (synth.icosphere(3, 1.0, 0.15, seed=3)[0], synth.icosphere(3, 1.0, 0.15, seed=3)[1][:777]),
    "one": lambda: (synth.icosphere(1)[0], synth.icosphere(1)[1][:1]),
}


@pytest.mark.parametrize("packing", [0, 1])
@pytest.mark.parametrize("k,m,bits,tb", [(18, 4, 16, 4096), (24, 8, 8, 16384), (6, 2, 8, 4096), (26, 16, 1, 8192),
                                         (24, 8, 0, 8192)])
@pytest.mark.parametrize("mesh", list(MESHES))
def test_plan_is_the_host_build_shape(cb, mesh, k, m, bits, tb, packing):
    v, t = MESHES[mesh]()
    cb.set_option(cb.OPT_TREELET_PACKING, packing)
    try:
        host = _host_blob(cb, v, t, k, m, bits, tb)
        plan, h = _plan_blob(cb, len(v), len(t), k, m, bits, tb)
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
    assert plan.shape == host.shape
    hs, records = _structure(host)
    ps, _ = _structure(plan)
    if m == 2:
        assert records == 2 * len(t) - 1  # a binary tree with one triangle per leaf
    assert (hs == ps).all()
    assert (ps == plan).all()  # the plan's own bounds, table and exponent are zero
    assert h.info["n_nodes"] == records and h.info["n_tris"] == len(t)


def test_plan_shape_ignores_geometry(cb):
    """Two different meshes of the same size: the same structure."""
    v1, t1 = synth.icosphere(3, 1.0, 0.15, seed=1)
    v2, t2 = synth.icosphere(3, 2.5, 0.3, seed=2)
    rng = np.random.default_rng(5)
    t2 = t2[rng.permutation(len(t2))]
    a, _ = _structure(_host_blob(cb, v1, t1, 24, 8, 8, 4096))
    b, _ = _structure(_host_blob(cb, v2, t2, 24, 8, 8, 4096))
    assert (a == b).all()


def test_plan_argument_errors(cb):
    for args in [(100, 50, 5, 4, 8, 4096), (100, 50, 18, 3, 8, 4096), (100, 50, 18, 4, 7, 4096),
                 (100, 50, 18, 4, 8, 3000), (100, 50, 18, 4, 8, 1 << 18)]:
        with pytest.raises(cb.CbvhError) as e:
            cb.BVH.plan(*args, device=None)
        assert e.value.code == -1
    with pytest.raises(cb.CbvhError) as e:  # Stream VByte records: sizes follow the geometry
        cb.BVH.plan(100, 50, 18, 4, 2, 4096, device=None)
    assert e.value.code == -1
    for nv, nt in [(2, 10), (100, 0)]:
        with pytest.raises(cb.CbvhError) as e:
            cb.BVH.plan(nv, nt, 18, 4, 8, 4096, device=None)
        assert e.value.code == -2


def test_build_device_state_errors_before_cuda(cb):
    """A handle from cbvh_build is not a plan; a plan must be attached; NULLs are refused."""
    L = cb._load()
    v, t = synth.icosphere(1)
    host = cb.BVH(v, t, 18, 4, 8, 4096, device=None)
    plan = cb.BVH.plan(len(v), len(t), 18, 4, 8, 4096, device=None)
    buf = (C.c_uint8 * 1024)()
    p = C.cast(buf, C.c_void_p)
    assert L.cbvh_build_device(host.handle, p, p, p, 1024, 0, None) == -9
    assert L.cbvh_build_device(plan.handle, p, p, p, 1024, 0, None) == -9  # not attached
    assert L.cbvh_build_device(plan.handle, None, p, p, 1024, 0, None) == -1
    nb = C.c_int64()
    assert L.cbvh_build_device_workspace_bytes(plan.handle, C.byref(nb)) == 0
    nt, nn = len(t), plan.info["n_nodes"]
    assert nb.value >= 100 * nt + 24 * nn
