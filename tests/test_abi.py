"""The C-ABI library on the CPU: it builds, loads and exports every entry point the header
declares, its host builder/encoder reproduces the oracle's blob byte for byte, and host-side
argument errors come back as error codes (no GPU compute is run here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def cb():
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "cbvh.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cbvh_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(cb):
    """Both builds: libcbvh.so and the bounds-checked libcbvh_checked.so."""
    from paper_2012_05348_gb300 import _build
    syms = declared_symbols()
    assert len(syms) >= 10
    for path in (_build.LIB, _build.LIB_CHECKED):
        lib = C.CDLL(path)
        for s in syms:
            assert hasattr(lib, s), (path, s)


CONFIGS = [(18, 4, 16, 4096), (24, 8, 8, 16384), (6, 2, 8, 4096), (26, 16, 16, 8192), (18, 4, 0, 4096),
           (24, 8, 16, 65536), (18, 2, 16, 131072), (18, 16, 8, 32768), (18, 4, 1, 4096), (26, 8, 1, 16384),
           (18, 4, 2, 4096), (24, 8, 2, 16384), (26, 16, 2, 8192), (6, 2, 2, 131072)]


@pytest.fixture(params=[0, 1], ids=["top_down", "bottom_up"])
def packing(cb, request):
    cb.set_option(cb.OPT_TREELET_PACKING, request.param)
    yield request.param
    cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)


@pytest.mark.parametrize("k,m,bits,tb", CONFIGS)
def test_blob_identical_to_oracle(cb, packing, k, m, bits, tb):
    v, t = synth.icosphere(3, 1.0, 0.15, seed=k + m + bits)
    o = oracle.BVH(v, t, k, m, bits, tb, packing=packing)
    h = cb.BVH(v, t, k, m, bits, tb, device=None)
    assert h.info["n_nodes"] == o.n_nodes and h.info["n_treelets"] == o.n_treelets
    assert h.info["lattice_exp"] == o.e and h.info["depth"] == o.depth
    bo, bl = o.blob(), h.blob_host()
    assert len(bo) == len(bl) and (bo == bl).all()


def test_blob_identical_to_oracle_terrain_and_odd_meshes(cb, packing):
    va, ta, _ = synth.heightfield(96, seed=31)
    for v, t in [(va, ta), synth.box_mesh((1.0, 2.0, 3.0)), synth.capsule(0.5, 0.1, 2000, seed=3),
                 (np.array([[0, 0, 0], [1e-3, 0, 0], [0, 2e-3, 1e-4]], np.float32), np.array([[0, 1, 2]], np.int32)),
                 (np.array([[1e6, 1e6, 1e6], [1e6 + 64, 1e6, 1e6], [1e6, 1e6 + 64, 1e6 - 32]], np.float32),
                  np.array([[0, 1, 2]], np.int32))]:
        for k, m, bits, tb in [(24, 8, 8, 16384), (18, 4, 16, 4096), (18, 4, 1, 4096)]:
            if bits == 1 and np.abs(v).max() > 60000:  # beyond half precision: both refuse
                with pytest.raises(oracle.OracleError):
                    oracle.BVH(v, t, k, m, bits, tb, packing=packing)
                with pytest.raises(cb.CbvhError):
                    cb.BVH(v, t, k, m, bits, tb, device=None)
                continue
            o = oracle.BVH(v, t, k, m, bits, tb, packing=packing)
            h = cb.BVH(v, t, k, m, bits, tb, device=None)
            assert (o.blob() == h.blob_host()).all()


def test_build_errors(cb):
    v, t = synth.icosphere(1, seed=1)
    for args, code in [((5, 4, 8, 4096), -1), ((18, 3, 8, 4096), -1), ((18, 4, 12, 4096), -1),
                       ((18, 4, 8, 5000), -1), ((18, 4, 8, 2048), -1)]:
        with pytest.raises(cb.CbvhError) as e:
            cb.BVH(v, t, *args, device=None)
        assert e.value.code == code
    bad = t.copy()
    bad[3, 1] = -1
    with pytest.raises(cb.CbvhError) as e:
        cb.BVH(v, bad, device=None)
    assert e.value.code == -2
    deg = t.copy()
    deg[0] = (2, 2, 5)
    with pytest.raises(cb.CbvhError) as e:
        cb.BVH(v, deg, device=None)
    assert e.value.code == -2
    nan = v.copy()
    nan[0, 0] = np.nan
    with pytest.raises(cb.CbvhError) as e:
        cb.BVH(nan, t, device=None)
    assert e.value.code == -2


def test_queries_without_device_blob_are_rejected(cb):
    v, t = synth.icosphere(1, seed=1)
    A = cb.BVH(v, t, device=None)
    B = cb.BVH(v, t, device=None)
    st = C.c_int32()
    rc = cb.lib.cbvh_collide(A.handle, B.handle, None, 0, None, None, None, 0, None, 0, None, 0, C.byref(st), None)
    assert rc == -9
    rc = cb.lib.cbvh_distance(A.handle, B.handle, None, 0, None, None, 0, C.byref(st), None)
    assert rc == -9
    out = C.c_int64()
    # the workspace holds per-warp stacks sized by the current device; without one the call
    # reports a CUDA error instead of guessing
    rc = cb.lib.cbvh_workspace_bytes(A.handle, B.handle, 100, 0, 1000, C.byref(out))
    assert rc in (0, -3)
    if rc == 0:
        assert out.value >= 256 + 400 + 12000
    else:
        assert cb.lib.cbvh_last_error()
    assert cb.lib.cbvh_workspace_bytes(A.handle, B.handle, -1, 0, 0, C.byref(out)) == -1


def test_batch_rejects_unattached_handles(cb):
    v, t = synth.icosphere(1, seed=1)
    A = cb.BVH(v, t, device=None)
    B = cb.BVH(v, t, device=None)
    q = (cb._Query * 1)()
    q[0] = cb._Query(A.handle, B.handle, 0, 0, None, 0, None, None)
    h = C.c_void_p()
    assert cb.lib.cbvh_batch_create(q, 1, C.byref(h)) == -9
    assert cb.lib.cbvh_set_option(99, 0) == -1
    assert cb.lib.cbvh_set_option(cb.OPT_STAGE_BYTES, 1 << 20) == -1
    assert cb.lib.cbvh_set_option(cb.OPT_TREELET_PACKING, 2) == -1
    assert cb.lib.cbvh_set_option(cb.OPT_SPLIT, 5) == -1
    assert cb.lib.cbvh_set_option(cb.OPT_WAIT_CAP, 0) == -1
    assert cb.lib.cbvh_set_option(cb.OPT_WAIT_CAP, (1 << 24) + 1) == -1
    assert cb.lib.cbvh_set_option(cb.OPT_WAIT_CAP, cb.WAIT_CAP_DEFAULT) == 0
    assert cb.lib.cbvh_probe_l2_read(None, 1 << 20, 1, None, None, None) == -1


def test_kernel_launch_counter_without_gpu(cb):
    """The counter is host state: readable without a device, and NULL is an argument error."""
    n = cb.kernel_launches()
    assert n >= 0 and cb.kernel_launches() == n
    assert cb.lib.cbvh_kernel_launches(None) == -1


def test_refit_host_checks(cb):
    """Refit entry points without a device: the workspace size is host arithmetic; an
    unattached handle is rejected before anything reaches the GPU."""
    import ctypes as C
    v, t = synth.icosphere(2, 1.0, 0.1, seed=1)
    h = cb.BVH(v, t, 18, 4, 8, 4096, device=None)
    nb = C.c_int64()
    assert cb.lib.cbvh_refit_workspace_bytes(h.handle, C.byref(nb)) == 0
    assert nb.value >= h.info["n_nodes"] * (24 + 16 * 9)
    assert cb.lib.cbvh_refit(h.handle, C.c_void_p(16), 3, C.c_void_p(16), C.c_void_p(256), nb.value,
                             C.c_void_p(16), None) == -9  # CBVH_ERR_STATE


@pytest.mark.parametrize("headroom", [1, 3])
def test_blob_identical_with_lattice_headroom(cb, headroom):
    """CBVH_OPT_LATTICE_HEADROOM: the library and the oracle choose the same coarser lattice
    (bounds below 2^(30 - headroom) steps) and write the same bytes."""
    v, t = synth.icosphere(3, 1.0, 0.15, seed=8)
    cb.set_option(cb.OPT_LATTICE_HEADROOM, headroom)
    try:
        h = cb.BVH(v, t, 24, 8, 8, 16384, device=None)
    finally:
        cb.set_option(cb.OPT_LATTICE_HEADROOM, 0)
    o = oracle.BVH(v, t, 24, 8, 8, 16384, headroom=headroom)
    o0 = oracle.BVH(v, t, 24, 8, 8, 16384)
    assert o.e == o0.e + headroom and h.info["lattice_exp"] == o.e
    assert (h.blob_host() == o.blob()).all()
    assert cb.lib.cbvh_set_option(cb.OPT_LATTICE_HEADROOM, 9) == -1
