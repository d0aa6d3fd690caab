"""cbvh_save / cbvh_load (CPU): a saved hierarchy loads back byte for byte with the same
parameters, and a damaged file is refused with CBVH_ERR_IO before anything could reach a
kernel -- every field the kernels follow (treelet offsets, record offsets, parents,
children, child treelets, leaf slots, depths, triangle indices) is checked, so corrupting
any one of them is caught, and random damage never crashes the loader."""

import numpy as np
import pytest

import synth

ERR_IO, ERR_STATE = -10, -9


@pytest.fixture(scope="module")
def cb():
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


def _records(blob):
    """(treelet offset, node count, record offsets from the treelet start) per treelet."""
    hdr = blob[:64].view(np.uint32)
    bits, K = int(blob[9]), int(blob[7])
    ntl, rec, root = int(hdr[6]), int(hdr[7]), int(hdr[8])
    toff = blob[64:64 + 8 * (ntl + 1)].view(np.uint64).astype(np.int64)
    out = []
    for t in range(ntl):
        T = int(toff[t])
        cnt = int(blob[T:T + 4].view(np.uint32)[0])
        if bits == 2:
            offs = [4 * int(x) for x in blob[T + 16:T + 16 + 2 * cnt].view(np.uint16)]
        else:
            offs = [16 + (root + (l - 1) * rec if l else 0) for l in range(cnt)]
        out.append((T, cnt, offs))
    return out


def _save(cb, h, tmp_path, name="h.cbvh"):
    p = str(tmp_path / name)
    h.save(p)
    return p


def _write(path, head, blob):
    with open(path, "wb") as f:
        f.write(head)
        f.write(blob.tobytes())


def _refused(cb, path, code=ERR_IO):
    with pytest.raises(cb.CbvhError) as e:
        cb.BVH.load(path, device=None)
    assert e.value.code == code


MESHES = {"sphere": lambda: synth.icosphere(3, 1.0, 0.15, seed=9),
          "terrain": lambda: synth.heightfield(24, 4.0, seed=4)[:2],
          "one": lambda: (synth.icosphere(1)[0], synth.icosphere(1)[1][:1])}


@pytest.mark.parametrize("packing", [0, 1])
@pytest.mark.parametrize("k,m,bits,tb", [(18, 4, 16, 4096), (24, 8, 8, 16384), (6, 2, 8, 4096), (26, 16, 1, 8192),
                                         (24, 8, 0, 8192), (18, 4, 2, 4096), (24, 8, 2, 65536)])
@pytest.mark.parametrize("mesh", list(MESHES))
def test_round_trip(cb, tmp_path, mesh, k, m, bits, tb, packing):
    v, t = MESHES[mesh]()
    cb.set_option(cb.OPT_TREELET_PACKING, packing)
    try:
        h = cb.BVH(v, t, k, m, bits, tb, device=None)
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
    g = cb.BVH.load(_save(cb, h, tmp_path), device=None)
    assert (g.blob_host() == h.blob_host()).all()
    assert g.info == h.info and g.n_verts == len(v)
    # a loaded hierarchy saves to the same file
    p2 = _save(cb, g, tmp_path, "again.cbvh")
    assert open(p2, "rb").read() == open(str(tmp_path / "h.cbvh"), "rb").read()


def test_plan_is_not_saved(cb, tmp_path):
    p = cb.BVH.plan(100, 50, 18, 4, 8, 4096, device=None)
    with pytest.raises(cb.CbvhError) as e:
        p.save(str(tmp_path / "plan.cbvh"))
    assert e.value.code == ERR_STATE


def test_missing_and_truncated_files(cb, tmp_path):
    _refused(cb, str(tmp_path / "nothing.cbvh"))
    v, t = synth.icosphere(2, 1.0, 0.1, seed=1)
    path = _save(cb, cb.BVH(v, t, 18, 4, 8, 4096, device=None), tmp_path)
    data = open(path, "rb").read()
    for cut in (0, 8, 16, 40, 80, len(data) // 2, len(data) - 1):
        bad = str(tmp_path / f"cut{cut}.cbvh")
        open(bad, "wb").write(data[:cut])
        _refused(cb, bad)
    bad = str(tmp_path / "long.cbvh")
    open(bad, "wb").write(data + b"\0" * 16)
    _refused(cb, bad)


def _mutations(blob, bits):
    """(name, mutated blob) for every kind of field the loader must check."""
    recs = _records(blob)
    hdr_u32 = lambda b, i, v: b[:64].view(np.uint32).__setitem__(i, v)  # noqa: E731
    out = []

    def mut(name, fn):
        b = blob.copy()
        fn(b)
        out.append((name, b))

    mut("blob magic", lambda b: b.__setitem__(0, 0x00))
    mut("k", lambda b: b.__setitem__(6, 7))
    mut("branching", lambda b: b.__setitem__(8, 3))
    mut("quant_bits", lambda b: b.__setitem__(9, 4))
    mut("node count", lambda b: hdr_u32(b, 5, int(b[:64].view(np.uint32)[5]) + 1))
    mut("depth", lambda b: hdr_u32(b, 10, int(b[:64].view(np.uint32)[10]) + 1))
    mut("record size", lambda b: hdr_u32(b, 7, int(b[:64].view(np.uint32)[7]) + 4))
    ntl = len(recs)
    if ntl >= 3:
        def swap_offsets(b):
            t = b[64:64 + 8 * (ntl + 1)].view(np.uint64)
            t[1], t[2] = t[2], t[1]
        mut("treelet offsets", swap_offsets)
    T0, cnt0, offs0 = recs[0]
    mut("treelet node count", lambda b: b[T0:T0 + 4].view(np.uint32).__setitem__(0, cnt0 + 1))
    # the first inner record of the first treelet with local children, and a leaf record
    inner = leaf = None
    for T, cnt, offs in recs:
        for l in range(cnt):
            w0, w1 = blob[T + offs[l]:T + offs[l] + 8].view(np.uint32)
            nc, ext = (int(w0) >> 16) & 31, (int(w0) >> 21) & 1
            if nc and not ext and inner is None:
                inner = (T + offs[l], cnt)
            if nc == 0 and leaf is None:
                leaf = T + offs[l]
    if inner is not None:
        R, cnt = inner
        mut("first child", lambda b: b[R + 4:R + 8].view(np.uint32).__setitem__(0, cnt + 5))
        mut("child count", lambda b: b[R:R + 4].view(np.uint32).__setitem__(
            0, (int(b[R:R + 4].view(np.uint32)[0]) & ~(31 << 16)) | (31 << 16)))
    if leaf is not None:
        nt = int(blob[16:20].view(np.uint32)[0])
        mut("leaf slot", lambda b: b[leaf + 4:leaf + 8].view(np.uint32).__setitem__(0, nt))
    ext_rec = None
    for T, cnt, offs in recs:
        for l in range(cnt):
            w0 = int(blob[T + offs[l]:T + offs[l] + 4].view(np.uint32)[0])
            if (w0 >> 21) & 1:
                ext_rec = T + offs[l]
                break
        if ext_rec is not None:
            break
    if ext_rec is not None:
        mut("child treelet", lambda b: b[ext_rec + 4:ext_rec + 8].view(np.uint32).__setitem__(0, ntl))
    # two inner records of one treelet at the same depth with local children: re-parent a
    # child of the second to the first (depths stay consistent), and point the second's
    # child range at the first's (its nodes would be referenced twice)
    pair = None
    for T, cnt, offs in recs:
        by_depth = {}
        for l in range(cnt):
            w0, w1 = (int(x) for x in blob[T + offs[l]:T + offs[l] + 8].view(np.uint32))
            if (w0 >> 16) & 31 and not (w0 >> 21) & 1:
                by_depth.setdefault(w0 >> 24, []).append((l, w1))
        for d, ls in sorted(by_depth.items()):
            if len(ls) >= 2:
                pair = (T, offs, ls[0], ls[1])
                break
        if pair is not None:
            break
    if pair is not None:
        T, offs, (l1, c1), (l2, c2) = pair
        R = T + offs[c2]
        mut("child's parent field", lambda b: b[R:R + 4].view(np.uint32).__setitem__(
            0, (int(b[R:R + 4].view(np.uint32)[0]) & ~0xffff) | l1))
        R2 = T + offs[l2]
        mut("child referenced twice", lambda b: b[R2 + 4:R2 + 8].view(np.uint32).__setitem__(0, c1))
    if len(offs0) > 1:
        R = T0 + offs0[1]
        mut("parent", lambda b: b[R:R + 4].view(np.uint32).__setitem__(
            0, (int(b[R:R + 4].view(np.uint32)[0]) & ~0xffff) | 0x7fff))
    off_tris = int(blob[48:56].view(np.uint64)[0])
    nt = int(blob[16:20].view(np.uint32)[0])
    mut("triangle index", lambda b: b[off_tris + 12:off_tris + 16].view(np.uint32).__setitem__(0, nt + 3))
    if bits == 2:
        T, cnt, offs = next(r for r in recs if r[1] > 2)
        mut("record offset", lambda b: b[T + 18:T + 20].view(np.uint16).__setitem__(0, 0x3fff))
        R = T + offs[-1]
        mut("control word", lambda b: b[R + 8:R + 16].view(np.uint64).__setitem__(0, np.uint64(2 ** 64 - 1)))
    return out


@pytest.mark.parametrize("bits", [8, 2])
def test_each_damaged_field_is_refused(cb, tmp_path, bits):
    v, t = synth.icosphere(3, 1.0, 0.15, seed=5)
    h = cb.BVH(v, t, 18, 4, bits, 4096, device=None)
    blob = h.blob_host()
    head = open(_save(cb, h, tmp_path), "rb").read()[:16]
    bad_head = bytearray(head)
    bad_head[0] = ord("X")
    _write(str(tmp_path / "head.cbvh"), bytes(bad_head), blob)
    _refused(cb, str(tmp_path / "head.cbvh"))
    muts = _mutations(blob, bits)
    assert len(muts) >= 16
    for name, b in muts:
        p = str(tmp_path / f"m_{name.replace(' ', '_')}.cbvh")
        _write(p, head, b)
        with pytest.raises(cb.CbvhError) as e:
            cb.BVH.load(p, device=None)
        assert e.value.code == ERR_IO, name


@pytest.mark.parametrize("bits", [16, 2])
def test_random_damage_never_crashes(cb, tmp_path, bits):
    """Single-byte damage anywhere in the header, the treelet table, the treelet headers,
    the offset tables and the topology words: the loader answers OK or CBVH_ERR_IO."""
    v, t = synth.icosphere(3, 1.0, 0.15, seed=7)
    h = cb.BVH(v, t, 24, 8, bits, 4096, device=None)
    blob = h.blob_host()
    head = open(_save(cb, h, tmp_path), "rb").read()[:16]
    recs = _records(blob)
    spots = list(range(0, 64 + 8 * (len(recs) + 1)))
    for T, cnt, offs in recs:
        spots += list(range(T, T + 16 + (2 * cnt if bits == 2 else 0)))
        for o in offs:
            spots += list(range(T + o, T + o + 8))
    rng = np.random.default_rng(11)
    p = str(tmp_path / "fuzz.cbvh")
    refused = 0
    for i in rng.choice(len(spots), 400, replace=False):
        b = blob.copy()
        b[spots[i]] ^= np.uint8(1 << int(rng.integers(8)))
        _write(p, head, b)
        try:
            cb.BVH.load(p, device=None)
        except cb.CbvhError as e:
            assert e.code == ERR_IO
            refused += 1
    assert refused > 300  # almost every damaged topology byte is caught
