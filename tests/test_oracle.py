"""Pins of the FP64 oracle against things other than itself (CPU only).

- exact lattice arithmetic against Python's exact rationals (fractions.Fraction);
- the triangle primitives against closed forms and against an exhaustive active-set
  solution of the distance QP (every pair of sub-simplices), and scipy's SLSQP;
- the BVH traversal of Algorithm 1 against brute force over all triangle pairs;
- CD/PQ against closed-form box-box distances and a convex-hull QP;
- the encoding against its invariants (conservative, nested, in range) and the
  independent blob decoder;
- the near-contact filter against a brute-force recomputation.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1),
        (0, 1, -1), (1, 1, 1), (1, 1, -1), (1, -1, 1), (-1, 1, 1)]


# ------------------------------------------------------------------ exact lattice
def _frac_floor(x: Fraction) -> int:
    return math.floor(x)


def test_floor_sum3_matches_exact_rationals():
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(3000):
        e = rng.integers(-60, 60, size=3)
        v = rng.uniform(-1, 1, size=3) * np.exp2(e)
        cases.append(tuple(float(x) for x in v))
    # adversarial: integers plus tiny residues of either sign, cancellation, huge spread
    for k in range(1, 40):
        t = 2.0 ** -k
        cases += [(5.0, t, -t), (5.0, -t, 0.0), (5.0, t, 0.0), (-3.0, 1.0 - t, -t), (2.0 ** 29, -0.5, -t),
                  (1e16, -1e16, t), (1e16, -1e16, -t), (7.5, 0.5, -2.0 ** -1074)]
    for a, b, c in cases:
        exact = Fraction(a) + Fraction(b) + Fraction(c)
        assert oracle.floor_sum3(a, b, c) == _frac_floor(exact), (a, b, c)
        assert oracle.ceil_sum3(a, b, c) == math.ceil(exact), (a, b, c)


def test_lattice_dv_matches_exact_rationals():
    rng = np.random.default_rng(8)
    for _ in range(2000):
        v = (rng.uniform(-3, 3, size=3) * np.exp2(rng.integers(-20, 3, size=3))).astype(np.float32)
        j = int(rng.integers(0, 13))
        e = int(rng.integers(-40, -10))
        d = DIRS[j]
        x = sum(Fraction(int(d[c])) * Fraction(float(v[c])) for c in range(3)) / Fraction(2) ** e
        lo, hi = oracle.lattice_dv(v, j, e)
        assert lo == math.floor(x) and hi == math.ceil(x)


def _tiny_mesh(seed, n=40):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, size=(n, 1, 3))
    v = (c + rng.uniform(-0.2, 0.2, size=(n, 3, 3))).reshape(-1, 3).astype(np.float32)
    return v, np.arange(3 * n, dtype=np.int32).reshape(n, 3)


@pytest.mark.parametrize("k,m,bits", [(6, 2, 8), (18, 4, 16), (24, 8, 8), (26, 16, 16), (18, 4, 0)])
def test_exact_node_lattice_and_exponent(k, m, bits):
    v, t = _tiny_mesh(3 + k + m)
    h = oracle.BVH(v, t, k, m, bits, 4096)
    K = k // 2
    # exponent: smallest e with |d.v| / 2^e < 2^30 for every used vertex and direction
    vals = [sum(Fraction(d[c]) * Fraction(float(p[c])) for c in range(3)) for p in v for d in DIRS[:K]]
    M = max(abs(x) for x in vals)
    assert M / Fraction(2) ** h.e < 2 ** 30
    assert not (M / Fraction(2) ** (h.e - 1) < 2 ** 30)
    tr = h.tree()
    lat = h.lattice()["exact"]
    # the triangle set of every node, from the tree
    sets = [None] * h.n_nodes
    for x in range(h.n_nodes - 1, -1, -1):
        if tr["nchild"][x] == 0:
            sets[x] = [int(tr["tri"][x])]
        else:
            sets[x] = sum((sets[tr["first"][x] + c] for c in range(tr["nchild"][x])), [])
    assert sorted(sets[0]) == list(range(len(t)))
    scale = Fraction(2) ** h.e
    for x in range(h.n_nodes):
        pts = [v[i] for tri in sets[x] for i in t[tri]]
        for j in range(K):
            xs = [sum(Fraction(DIRS[j][c]) * Fraction(float(p[c])) for c in range(3)) / scale for p in pts]
            assert lat[x, j, 0] == math.floor(min(xs)) and lat[x, j, 1] == math.ceil(max(xs))


def _centroid_keys(v, t):
    p = v[t].astype(np.float64)
    return (p[:, 0] + p[:, 1]) + p[:, 2]


@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_tree_split_properties(m):
    """Every inner node has min(n, m) children, child sizes come from repeated floor/ceil
    halving, and each binary split separates its halves along the axis of largest
    centroid extent (checked by regrouping the children in split order)."""
    v, t = synth.icosphere(2, 1.0, 0.15, seed=11)
    h = oracle.BVH(v, t, 18, m, 16, 4096)
    tr = h.tree()
    key = _centroid_keys(v, t)
    sets = [None] * h.n_nodes
    for x in range(h.n_nodes - 1, -1, -1):
        if tr["nchild"][x] == 0:
            sets[x] = [int(tr["tri"][x])]
        else:
            sets[x] = sum((sets[tr["first"][x] + c] for c in range(tr["nchild"][x])), [])

    def check_split(groups):
        # groups: list of triangle lists in split order that came from one group of the
        # previous round; reconstruct the binary tree of splits bottom-up
        if len(groups) == 1:
            return groups[0]
        n = sum(len(g) for g in groups)
        left_n = n // 2
        acc, cut = 0, 0
        while acc < left_n:
            acc += len(groups[cut])
            cut += 1
        assert acc == left_n
        L, R = check_split(groups[:cut]), check_split(groups[cut:])
        both = L + R
        ext = key[both].max(0) - key[both].min(0)
        ax = int(np.argmax(ext))  # first maximum: ties resolved x < y < z
        kl = sorted((key[i, ax], i) for i in L)
        kr = sorted((key[i, ax], i) for i in R)
        assert kl[-1] < kr[0]
        return both

    for x in range(h.n_nodes):
        nc = tr["nchild"][x]
        if nc == 0:
            assert len(sets[x]) == 1
            continue
        n = len(sets[x])
        assert nc == min(n, m)
        check_split([sets[tr["first"][x] + c] for c in range(nc)])


@pytest.mark.parametrize("packing", [oracle.PACKING_TOP_DOWN, oracle.PACKING_BOTTOM_UP])
@pytest.mark.parametrize("k,m,bits,tb", [(18, 4, 16, 4096), (24, 8, 8, 16384), (6, 2, 8, 4096),
                                         (26, 16, 16, 8192), (18, 4, 0, 4096), (24, 8, 16, 65536),
                                         (18, 4, 1, 4096), (24, 8, 1, 16384), (18, 4, 2, 4096), (24, 8, 2, 16384),
                                         (26, 16, 2, 8192)])
def test_encoding_invariants(k, m, bits, tb, packing):
    v, t = synth.icosphere(3, 1.0, 0.15, seed=5)
    h = oracle.BVH(v, t, k, m, bits, tb, packing=packing)
    tr = h.tree()
    L = h.lattice()
    ex, dec, decf = L["exact"], L["decoded"], L["decf"]
    pl = h.placement()
    # conservative and nested
    assert (dec[..., 0] <= ex[..., 0]).all() and (dec[..., 1] >= ex[..., 1]).all()
    par = tr["parent"][1:]
    assert (dec[1:, :, 0] >= dec[par, :, 0]).all() and (dec[1:, :, 1] <= dec[par, :, 1]).all()
    # correctors fit b bits
    if bits >= 8:
        assert pl["delta"].max() <= (1 << bits) - 1
    if bits == oracle.QUANT_SVB:  # lossless: the decoded intervals are the exact ones
        assert (dec == ex).all()
    # the FP32 bounds contain the exact real bounds d.v of every vertex of the node
    e = h.e
    for x in range(0, h.n_nodes, 7):
        assert (decf[x, :, 0].astype(np.float64) <= np.ldexp(ex[x, :, 0].astype(np.float64), e)).all()
        assert (decf[x, :, 1].astype(np.float64) >= np.ldexp(ex[x, :, 1].astype(np.float64), e)).all()
    # treelet roots (local 0) are exact; nodes of one treelet stay within the byte budget
    roots = pl["local"] == 0
    assert (dec[roots] == ex[roots]).all()
    counts = np.bincount(pl["treelet"])
    # (Stream VByte: formed with the largest record and its offset-table entry)
    form_root, form_rec = (h.root_bytes + 8, h.rec_bytes + 2) if bits == oracle.QUANT_SVB else (h.root_bytes,
                                                                                               h.rec_bytes)
    assert (16 + form_root + (counts - 1) * form_rec <= tb).all()
    blob = h.blob()
    toff = blob[64:64 + 8 * (h.n_treelets + 1)].view(np.uint64).astype(np.int64)
    assert (np.diff(toff) <= tb).all()  # the bytes actually written, padding included
    assert (toff % 16 == 0).all()
    if bits == oracle.QUANT_SVB:  # every absolute root record 8-byte aligned, every record 4
        for t in range(h.n_treelets):
            c = int(blob[toff[t]:toff[t] + 4].view(np.uint32)[0])
            offs = 4 * blob[toff[t] + 16:toff[t] + 16 + 2 * c].view(np.uint16).astype(np.int64)
            assert offs[0] % 8 == 0 and offs[0] >= 16 + 2 * c and (np.diff(offs) > 0).all()
    # the independent decoder reproduces the encoder, node by node
    lat, f, meta = oracle.decode_blob(blob)
    order = np.lexsort((pl["local"], pl["treelet"]))
    if bits >= 8 or bits == oracle.QUANT_SVB:
        assert (lat == dec[order]).all()
    assert (f.view(np.uint32) == decf[order].view(np.uint32)).all()
    assert ((meta[:, 0] >> 16) & 31 == tr["nchild"][order]).all()
    # treelets hold whole sibling groups: a node and its siblings share a treelet, and a
    # non-root node's parent is in the same treelet
    par_all = tr["parent"]
    nonroot = ~roots
    assert (pl["treelet"][nonroot] == pl["treelet"][par_all[nonroot]]).all()
    fit = (tb - 16 - form_root) // form_rec + 1
    if packing == oracle.PACKING_BOTTOM_UP:
        # bottom-up rule, checked against its statement: an inner node's children were cut
        # off exactly when the node plus the nodes of their treelets would not fit one treelet
        for x in range(h.n_nodes):
            nc = tr["nchild"][x]
            if nc == 0:
                continue
            kids = tr["first"][x] + np.arange(nc)
            cut = pl["treelet"][kids[0]] != pl["treelet"][x]
            assert (pl["treelet"][kids] != pl["treelet"][x]).all() == cut
            if cut:
                assert 1 + counts[pl["treelet"][kids]].sum() > fit
        # treelets are numbered in node order of their roots
        rn = np.flatnonzero(roots)
        assert (pl["treelet"][rn] == np.arange(len(rn))).all()


def _adjacent_f32(decf, L, e):
    """decf[..., 0] is the largest FP32 value <= L_lo 2^e and decf[..., 1] the smallest >=
    L_hi 2^e (exact comparisons: |L| < 2^31, so L 2^e and every FP32 value are exact in FP64)."""
    lo, hi = decf[..., 0], decf[..., 1]
    xlo = np.ldexp(L[..., 0].astype(np.float64), e)
    xhi = np.ldexp(L[..., 1].astype(np.float64), e)
    up = np.nextafter(lo, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(hi, np.float32(-np.inf)).astype(np.float64)
    assert (lo.astype(np.float64) <= xlo).all() and (up > xlo).all()
    assert (hi.astype(np.float64) >= xhi).all() and (dn < xhi).all()


def _predictor_corrector_mesh(kind):
    if kind == "sphere":
        return synth.icosphere(3, 1.0, 0.15, seed=5)
    # adversarial: coordinates on a coarse power-of-two grid, so that many parent ranges
    # sit exactly at (2^b - 1) 2^s and at powers of two, where an off-by-one in the shift
    # or in a corrector's rounding shows
    rng = np.random.default_rng(41)
    n = 300
    c = rng.integers(-64, 64, size=(n, 1, 3)).astype(np.float64)
    v = (c + rng.integers(-5, 6, size=(n, 3, 3))) * 2.0 ** -5
    v[:, 2] += 2.0 ** -9  # keep every triangle non-degenerate
    v = v.reshape(-1, 3).astype(np.float32)
    return v, np.arange(3 * n, dtype=np.int32).reshape(n, 3)


@pytest.mark.parametrize("mesh", ["sphere", "grid"])
@pytest.mark.parametrize("packing", [oracle.PACKING_TOP_DOWN, oracle.PACKING_BOTTOM_UP])
@pytest.mark.parametrize("k,m,bits,tb", [(24, 8, 8, 16384), (18, 4, 16, 4096), (6, 2, 8, 4096), (26, 16, 8, 8192),
                                         (18, 4, 0, 4096), (18, 4, 2, 4096), (24, 8, 16, 65536)])
def test_predictor_corrector_against_its_definition(k, m, bits, tb, packing, mesh):
    """The encoder's shift, correctors and decoded intervals, recomputed top-down from the
    node's exact lattice interval C and the parent's decoded interval P, as the abstract and
    Sec. III-B describe them (the prediction is the parent's decoded bounds, the correction a
    small outward integer delta):
      s     = smallest s >= 0 with (P_hi - P_lo) >> s <= 2^b - 1, i.e. max(0, bitlen - b);
      d_lo  = floor((C_lo - P_lo) / 2^s),  d_hi = floor((P_hi - C_hi) / 2^s);
      C'    = [P_lo + d_lo 2^s, P_hi - d_hi 2^s]  (the tightest such interval around C).
    Treelet roots are absolute (exact); FP32 and FP16 records are absolute; Stream VByte
    records hold the unshifted exact deltas.  The decoded FP32 bounds are the adjacent
    floats: lo the largest FP32 <= C'_lo 2^e, hi the smallest >= C'_hi 2^e."""
    v, t = _predictor_corrector_mesh(mesh)
    h = oracle.BVH(v, t, k, m, bits, tb, packing=packing)
    tr, L, pl = h.tree(), h.lattice(), h.placement()
    ex, dec, decf, delta = L["exact"], L["decoded"], L["decf"], pl["delta"]
    par, local = tr["parent"], pl["local"]
    K = k // 2
    want_dec = np.empty_like(ex)
    want_delta = np.zeros_like(delta)
    for x in range(h.n_nodes):  # parents precede their children in node order
        C = [(int(ex[x, j, 0]), int(ex[x, j, 1])) for j in range(K)]
        if local[x] == 0 or bits in (0, 1):
            want_dec[x] = ex[x]
            continue
        assert par[x] < x
        for j in range(K):
            P_lo, P_hi = int(want_dec[par[x], j, 0]), int(want_dec[par[x], j, 1])
            C_lo, C_hi = C[j]
            assert P_lo <= C_lo <= C_hi <= P_hi
            if bits == oracle.QUANT_SVB:
                want_delta[x, j] = (C_lo - P_lo, P_hi - C_hi)
                want_dec[x, j] = (C_lo, C_hi)
                continue
            s = max(0, (P_hi - P_lo).bit_length() - bits)
            assert (P_hi - P_lo) >> s <= (1 << bits) - 1 and (s == 0 or (P_hi - P_lo) >> (s - 1) > (1 << bits) - 1)
            d_lo, d_hi = (C_lo - P_lo) // 2 ** s, (P_hi - C_hi) // 2 ** s
            lo, hi = P_lo + d_lo * 2 ** s, P_hi - d_hi * 2 ** s
            # outward, and one more step of 2^s inward would cut the exact interval
            assert lo <= C_lo < lo + 2 ** s and hi - 2 ** s < C_hi <= hi
            want_delta[x, j] = (d_lo, d_hi)
            want_dec[x, j] = (lo, hi)
    assert (dec == want_dec).all()
    if bits >= 8 or bits == oracle.QUANT_SVB:
        assert (delta == want_delta).all()
    if bits != oracle.QUANT_FP16:  # FP16 rounding has its own pin below
        _adjacent_f32(decf, want_dec, h.e)


def _golden_svb():
    path = os.path.join(os.path.dirname(__file__), "golden", "stream_vbyte.txt")
    cases = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        vals, ctl, data = (x.split() for x in line.split("|"))
        cases.append(([int(v, 0) for v in vals], bytes.fromhex("".join(ctl)), bytes.fromhex("".join(data))))
    return cases


@pytest.mark.parametrize("vals,ctl,data", _golden_svb())
def test_stream_vbyte_format(vals, ctl, data):
    """The Stream VByte coder of quant_bits = 2 against byte strings worked out by hand from
    the format's published definition (Lemire, Kurz and Rupp 2018)."""
    got_ctl, got_data = oracle.svb_encode(vals)
    assert got_data == data
    assert got_ctl[:len(ctl)] == ctl and got_ctl[len(ctl):] == bytes(8 - len(ctl))


def test_stream_vbyte_records_hold_the_parent_deltas():
    """A Stream VByte record's deltas are exactly C_lo - P_lo and P_hi - C_hi against the
    parent's exact interval, read back from the blob bytes by the format's rule; and the
    footprint lies between the 8-bit and the FP32 encodings of the same tree."""
    v, t = synth.icosphere(3, 1.0, 0.15, seed=5)
    h = oracle.BVH(v, t, 18, 4, oracle.QUANT_SVB, 4096)
    tr, pl, ex = h.tree(), h.placement(), h.lattice()["exact"]
    blob = h.blob()
    toff = blob[64:64 + 8 * (h.n_treelets + 1)].view(np.uint64).astype(np.int64)
    K = h.K
    for x in range(1, h.n_nodes, 5):
        if pl["local"][x] == 0:
            continue
        T = toff[pl["treelet"][x]]
        off = 4 * int(blob[T + 16 + 2 * pl["local"][x]:T + 18 + 2 * pl["local"][x]].view(np.uint16)[0])
        R = T + off
        ctl = int.from_bytes(blob[R + 8:R + 16].tobytes(), "little")
        q = R + 16
        vals = []
        for i in range(2 * K):
            n = ((ctl >> (2 * i)) & 3) + 1
            vals.append(int.from_bytes(blob[q:q + n].tobytes(), "little"))
            q += n
        p = tr["parent"][x]
        want = [(ex[x, j, 0] - ex[p, j, 0], ex[p, j, 1] - ex[x, j, 1])[s] for j in range(K) for s in (0, 1)]
        assert vals == want
    b8 = oracle.BVH(v, t, 18, 4, 8, 4096).blob_bytes
    b32 = oracle.BVH(v, t, 18, 4, 0, 4096).blob_bytes
    assert b8 < h.blob_bytes < b32


def test_half_precision_rounding_is_outward_and_tight():
    """The FP16 descriptor mode's conversion against numpy's binary16 (round to nearest):
    the rounded-down and rounded-up halves bracket v, are adjacent (or equal when v is a
    half), and one of them is numpy's nearest half; every non-negative bit pattern decodes
    to numpy's value."""
    bits = np.arange(0, 0x7c00, dtype=np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    for b in list(range(0, 0x7c00, 97)) + [0x0001, 0x03ff, 0x0400, 0x3c00, 0x7bff]:
        assert oracle.half_value(b) == ref[b]
        assert oracle.half_value(0x8000 | b) == -ref[b]
    assert oracle.half_value(0x7c00) == np.inf
    rng = np.random.default_rng(17)
    vals = np.concatenate([rng.uniform(-1, 1, 200) * 10.0 ** rng.integers(-9, 5, 200),
                           [0.0, 1.0, -1.0, 65504.0, 65504.5, -70000.0, 1e-9, -3e-8, 2.0 ** -24, 0.1]])
    for v in vals:
        lo, hi = oracle.half_rd(v), oracle.half_ru(v)
        vl, vh = oracle.half_value(lo), oracle.half_value(hi)
        assert vl <= v <= vh
        if abs(v) <= 65504.0:
            nearest = float(np.float16(v))
            assert nearest in (vl, vh)
            if v > 0:
                assert hi - lo in (0, 1)
            elif v < 0:
                assert (lo & 0x7fff) - (hi & 0x7fff) in (0, 1)
            if nearest == v:
                assert vl == vh == v
    assert oracle.half_value(oracle.half_ru(70000.0)) == np.inf
    assert oracle.half_value(oracle.half_rd(70000.0)) == 65504.0
    assert oracle.half_value(oracle.half_rd(-70000.0)) == -np.inf


def test_bad_arguments_and_meshes():
    v, t = synth.icosphere(1, seed=1)
    for args in [(5, 4, 8, 4096), (18, 3, 8, 4096), (18, 4, 12, 4096), (18, 4, 8, 5000), (18, 4, 8, 2048)]:
        with pytest.raises(oracle.OracleError):
            oracle.BVH(v, t, *args)
    bad = t.copy()
    bad[0, 0] = len(v)
    with pytest.raises(oracle.OracleError):
        oracle.BVH(v, bad, 18, 4, 8, 4096)
    deg = t.copy()
    deg[0] = (0, 0, 1)
    with pytest.raises(oracle.OracleError):
        oracle.BVH(v, deg, 18, 4, 8, 4096)


# ------------------------------------------------------------------ triangle primitives
def _qp_exact(V, U):
    """Triangle-triangle distance by exhaustive active sets: for every pair of non-empty
    vertex subsets, minimise over their affine hulls; keep solutions with non-negative
    barycentric weights.  The optimum of the convex QP lies in the relative interior of
    some face pair, where it equals that affine minimum."""
    best = math.inf
    subsets = [s for r in (1, 2, 3) for s in itertools.combinations(range(3), r)]
    for S in subsets:
        for T in subsets:
            E = np.array([V[i] - V[S[0]] for i in S[1:]]).reshape(-1, 3).T
            F = np.array([U[j] - U[T[0]] for j in T[1:]]).reshape(-1, 3).T
            M = np.concatenate([E, -F], axis=1)
            r0 = V[S[0]] - U[T[0]]
            if M.shape[1]:
                x, *_ = np.linalg.lstsq(M, -r0, rcond=None)
            else:
                x = np.zeros(0)
            a, b = x[:len(S) - 1], x[len(S) - 1:]
            lam = np.concatenate([[1 - a.sum()], a])
            mu = np.concatenate([[1 - b.sum()], b])
            if lam.min() < -1e-12 or mu.min() < -1e-12:
                continue
            best = min(best, float(np.linalg.norm(r0 + M @ x)))
    return best


def test_tri_primitives_closed_forms():
    T = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    for h in (0.5, 1e-3, 2.0):
        U = T + [0, 0, h]
        assert oracle.tri_dist(T, U) == pytest.approx(h, rel=1e-14)
        assert not oracle.tri_intersect(T, U)[0]
    # coplanar overlap and coplanar separation (gap along x of 0.25)
    assert oracle.tri_intersect(T, T + [0.2, 0.2, 0])[0]
    U = np.array([[1.25, 0, 0], [2, 0, 0], [1.25, 1, 0]], float)
    assert not oracle.tri_intersect(T, U)[0]
    assert oracle.tri_dist(T, U) == pytest.approx(0.25, rel=1e-14)
    # a vertical triangle piercing T
    U = np.array([[0.2, 0.2, -1], [0.3, 0.2, 1], [0.2, 0.3, 1]], float)
    assert oracle.tri_intersect(T, U)[0] and oracle.tri_dist(T, U) == 0.0
    # touching at a single point (closed): vertex of U on T's interior
    U = np.array([[0.2, 0.2, 0], [0.2, 0.2, 1], [0.3, 0.4, 1]], float)
    assert oracle.tri_intersect(T, U)[0]
    # skew edges: edge x-axis segment vs a segment parallel to y at height z=h, x=0.5
    h = 0.3
    U = np.array([[0.5, -1, h], [0.5, -2, h + 5], [0.5, -0.0001, h + 5]], float)
    # closest features: T's edge (0,0,0)-(1,0,0) and U's edge from (0.5,-1,h) .. -> distance
    d = oracle.tri_dist(T, U)
    assert d == pytest.approx(_qp_exact(T, U), abs=1e-12)
    # segment-segment closed form: perpendicular skew lines at distance h
    assert oracle.seg_seg([0, 0, 0], [1, 0, 0], [0.5, -1, h], [0.5, 1, h]) == pytest.approx(h, rel=1e-14)
    # parallel segments, offset: endpoint-to-segment
    assert oracle.seg_seg([0, 0, 0], [1, 0, 0], [2, 1, 0], [3, 1, 0]) == pytest.approx(math.sqrt(2), rel=1e-14)
    # point above the interior / beyond a vertex
    assert oracle.pt_tri([0.2, 0.2, 0.7], T) == pytest.approx(0.7, rel=1e-14)
    assert oracle.pt_tri([-3, -4, 0], T) == pytest.approx(5.0, rel=1e-14)


def test_tri_primitives_against_exhaustive_qp():
    rng = np.random.default_rng(123)
    n_hit = n_miss = 0
    for _ in range(600):
        V = rng.uniform(-1, 1, size=(3, 3))
        U = rng.uniform(-1, 1, size=(3, 3)) * rng.uniform(0.2, 1.5) + rng.uniform(-0.8, 0.8, size=3)
        hit, margin = oracle.tri_intersect(V, U)
        d = oracle.tri_dist(V, U)
        q = _qp_exact(V, U)
        if hit:
            if margin < 1e-6:
                continue
            n_hit += 1
            assert d == 0.0 and q < 1e-9
        else:
            n_miss += 1
            assert q > 0 and d == pytest.approx(q, rel=1e-9, abs=1e-12)
    assert n_hit > 50 and n_miss > 50


def test_tri_dist_against_slsqp():
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(9)
    for _ in range(40):
        V = rng.uniform(-1, 1, size=(3, 3))
        U = rng.uniform(-1, 1, size=(3, 3)) + rng.uniform(1.0, 2.0, size=3)
        f = lambda z: float(np.sum((z[:3] @ V - z[3:] @ U) ** 2))  # noqa: E731
        cons = [{"type": "eq", "fun": lambda z: z[:3].sum() - 1}, {"type": "eq", "fun": lambda z: z[3:].sum() - 1}]
        r = opt.minimize(f, np.full(6, 1 / 3), method="SLSQP", bounds=[(0, 1)] * 6, constraints=cons,
                         options={"ftol": 1e-16, "maxiter": 500})
        assert oracle.tri_dist(V, U) == pytest.approx(math.sqrt(r.fun), rel=1e-5, abs=1e-8)


# ------------------------------------------------------------------ traversal pins
@pytest.fixture(scope="module")
def c1_small():
    c = synth.C1(24)
    A = oracle.BVH(*c["A"], 18, 4, 16, 4096)
    B = oracle.BVH(*c["B"], 18, 4, 16, 4096)
    return c, A, B


def test_algorithm1_cd_equals_brute_force(c1_small):
    c, A, B = c1_small
    hit, off, ij, st = oracle.collide(A, B, c["poses"])
    hb, ob, ijb = oracle.brute_collide(A, B, c["poses"])
    assert hit.sum() > 3 and (hit == 0).sum() > 3
    assert (hit == hb).all() and (off == ob).all() and (ij == ijb).all()
    # compressed (decoded FP32) bounding volumes prune to the same answer
    hd, od, ijd, std = oracle.collide(A, B, c["poses"], use_decoded=True)
    assert (hd == hit).all() and (od == off).all() and (ijd == ij).all()
    assert st["bv_tests"] > 0 and std["bv_tests"] >= st["bv_tests"] * 0.9


def test_algorithm1_pq_equals_brute_force(c1_small):
    c, A, B = c1_small
    d, _ = oracle.distance(A, B, c["poses"])
    db = oracle.brute_distance(A, B, c["poses"])
    dd, _ = oracle.distance(A, B, c["poses"], use_decoded=True)
    assert (d == db).all() and (dd == db).all()
    hit, *_ = oracle.collide(A, B, c["poses"])
    assert ((d == 0) == (hit == 1)).all()


def test_box_box_closed_form():
    va, ta = synth.box_mesh((1.0, 0.6, 0.4))
    vb, tb = synth.box_mesh((0.5, 0.5, 0.5))
    A = oracle.BVH(va, ta, 18, 4, 16, 4096)
    B = oracle.BVH(vb, tb, 18, 4, 16, 4096)
    rng = np.random.default_rng(4)
    # half sizes of the two boxes as the FP32 meshes store them
    half = np.abs(va.astype(np.float64)).max(0) + np.abs(vb.astype(np.float64)).max(0)
    P, expect = [], []
    while len(P) < 60:
        tr = rng.uniform(-1.5, 1.5, size=3)
        gap = np.abs(tr) - half
        if (gap > 1e-3).any():
            expect.append(float(np.linalg.norm(np.maximum(gap, 0))))
        elif (np.abs(gap) > 1e-3).all() and (gap < 0).all() and ((np.abs(tr) + 0.25 > np.array([0.5, 0.3, 0.2])).any()):
            expect.append(0.0)
        else:
            continue
        P.append(np.concatenate([np.eye(3).ravel(), tr]))
    P = np.array(P, np.float32)
    d, _ = oracle.distance(A, B, P)
    hit, *_ = oracle.collide(A, B, P)
    tr = P[:, 9:].astype(np.float64)
    exp = np.linalg.norm(np.maximum(np.abs(tr) - half, 0), axis=1)
    assert np.allclose(d, exp, rtol=1e-12, atol=1e-12)
    assert ((hit == 1) == (exp == 0)).all()


def test_convex_icospheres_against_hull_qp():
    opt = pytest.importorskip("scipy.optimize")
    va, ta = synth.icosphere(1, 1.0, 0.0, seed=1)
    vb, tb = synth.icosphere(1, 0.7, 0.0, seed=2)
    A = oracle.BVH(va, ta, 24, 8, 8, 16384)
    B = oracle.BVH(vb, tb, 24, 8, 8, 16384)
    P = synth.poses_box(6, seed=77, lo=1.0, hi=1.6)
    d, _ = oracle.distance(A, B, P)
    for p, dp in zip(P, d):
        R, t = p[:9].reshape(3, 3).astype(np.float64), p[9:].astype(np.float64)
        wb = vb.astype(np.float64) @ R.T + t
        na, nb = len(va), len(wb)
        Va = va.astype(np.float64)

        def f(z):
            r = z[:na] @ Va - z[na:] @ wb
            return float(r @ r)

        def g(z):
            r = z[:na] @ Va - z[na:] @ wb
            return np.concatenate([2 * Va @ r, -2 * wb @ r])
        cons = [{"type": "eq", "fun": lambda z: z[:na].sum() - 1, "jac": lambda z: np.r_[np.ones(na), np.zeros(nb)]},
                {"type": "eq", "fun": lambda z: z[na:].sum() - 1, "jac": lambda z: np.r_[np.zeros(na), np.ones(nb)]}]
        z0 = np.r_[np.full(na, 1 / na), np.full(nb, 1 / nb)]
        r = opt.minimize(f, z0, jac=g, method="SLSQP", bounds=[(0, 1)] * (na + nb), constraints=cons,
                         options={"ftol": 1e-15, "maxiter": 1000})
        assert dp > 0
        assert dp == pytest.approx(math.sqrt(max(r.fun, 0)), rel=1e-4, abs=1e-6)


def test_near_contact_filter_against_brute_force(c1_small):
    c, A, B = c1_small
    va, ta = c["A"]
    vb, tb = c["B"]
    D = synth.scene_diameter(va, vb)
    eps = 1e-3 * D  # a wide band so that several poses are flagged
    near, margin = oracle.near_contact(A, B, c["poses"][:10], eps)
    n_off, n_ij = oracle.near_pairs(A, B, c["poses"][:10], eps)
    for p in range(10):
        pose = c["poses"][p]
        R, t = pose[:9].reshape(3, 3).astype(np.float64), pose[9:].astype(np.float64)
        TA = va.astype(np.float64)[ta]
        TB = vb.astype(np.float64)[tb] @ R.T + t
        lo_a, hi_a = TA.min(1), TA.max(1)
        lo_b, hi_b = TB.min(1), TB.max(1)
        flagged = False
        mmin = math.inf
        amb = []
        for i in range(len(TA)):
            ok = ((lo_a[i] - eps <= hi_b) & (lo_b <= hi_a[i] + eps)).all(1)
            for j in np.nonzero(ok)[0]:
                hit, m = oracle.tri_intersect(TA[i], TB[j])
                q = m if hit else oracle.tri_dist(TA[i], TB[j])
                mmin = min(mmin, q)
                if (hit and m < eps) or (not hit and q <= eps):
                    flagged = True
                    amb.append((i, int(j)))
        assert flagged == bool(near[p])
        assert sorted(amb) == [tuple(x) for x in n_ij[n_off[p]:n_off[p + 1]].tolist()]
        if math.isfinite(mmin) and mmin <= eps:
            assert margin[p] == pytest.approx(mmin, rel=1e-12)



@pytest.mark.parametrize("k,m,bits", [(18, 4, 8), (24, 8, 16), (18, 4, 1), (6, 2, 0)])
def test_refit_bounds_exact_and_encoding_valid(k, m, bits):
    """or_refit (deforming meshes): the tree and lattice exponent stay; every node's lattice
    bounds are the exact floor/ceil (rationals) of the new vertices' projections; the new
    blob decodes, with the independent decoder, to bounds that contain them; refitting back
    to the original vertices restores the original blob byte for byte."""
    v, t = _tiny_mesh(11 + k)
    h = oracle.BVH(v, t, k, m, bits, 4096)
    blob0, e0, tr0 = h.blob(), h.e, h.tree()
    rng = np.random.default_rng(5)
    v2 = (v * 1.1 + rng.uniform(-0.05, 0.05, size=v.shape)).astype(np.float32)
    h.refit(v2)
    assert h.e == e0
    tr = h.tree()
    assert all((tr[key] == tr0[key]).all() for key in tr)
    K = k // 2
    lat = h.lattice()
    sets = [None] * h.n_nodes
    for x in range(h.n_nodes - 1, -1, -1):
        sets[x] = [int(tr["tri"][x])] if tr["nchild"][x] == 0 else \
            sum((sets[tr["first"][x] + c] for c in range(tr["nchild"][x])), [])
    scale = Fraction(2) ** h.e
    for x in range(0, h.n_nodes, 3):
        pts = [v2[i] for tri in sets[x] for i in t[tri]]
        for j in range(K):
            xs = [sum(Fraction(DIRS[j][c]) * Fraction(float(p[c])) for c in range(3)) / scale for p in pts]
            assert lat["exact"][x, j, 0] == math.floor(min(xs)) and lat["exact"][x, j, 1] == math.ceil(max(xs))
    _, f, _ = oracle.decode_blob(h.blob())
    pl = h.placement()
    order = np.lexsort((pl["local"], pl["treelet"]))
    ex = lat["exact"][order].astype(np.float64)
    assert (f[..., 0].astype(np.float64) <= np.ldexp(ex[..., 0], h.e)).all()
    assert (f[..., 1].astype(np.float64) >= np.ldexp(ex[..., 1], h.e)).all()
    h.refit(v)
    assert (h.blob() == blob0).all()


def test_lattice_headroom_exponent():
    """With headroom h the exponent is the smallest with every |d.v| / 2^e < 2^(30 - h)."""
    v, t = _tiny_mesh(4)
    for h_bits in (0, 2, 5):
        h = oracle.BVH(v, t, 18, 4, 8, 4096, headroom=h_bits)
        vals = [sum(Fraction(d[c]) * Fraction(float(p[c])) for c in range(3)) for p in v for d in DIRS[:9]]
        M = max(abs(x) for x in vals)
        assert M / Fraction(2) ** h.e < 2 ** (30 - h_bits)
        assert not (M / Fraction(2) ** (h.e - 1) < 2 ** (30 - h_bits))


def test_refit_rejects_vertices_outside_the_lattice():
    v, t = _tiny_mesh(2)
    h = oracle.BVH(v, t, 18, 4, 8, 4096)
    blob0 = h.blob()
    with pytest.raises(oracle.OracleError):
        h.refit(v * 4096.0)  # far beyond the 2^30 steps of the build's lattice
    bad = v.copy()
    bad[0, 0] = np.nan
    with pytest.raises(oracle.OracleError):
        h.refit(bad)
    assert (h.blob() == blob0).all()
