"""FP64 CPU oracle for compressed k-DOP BVH collision detection and proximity query.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline
leg are the only callers.  The CUDA engine never imports this package, and this package
never imports the engine; the two share no code.  See ``oracle.c`` for what each function
computes and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
# Treelet formation: 0 grows treelets top-down (breadth-first from each root), 1 packs them
# bottom-up (a subtree joins its parent's treelet while it fits).  Blobs are compared with
# the library's at equal packing.
PACKING_TOP_DOWN, PACKING_BOTTOM_UP = 0, 1
PACKING_DEFAULT = PACKING_TOP_DOWN


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, FP64, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
        L.or_last_error.restype = C.c_char_p
        L.or_build.argtypes = [P, I64, P, I64, I32, I32, I32, I32, I32, I32, C.POINTER(C.c_void_p)]
        L.or_build.restype = I32
        L.or_free.argtypes = [P]
        L.or_info.argtypes = [P, P]
        L.or_blob.argtypes = [P]
        L.or_blob.restype = C.c_void_p
        L.or_tree.argtypes = [P, P, P, P, P]
        L.or_lattice.argtypes = [P, P, P, P, P]
        L.or_placement.argtypes = [P, P, P, P, P]
        L.or_refit.argtypes = [P, P]
        L.or_refit.restype = I32
        L.or_decode_blob.argtypes = [P, I64, P, P, P]
        L.or_decode_blob.restype = I64
        L.or_floor_sum3.argtypes = [D, D, D]
        L.or_floor_sum3.restype = I64
        L.or_ceil_sum3.argtypes = [D, D, D]
        L.or_ceil_sum3.restype = I64
        L.or_half_rd.argtypes = [D]
        L.or_half_rd.restype = C.c_uint32
        L.or_half_ru.argtypes = [D]
        L.or_half_ru.restype = C.c_uint32
        L.or_half_value.argtypes = [C.c_uint32]
        L.or_half_value.restype = D
        L.or_lattice_dv.argtypes = [P, I32, I32, P, P]
        L.or_svb_encode.argtypes = [P, I32, P, P]
        L.or_svb_encode.restype = I32
        L.or_tri_intersect.argtypes = [P, P, P]
        L.or_tri_intersect.restype = I32
        L.or_tri_dist.argtypes = [P, P]
        L.or_tri_dist.restype = D
        L.or_pt_tri.argtypes = [P, P]
        L.or_pt_tri.restype = D
        L.or_seg_seg.argtypes = [P, P, P, P]
        L.or_seg_seg.restype = D
        L.or_collide.argtypes = [P, P, P, I64, I32, P, P, I32, P]
        L.or_collide.restype = C.c_void_p
        L.or_brute_collide.argtypes = [P, P, P, I64, P, P]
        L.or_brute_collide.restype = C.c_void_p
        L.or_distance.argtypes = [P, P, P, I64, I32, P, P]
        L.or_brute_distance.argtypes = [P, P, P, I64, P]
        L.or_near_contact.argtypes = [P, P, P, I64, D, P, P]
        L.or_near_pairs.argtypes = [P, P, P, I64, D, P]
        L.or_near_pairs.restype = C.c_void_p
        L.or_pairs_total.argtypes = [P]
        L.or_pairs_total.restype = I64
        L.or_pairs_copy.argtypes = [P, P, P]
        L.or_pairs_free.argtypes = [P]
        L.or_num_threads.restype = I32
        L.or_set_threads.argtypes = [I32]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


class BVH:
    """The oracle's BVH of one mesh: its tree, exact lattice bounds, encoding and blob."""

    def __init__(self, verts, tris, k: int, m: int, bits: int, treelet_bytes: int, packing: int = PACKING_DEFAULT,
                 headroom: int = 0):
        L = lib()
        self.verts = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
        h = C.c_void_p()
        rc = L.or_build(_p(self.verts), len(self.verts), _p(self.tris), len(self.tris), k, m, bits,
                        treelet_bytes, packing, headroom, C.byref(h))
        if rc != 0:
            raise OracleError(rc, L.or_last_error().decode())
        self._h = h
        info = np.zeros(10, np.int64)
        L.or_info(h, _p(info))
        (self.n_nodes, self.n_treelets, self.e, self.depth, self.blob_bytes, self.lbits,
         self.max_tdepth, self.K, self.rec_bytes, self.root_bytes) = (int(x) for x in info)
        self.k, self.m, self.bits, self.treelet_bytes, self.packing = k, m, bits, treelet_bytes, packing

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_free(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def refit(self, verts) -> None:
        """New positions for the build's vertices: same tree, treelets and lattice exponent;
        exact bounds, encoding and blob redone (or_refit)."""
        v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
        if v.shape != self.verts.shape:
            raise ValueError("refit needs the build's vertex count")
        rc = lib().or_refit(self._h, _p(v))
        if rc != 0:
            raise OracleError(rc, lib().or_last_error().decode())
        self.verts = v

    def blob(self) -> np.ndarray:
        ptr = lib().or_blob(self._h)
        return np.ctypeslib.as_array((C.c_uint8 * self.blob_bytes).from_address(ptr)).copy()

    def tree(self):
        n = self.n_nodes
        par, first, nch, tri = (np.empty(n, np.int32) for _ in range(4))
        lib().or_tree(self._h, _p(par), _p(first), _p(nch), _p(tri))
        return dict(parent=par, first=first, nchild=nch, tri=tri)

    def lattice(self):
        """exact / decoded lattice (int64), decoded FP32 bounds, FP64 bounds: each (n, K, 2)."""
        s = (self.n_nodes, self.K, 2)
        ex, dec, f, b = np.empty(s, np.int64), np.empty(s, np.int64), np.empty(s, np.float32), np.empty(s)
        lib().or_lattice(self._h, _p(ex), _p(dec), _p(f), _p(b))
        return dict(exact=ex, decoded=dec, decf=f, fp64=b)

    def placement(self):
        n = self.n_nodes
        tl, lo, ext = np.empty(n, np.int32), np.empty(n, np.int32), np.empty(n, np.uint8)
        delta = np.empty((n, self.K, 2), np.uint32)
        lib().or_placement(self._h, _p(tl), _p(lo), _p(ext), _p(delta))
        return dict(treelet=tl, local=lo, ext=ext, delta=delta)


def decode_blob(blob: np.ndarray):
    """Independent decode of a blob: (lattice int32 (n,K,2), FP32 bounds (n,K,2), meta (n,4)),
    nodes in blob order."""
    blob = np.ascontiguousarray(blob, dtype=np.uint8)
    K = int(blob[7])
    n = int.from_bytes(blob[20:24].tobytes(), "little")
    lat = np.zeros((n, K, 2), np.int32)
    f = np.zeros((n, K, 2), np.float32)
    meta = np.zeros((n, 4), np.uint32)
    got = lib().or_decode_blob(_p(blob), len(blob), _p(lat), _p(f), _p(meta))
    if got != n:
        raise OracleError(int(got), lib().or_last_error().decode())
    return lat, f, meta


def _poses(P):
    return np.ascontiguousarray(P, dtype=np.float32).reshape(-1, 12)


def _take_pairs(handle, n):
    L = lib()
    tot = L.or_pairs_total(handle)
    off = np.zeros(n + 1, np.int64)
    ij = np.zeros((max(tot, 1), 2), np.int32)
    L.or_pairs_copy(handle, _p(off), _p(ij))
    L.or_pairs_free(handle)
    return off, ij[:tot]


def collide(A: BVH, B: BVH, poses, use_decoded: bool = False):
    """Algorithm 1 CD: (hit uint8 (n,), offsets int64 (n+1,), pairs int32 (P, 2), stats)."""
    P = _poses(poses)
    n = len(P)
    hit = np.zeros(n, np.uint8)
    cnt = np.zeros(n, np.int64)
    st = np.zeros(2, np.int64)
    h = lib().or_collide(A.handle, B.handle, _p(P), n, int(use_decoded), _p(hit), _p(cnt), 1, _p(st))
    off, ij = _take_pairs(h, n)
    return hit, off, ij, dict(bv_tests=int(st[0]), leaf_tests=int(st[1]))


def brute_collide(A: BVH, B: BVH, poses):
    P = _poses(poses)
    n = len(P)
    hit = np.zeros(n, np.uint8)
    cnt = np.zeros(n, np.int64)
    h = lib().or_brute_collide(A.handle, B.handle, _p(P), n, _p(hit), _p(cnt))
    off, ij = _take_pairs(h, n)
    return hit, off, ij


def distance(A: BVH, B: BVH, poses, use_decoded: bool = False):
    P = _poses(poses)
    d = np.zeros(len(P))
    st = np.zeros(2, np.int64)
    lib().or_distance(A.handle, B.handle, _p(P), len(P), int(use_decoded), _p(d), _p(st))
    return d, dict(bv_tests=int(st[0]), leaf_tests=int(st[1]))


def brute_distance(A: BVH, B: BVH, poses):
    P = _poses(poses)
    d = np.zeros(len(P))
    lib().or_brute_distance(A.handle, B.handle, _p(P), len(P), _p(d))
    return d


def near_contact(A: BVH, B: BVH, poses, eps: float):
    P = _poses(poses)
    near = np.zeros(len(P), np.uint8)
    margin = np.zeros(len(P))
    lib().or_near_contact(A.handle, B.handle, _p(P), len(P), float(eps), _p(near), _p(margin))
    return near.astype(bool), margin


def near_pairs(A: BVH, B: BVH, poses, eps: float):
    """Per pose, the triangle pairs within eps of a contact decision: (offsets, pairs)."""
    P = _poses(poses)
    cnt = np.zeros(len(P), np.int64)
    h = lib().or_near_pairs(A.handle, B.handle, _p(P), len(P), float(eps), _p(cnt))
    return _take_pairs(h, len(P))


def _tri(T):
    return np.ascontiguousarray(T, dtype=np.float64).reshape(3, 3)


def tri_intersect(T1, T2):
    """(hit, margin) of the closed triangle-triangle intersection test."""
    m = np.zeros(1)
    h = lib().or_tri_intersect(_p(_tri(T1)), _p(_tri(T2)), _p(m))
    return bool(h), float(m[0])


def tri_dist(T1, T2) -> float:
    return float(lib().or_tri_dist(_p(_tri(T1)), _p(_tri(T2))))


def pt_tri(p, T) -> float:
    return float(lib().or_pt_tri(_p(np.ascontiguousarray(p, np.float64)), _p(_tri(T))))


def seg_seg(a, b, c, d) -> float:
    f = lambda x: _p(np.ascontiguousarray(x, np.float64))  # noqa: E731
    return float(lib().or_seg_seg(f(a), f(b), f(c), f(d)))


# quant_bits value of the half-precision descriptor mode
QUANT_FP16 = 1
# quant_bits value of the Stream VByte mode: exact lattice deltas to the parent, 1-4 bytes each
QUANT_SVB = 2


def svb_encode(values) -> tuple[bytes, bytes]:
    """Stream VByte coding of up to 32 unsigned 32-bit values: (8-byte control word, data)."""
    v = np.ascontiguousarray(values, dtype=np.uint32)
    if len(v) > 32:
        raise ValueError("at most 32 values per control word")
    ctl = np.zeros(8, np.uint8)
    data = np.zeros(4 * max(len(v), 1), np.uint8)
    n = lib().or_svb_encode(_p(v), len(v), _p(ctl), _p(data))
    return ctl.tobytes(), data[:n].tobytes()


def half_rd(v: float) -> int:
    """Bits of the largest IEEE binary16 value <= v."""
    return int(lib().or_half_rd(float(v)))


def half_ru(v: float) -> int:
    """Bits of the smallest IEEE binary16 value >= v."""
    return int(lib().or_half_ru(float(v)))


def half_value(bits: int) -> float:
    """Value of an IEEE binary16 bit pattern."""
    return float(lib().or_half_value(int(bits)))


def floor_sum3(a: float, b: float, c: float) -> int:
    return int(lib().or_floor_sum3(a, b, c))


def ceil_sum3(a: float, b: float, c: float) -> int:
    return int(lib().or_ceil_sum3(a, b, c))


def lattice_dv(v, j: int, e: int):
    v = np.ascontiguousarray(v, np.float32)
    lo, hi = np.zeros(1, np.int64), np.zeros(1, np.int64)
    lib().or_lattice_dv(_p(v), j, e, _p(lo), _p(hi))
    return int(lo[0]), int(hi[0])


def filtered_poses(A: BVH, B: BVH, draw, n: int, eps: float, max_rounds: int = 50):
    """Keep drawing candidate poses with ``draw(count, round)`` and drop the ones the
    near-contact filter flags, until ``n`` remain (deterministic for a deterministic draw)."""
    keep = []
    have = 0
    for r in range(max_rounds):
        cand = _poses(draw(max(16, 2 * (n - have)), r))
        near, _ = near_contact(A, B, cand, eps)
        good = cand[~near]
        keep.append(good)
        have += len(good)
        if have >= n:
            break
    P = np.concatenate(keep)[:n]
    if len(P) < n:
        raise RuntimeError("near-contact filter rejected too many poses")
    return P
