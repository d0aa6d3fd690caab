"""Python binding of libcbvh, the GB300 engine for compressed k-DOP BVH collision detection
(CD) and proximity query (PQ) -- Tan, Weller & Zachmann, arXiv 2012.05348, Algorithm 1.

Argument marshalling only: every step of a query runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  The functions mirror the C ABI in
include/cbvh.h (cbvh_build, cbvh_collide, cbvh_distance, ...).

Importing fails loudly when libcbvh.so has not been built (``__graft_entry__.build()`` or
``python -m paper_2012_05348_gb300._build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = ["BVH", "Batch", "collide", "distance", "probe_l2_read", "workspace_bytes", "query_stats", "profile_enable", "profile_collect",
           "set_option", "kernel_launches", "OPT_STAGE_BYTES", "OPT_LATTICE_HEADROOM", "OPT_WAIT_CAP", "WAIT_CAP_DEFAULT", "OPT_SPLIT", "OPT_BUDGET0", "OPT_TREELET_PACKING",
           "PACK_TOP_DOWN", "PACK_BOTTOM_UP", "SPLIT_POSE", "SPLIT_ROUNDS", "SPLIT_QUEUE", "SPLIT_ROUNDS_QUEUE", "SPLIT_AUTO",
           "SPLIT_DEFAULT", "BUDGET0_DEFAULT", "CbvhError", "lib", "LIB_PATH", "EARLY_EXIT", "SORT_PAIRS", "ERR"]

# CBVH_CHECKED=1 in the environment loads the checked build (every index the traversal reads
# from a blob or computes is bounds-checked into the status word, CBVH_ERR_CHECK)
LIB_PATH = _build.LIB_CHECKED if os.environ.get("CBVH_CHECKED", "0") not in ("", "0") else _build.LIB
EARLY_EXIT = 1
SORT_PAIRS = 2
ERR = {0: "OK", -1: "ARG", -2: "MESH", -3: "CUDA", -4: "CAPACITY", -5: "STACK", -6: "TIMEOUT", -7: "WORKSPACE",
       -8: "CHECK", -9: "STATE", -10: "IO"}



class _Info(C.Structure):
    _fields_ = [("n_tris", C.c_int64), ("n_nodes", C.c_int64), ("n_treelets", C.c_int64),
                ("blob_bytes", C.c_int64), ("node_bytes", C.c_int64), ("k", C.c_int32), ("branching", C.c_int32),
                ("quant_bits", C.c_int32), ("treelet_bytes", C.c_int32), ("lattice_exp", C.c_int32),
                ("depth", C.c_int32), ("max_treelet_depth", C.c_int32), ("local_bits", C.c_int32)]


def _declare(L):
    P, I64, I32, U32 = C.c_void_p, C.c_int64, C.c_int, C.c_uint32
    L.cbvh_last_error.restype = C.c_char_p
    L.cbvh_build.argtypes = [P, I64, P, I64, I32, I32, I32, I32, C.POINTER(P)]
    L.cbvh_free.argtypes = [P]
    L.cbvh_info.argtypes = [P, C.POINTER(_Info)]
    L.cbvh_blob_host.argtypes = [P, C.POINTER(P), C.POINTER(I64)]
    L.cbvh_attach.argtypes = [P, P, I64, P]
    L.cbvh_decode_all.argtypes = [P, P, P, P]
    L.cbvh_workspace_bytes.argtypes = [P, P, I64, I32, I64, C.POINTER(I64)]
    L.cbvh_collide.argtypes = [P, P, P, I64, P, P, P, I64, P, U32, P, I64, P, P]
    L.cbvh_distance.argtypes = [P, P, P, I64, P, P, I64, P, P]
    L.cbvh_query_stats.argtypes = [P, P, P]
    L.cbvh_distance_noalloc.argtypes = [P, P, P, I64, P, P, P]
    L.cbvh_batch_create.argtypes = [P, I64, C.POINTER(P)]
    L.cbvh_batch_free.argtypes = [P]
    L.cbvh_batch_workspace_bytes.argtypes = [P, C.POINTER(I64)]
    L.cbvh_batch_upload.argtypes = [P, P, I64, P]
    L.cbvh_batch_launch.argtypes = [P, P, I64, P, P]
    L.cbvh_set_option.argtypes = [I32, I64]
    L.cbvh_profile_enable.argtypes = [I32]
    L.cbvh_profile_collect.argtypes = [P, P]
    L.cbvh_kernel_launches.argtypes = [C.POINTER(I64)]
    L.cbvh_refit_workspace_bytes.argtypes = [P, C.POINTER(I64)]
    L.cbvh_refit_prepare.argtypes = [P, P, I64, P]
    L.cbvh_refit.argtypes = [P, P, I64, P, P, I64, P, P]
    L.cbvh_build_plan.argtypes = [I64, I64, I32, I32, I32, I32, C.POINTER(P)]
    L.cbvh_save.argtypes = [P, C.c_char_p]
    L.cbvh_load.argtypes = [C.c_char_p, C.POINTER(P)]
    L.cbvh_build_device_workspace_bytes.argtypes = [P, C.POINTER(I64)]
    L.cbvh_build_device.argtypes = [P, P, P, P, I64, U32, P]
    L.cbvh_probe_l2_read.argtypes = [P, I64, I32, P, P, P]
    for f in ("cbvh_build", "cbvh_free", "cbvh_info", "cbvh_blob_host", "cbvh_attach", "cbvh_decode_all",
              "cbvh_workspace_bytes", "cbvh_collide", "cbvh_distance", "cbvh_query_stats", "cbvh_profile_enable",
              "cbvh_profile_collect", "cbvh_distance_noalloc", "cbvh_batch_create", "cbvh_batch_free",
              "cbvh_batch_workspace_bytes", "cbvh_batch_upload", "cbvh_batch_launch", "cbvh_set_option",
              "cbvh_kernel_launches", "cbvh_refit_workspace_bytes", "cbvh_refit_prepare", "cbvh_refit",
              "cbvh_build_plan", "cbvh_build_device_workspace_bytes", "cbvh_build_device", "cbvh_save",
              "cbvh_load", "cbvh_probe_l2_read"):
        getattr(L, f).restype = I32
    return L


_lib = None


def _load():
    """Load libcbvh.so once; raise if it has not been built (there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2012_05348_gb300._build` "
                              "(the engine has no CPU fallback)")
        _lib = _declare(C.CDLL(LIB_PATH))
    return _lib


def __getattr__(name):
    if name == "lib":
        return _load()
    raise AttributeError(name)


class CbvhError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"cbvh error {code} ({ERR.get(code, '?')}): {msg}")
        self.code = code


def _check(rc: int):
    if rc != 0:
        raise CbvhError(rc, _load().cbvh_last_error().decode())


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


class BVH:
    """A compressed k-DOP BVH: built on the host by cbvh_build, blob resident on the device
    in a torch-allocated buffer attached with cbvh_attach."""

    def __init__(self, verts, tris, k: int = 18, branching: int = 4, quant_bits: int = 16,
                 treelet_bytes: int = 4096, device="cuda"):
        v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
        t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
        h = C.c_void_p()
        _check(_load().cbvh_build(v.ctypes.data_as(C.c_void_p), len(v), t.ctypes.data_as(C.c_void_p), len(t), k,
                              branching, quant_bits, treelet_bytes, C.byref(h)))
        self._h = h
        self.n_verts = len(v)
        self._refresh_info()
        self.blob_dev = None
        if device is not None:
            self.attach(device)

    def _refresh_info(self):
        info = _Info()
        _check(_load().cbvh_info(self._h, C.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _Info._fields_}

    @classmethod
    def plan(cls, n_verts: int, n_tris: int, k: int = 18, branching: int = 4, quant_bits: int = 16,
             treelet_bytes: int = 4096, device="cuda"):
        """cbvh_build_plan: the hierarchy's shape for meshes of n_verts vertices and n_tris
        triangles (host, no mesh data), attached to a device buffer; fill it with
        build_device.  Queries refuse it until a device build succeeds."""
        self = cls.__new__(cls)
        h = C.c_void_p()
        _check(_load().cbvh_build_plan(int(n_verts), int(n_tris), k, branching, quant_bits, treelet_bytes,
                                       C.byref(h)))
        self._h = h
        self.n_verts = int(n_verts)
        self._refresh_info()
        self.blob_dev = None
        if device is not None:
            self.attach(device)
        return self

    def save(self, path: str) -> None:
        """cbvh_save: the hierarchy (its host blob and vertex count) to a file."""
        _check(_load().cbvh_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, device="cuda"):
        """cbvh_load: a hierarchy written by save, checked before it is accepted, attached
        to `device` (None: host only)."""
        self = cls.__new__(cls)
        h = C.c_void_p()
        _check(_load().cbvh_load(os.fsencode(path), C.byref(h)))
        self._h = h
        with open(path, "rb") as f:
            self.n_verts = int.from_bytes(f.read(16)[8:16], "little", signed=True)
        self._refresh_info()
        self.blob_dev = None
        if device is not None:
            self.attach(device)
        return self

    @classmethod
    def on_device(cls, verts, tris, k: int = 18, branching: int = 4, quant_bits: int = 16,
                  treelet_bytes: int = 4096, host_copy: bool = True, stream=None):
        """A hierarchy built on the GPU (cbvh_build_plan + cbvh_build_device) from device
        tensors verts float32 (n_verts, 3) and tris int32 (n_tris, 3)."""
        b = cls.plan(int(verts.shape[0]), int(tris.shape[0]), k, branching, quant_bits, treelet_bytes,
                     device=verts.device)
        return b.build_device(verts, tris, host_copy=host_copy, stream=stream)

    def build_device(self, verts, tris, host_copy: bool = True, stream=None):
        """cbvh_build_device: (re)build this plan's hierarchy on the GPU from device tensors
        verts float32 (n_verts, 3) and tris int32 (n_tris, 3) of the plan's counts.  The
        blob is byte-identical to the host build's; host_copy also refreshes blob_host()."""
        torch = _torch()
        if self.blob_dev is None:
            raise CbvhError(-9, "not attached")
        for name, t, dt, n in (("verts", verts, torch.float32, self.n_verts), ("tris", tris, torch.int32,
                                                                              self.info["n_tris"])):
            if (t.dtype != dt or t.device != self.blob_dev.device or not t.is_contiguous() or t.dim() != 2
                    or t.shape[1] != 3 or t.shape[0] != n):
                raise ValueError(f"{name}: need a contiguous {dt} tensor of shape ({n}, 3) on {self.blob_dev.device}")
        if getattr(self, "_build_ws", None) is None:
            nb = C.c_int64()
            _check(_load().cbvh_build_device_workspace_bytes(self._h, C.byref(nb)))
            self._build_ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=self.blob_dev.device)
        with torch.cuda.device(self.blob_dev.device):
            _check(_load().cbvh_build_device(self._h, _ptr(verts), _ptr(tris), _ptr(self._build_ws),
                                             self._build_ws.numel(), 1 if host_copy else 0, _stream_ptr(stream)))
        self._refit_ws = self._build_ws  # the build prepared the refit plan at the workspace's front
        self._refresh_info()
        return self

    @property
    def handle(self):
        return self._h

    def blob_host(self) -> np.ndarray:
        p, n = C.c_void_p(), C.c_int64()
        _check(_load().cbvh_blob_host(self._h, C.byref(p), C.byref(n)))
        return np.ctypeslib.as_array((C.c_uint8 * n.value).from_address(p.value)).copy()

    def attach(self, device="cuda", stream=None):
        torch = _torch()
        n = self.info["blob_bytes"]
        self.blob_dev = torch.empty(n, dtype=torch.uint8, device=device)
        with torch.cuda.device(self.blob_dev.device):
            _check(_load().cbvh_attach(self._h, _ptr(self.blob_dev), n, _stream_ptr(stream)))

    def refit(self, verts, tris, stream=None, check: bool = True):
        """cbvh_refit (deforming meshes): new positions for the build's vertices, device
        float32 (n_verts, 3); tris: the build's triangles, device int32 (n_tris, 3).  The
        attached blob is rewritten in place; the plan is prepared on first use."""
        torch = _torch()
        if self.blob_dev is None:
            raise CbvhError(-9, "not attached")
        if getattr(self, "_refit_ws", None) is None:
            nb = C.c_int64()
            _check(_load().cbvh_refit_workspace_bytes(self._h, C.byref(nb)))
            self._refit_ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=self.blob_dev.device)
            _check(_load().cbvh_refit_prepare(self._h, _ptr(self._refit_ws), self._refit_ws.numel(),
                                              _stream_ptr(stream)))
        status = torch.zeros(1, dtype=torch.int32, device=self.blob_dev.device)
        _check(_load().cbvh_refit(self._h, _ptr(verts), int(verts.shape[0]), _ptr(tris), _ptr(self._refit_ws),
                                  self._refit_ws.numel(), _ptr(status), _stream_ptr(stream)))
        if check:
            code = int(status.item())
            if code != 0:
                raise CbvhError(code, "device status")
        return status

    def decode_all(self, stream=None):
        """(lattice int32 (n, K, 2) or None, bounds float32 (n, K, 2)) on the device, blob order."""
        torch = _torch()
        n, K = self.info["n_nodes"], self.info["k"] // 2
        dev = self.blob_dev.device
        lat = torch.empty((n, K, 2), dtype=torch.int32, device=dev) if self.info["quant_bits"] else None
        f = torch.empty((n, K, 2), dtype=torch.float32, device=dev)
        _check(_load().cbvh_decode_all(self._h, _ptr(lat), _ptr(f), _stream_ptr(stream)))
        return lat, f

    def close(self):
        if getattr(self, "_h", None):
            _load().cbvh_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


OPT_STAGE_BYTES = 1
OPT_SPLIT = 2
OPT_BUDGET0 = 3
OPT_TREELET_PACKING = 4
OPT_LATTICE_HEADROOM = 5
OPT_WAIT_CAP = 6
WAIT_CAP_DEFAULT = 1 << 24
PACK_TOP_DOWN, PACK_BOTTOM_UP = 0, 1
# quant_bits values besides the delta widths 8 and 16
QUANT_FP32, QUANT_FP16, QUANT_SVB = 0, 1, 2
# CBVH_OPT_SPLIT values: warp per pose, rounds, work queue, rounds then work queue, and the
# default (work queue for collision with pair lists, rounds then work queue otherwise)
SPLIT_POSE, SPLIT_ROUNDS, SPLIT_QUEUE, SPLIT_ROUNDS_QUEUE, SPLIT_AUTO = 0, 1, 2, 3, 4
SPLIT_DEFAULT = SPLIT_AUTO
BUDGET0_DEFAULT = 256


def kernel_launches() -> int:
    """cbvh_kernel_launches: kernels the library has launched in this process so far."""
    out = C.c_int64()
    _check(_load().cbvh_kernel_launches(C.byref(out)))
    return out.value


def set_option(option: int, value: int) -> None:
    """cbvh_set_option: process-wide options (OPT_STAGE_BYTES, OPT_SPLIT, OPT_BUDGET0,
    OPT_TREELET_PACKING, OPT_LATTICE_HEADROOM, OPT_WAIT_CAP)."""
    _check(_load().cbvh_set_option(int(option), int(value)))


class _Query(C.Structure):
    _fields_ = [("A", C.c_void_p), ("B", C.c_void_p), ("mode", C.c_int32), ("flags", C.c_uint32),
                ("poses", C.c_void_p), ("n", C.c_int64), ("hit", C.c_void_p), ("dist", C.c_void_p),
                ("any_hit", C.c_void_p), ("min_dist", C.c_void_p)]


class Batch:
    """A batched query (cbvh_batch_*): many (A, B, kind, poses) work items run in one set of
    persistent launches.  Each item is a dict with keys A, B (BVH), kind ('collide' or
    'distance'), poses (device float32 (n, 12)) and, for collisions, early_exit (bool) and
    set (any hashable): collision items with the same set share one per-pose flag,
    ``any_hit[set]``, that is 1 iff some item of the set intersects at that pose, and each
    pose stops as soon as one item of its set intersects (the links of one robot over one
    list of configurations); distance items with the same set share one per-pose minimum,
    ``min_dist[set]``, the smallest distance over the set's items, and each item prunes
    with the set's best distance so far.  Outputs are allocated here: ``outputs[i]`` is
    uint8 hit flags or float32 distances (with a set, an item's flag may be 0 where another
    item of the set hit first, and an item's distance is only exact where it is the set's
    minimum).  ``launch()`` only enqueues work on the stream, so it can be captured in a
    CUDA graph."""

    def __init__(self, items, device="cuda"):
        torch = _torch()
        self.items = items
        self.outputs = []
        self.any_hit = {}
        self.min_dist = {}
        arr = (_Query * max(1, len(items)))()
        for i, it in enumerate(items):
            poses = it["poses"]
            n = int(poses.shape[0])
            kind = 1 if it["kind"] == "distance" else 0
            if kind == 0:
                out = torch.empty(n, dtype=torch.uint8, device=device)
                anyp = None
                if it.get("set") is not None:
                    if it["set"] not in self.any_hit:
                        self.any_hit[it["set"]] = torch.zeros(n, dtype=torch.uint8, device=device)
                    anyp = self.any_hit[it["set"]].data_ptr()
                arr[i] = _Query(it["A"].handle, it["B"].handle, 0, EARLY_EXIT if it.get("early_exit") else 0,
                                poses.data_ptr(), n, out.data_ptr(), None, anyp)
            else:
                out = torch.empty(n, dtype=torch.float32, device=device)
                mind = None
                if it.get("set") is not None:
                    if it["set"] not in self.min_dist:
                        self.min_dist[it["set"]] = torch.empty(n, dtype=torch.float32, device=device)
                    mind = self.min_dist[it["set"]].data_ptr()
                arr[i] = _Query(it["A"].handle, it["B"].handle, 1, 0, poses.data_ptr(), n, None, out.data_ptr(), None,
                                mind)
            self.outputs.append(out)
        self._arr = arr
        h = C.c_void_p()
        _check(_load().cbvh_batch_create(arr, len(items), C.byref(h)))
        self._h = h
        nb = C.c_int64()
        _check(_load().cbvh_batch_workspace_bytes(h, C.byref(nb)))
        self.workspace = torch.empty(nb.value, dtype=torch.uint8, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        _check(_load().cbvh_batch_upload(h, _ptr(self.workspace), nb.value, _stream_ptr(None)))

    def launch(self, stream=None):
        _check(_load().cbvh_batch_launch(self._h, _ptr(self.workspace), self.workspace.numel(), _ptr(self.status),
                                         _stream_ptr(stream)))

    def run(self, stream=None):
        self.launch(stream)
        code = int(self.status.item())
        if code != 0:
            raise CbvhError(code, "device status")
        return self.outputs

    def close(self):
        if getattr(self, "_h", None):
            _load().cbvh_batch_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


def workspace_bytes(A: BVH, B: BVH, n: int, mode: int, pair_capacity: int = 0) -> int:
    out = C.c_int64()
    _check(_load().cbvh_workspace_bytes(A.handle, B.handle, n, mode, pair_capacity, C.byref(out)))
    return out.value


@dataclass
class CollideResult:
    hit: object          # uint8 (n,)
    offsets: object      # int64 (n + 1,) or None
    pairs: object        # int32 (P, 2) or None
    status: int


def collide(A: BVH, B: BVH, poses, *, pairs: bool = True, sort: bool = True, early_exit: bool = False,
            capacity: int | None = None, stream=None, out=None, check: bool = True) -> CollideResult:
    """cbvh_collide on device poses (n, 12) float32.  With ``pairs`` the per-pose intersecting
    triangle pairs come back in CSR form; if the capacity is exceeded the call is repeated
    once with the exact size the device reported."""
    torch = _torch()
    n = int(poses.shape[0])
    dev = poses.device
    flags = (EARLY_EXIT if early_exit else 0) | (SORT_PAIRS if (pairs and sort) else 0)
    st = _stream_ptr(stream)
    cap = int(capacity if capacity is not None else max(1024, 16 * n)) if pairs else 0
    for _attempt in range(2):
        hit = torch.empty(n, dtype=torch.uint8, device=dev)
        off = torch.empty(n + 1, dtype=torch.int64, device=dev) if pairs else None
        prs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev) if pairs else None
        need = torch.zeros(1, dtype=torch.int64, device=dev) if pairs else None
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        wsb = workspace_bytes(A, B, n, 0, cap)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        _check(_load().cbvh_collide(A.handle, B.handle, _ptr(poses), n, _ptr(hit), _ptr(off), _ptr(prs), cap, _ptr(need),
                                flags, _ptr(ws), wsb, _ptr(status), st))
        code = int(status.item())
        if code == -4 and pairs:
            cap = int(need.item())
            continue
        if check and code != 0:
            raise CbvhError(code, "device status")
        total = int(need.item()) if pairs else 0
        return CollideResult(hit, off, prs[:total] if pairs else None, code)
    raise CbvhError(-4, "pair capacity still exceeded after resizing")


def query_stats(workspace, stream=None):
    """(BV-pair tests, leaf tests, expansions) of the last query that used this workspace."""
    out = np.zeros(3, np.int64)
    _check(_load().cbvh_query_stats(_ptr(workspace), out.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
    return int(out[0]), int(out[1]), int(out[2])


def profile_enable(on: bool = True):
    """Time every later traversal kernel launch of this thread with library-owned events."""
    _check(_load().cbvh_profile_enable(int(bool(on))))


def profile_collect():
    """{'collide' | 'distance' | 'compaction': (ms, queries)} since the last collect."""
    ms = np.zeros(3)
    n = np.zeros(3, np.int64)
    _check(_load().cbvh_profile_collect(ms.ctypes.data_as(C.c_void_p), n.ctypes.data_as(C.c_void_p)))
    return {"collide": (float(ms[0]), int(n[0])), "distance": (float(ms[1]), int(n[1])),
            "compaction": (float(ms[2]), int(n[2]))}


def probe_l2_read(nbytes: int = 64 << 20, reps: int = 20, device="cuda", stream=None) -> float:
    """cbvh_probe_l2_read: L2 read bandwidth (GB/s) streaming an nbytes device buffer."""
    torch = _torch()
    buf = torch.ones(nbytes // 4, dtype=torch.int32, device=device)
    sink = torch.zeros(1, dtype=torch.int32, device=device)
    out = C.c_double()
    with torch.cuda.device(buf.device):
        _check(_load().cbvh_probe_l2_read(_ptr(buf), nbytes, reps, _ptr(sink), C.byref(out), _stream_ptr(stream)))
    return out.value


def distance(A: BVH, B: BVH, poses, *, stream=None, check: bool = True):
    """cbvh_distance on device poses (n, 12) float32 -> float32 (n,)."""
    torch = _torch()
    n = int(poses.shape[0])
    dev = poses.device
    dist = torch.empty(n, dtype=torch.float32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    wsb = workspace_bytes(A, B, n, 1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    _check(_load().cbvh_distance(A.handle, B.handle, _ptr(poses), n, _ptr(dist), _ptr(ws), wsb, _ptr(status),
                             _stream_ptr(stream)))
    if check:
        code = int(status.item())
        if code != 0:
            raise CbvhError(code, "device status")
    return dist
