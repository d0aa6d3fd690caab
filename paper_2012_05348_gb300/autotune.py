"""Autotuner for the traversal engine.

Picks, for a pair of meshes and a query kind, the hierarchy parameters (branching factor,
treelet budget, quantisation bits) and the launch options (shared-memory treelet staging,
warp-per-pose or warp-per-node-pair mapping) that serve a sample of poses fastest on the
current GPU.  Every candidate is timed on the device (library-owned CUDA events around the
traversal kernels) after a warm-up; results are cached in a JSON file keyed by a hash of
the meshes, k and the query kind, so a later call returns at once.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import numpy as np

from . import (BUDGET0_DEFAULT, BVH, OPT_BUDGET0, OPT_SPLIT, OPT_STAGE_BYTES, OPT_TREELET_PACKING, PACK_TOP_DOWN,
               SPLIT_DEFAULT, collide, distance, profile_collect, profile_enable, set_option)

DEFAULT_SPACE = dict(branching=(4, 8, 16), treelet_bytes=(4096, 16384, 65536), quant_bits=(8, 16),
                     stage_bytes=(0, 16384), split=(4, 1, 2, 3, 0), budget0=(64, 256, 1024))


def mesh_key(verts_a, tris_a, verts_b, tris_b, k: int, kind: str) -> str:
    h = hashlib.sha1()
    for arr in (verts_a, tris_a, verts_b, tris_b):
        a = np.ascontiguousarray(arr)
        h.update(str(a.shape).encode())
        h.update(a.tobytes())
    h.update(f"k={k};kind={kind}".encode())
    return h.hexdigest()


def _time(fn, reps: int) -> float:
    fn()  # warm-up
    profile_collect()
    profile_enable(True)
    for _ in range(reps):
        fn()
    profile_enable(False)
    r = profile_collect()
    ms = r["collide"][0] + r["distance"][0]
    return ms / reps


def autotune(mesh_a, mesh_b, poses, k: int = 24, kind: str = "collide", early_exit: bool = False,
             space: dict | None = None, cache: str | None = None, reps: int = 2, device="cuda"):
    """Return (best config dict, list of (config, ms) for every candidate timed).

    mesh_a / mesh_b: (verts, tris); poses: device float32 (n, 12) sample of the workload."""
    space = dict(DEFAULT_SPACE, **(space or {}))
    key = mesh_key(*mesh_a, *mesh_b, k, kind + ("/early" if early_exit else ""))
    store = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            store = json.load(f)
        if key in store:
            return store[key]["best"], store[key]["trials"]
    trials = []
    for m, tb, bits in itertools.product(space["branching"], space["treelet_bytes"], space["quant_bits"]):
        try:
            A = BVH(*mesh_a, k, m, bits, tb, device=device)
            B = BVH(*mesh_b, k, m, bits, tb, device=device)
        except Exception:  # budget too small for this branching and k
            continue
        for stage, split, b0 in itertools.product(space["stage_bytes"], space["split"], space["budget0"]):
            if not split and b0 != space["budget0"][0]:
                continue  # the budget only matters when tasks are handed on
            set_option(OPT_STAGE_BYTES, stage)
            set_option(OPT_SPLIT, split)
            set_option(OPT_BUDGET0, b0)
            if kind == "collide":
                fn = lambda: collide(A, B, poses, pairs=False, early_exit=early_exit)  # noqa: E731
            else:
                fn = lambda: distance(A, B, poses)  # noqa: E731
            ms = _time(fn, reps)
            trials.append((dict(branching=m, treelet_bytes=tb, quant_bits=bits, stage_bytes=stage, split=split,
                                budget0=b0), ms))
    apply({})
    best = min(trials, key=lambda t: t[1])[0]
    if cache:
        store[key] = dict(best=best, trials=trials)
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1)
        os.replace(tmp, cache)
    return best, trials


def apply(config: dict) -> None:
    """Set the launch options of a tuned configuration (the hierarchy parameters are used when
    building the BVHs); an empty dict restores the defaults."""
    set_option(OPT_STAGE_BYTES, int(config.get("stage_bytes", 0)))
    set_option(OPT_SPLIT, int(config.get("split", SPLIT_DEFAULT)))
    set_option(OPT_BUDGET0, int(config.get("budget0", BUDGET0_DEFAULT)))
