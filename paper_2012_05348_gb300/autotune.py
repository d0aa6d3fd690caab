"""Autotuner for the traversal engine.

Picks, for a workload (one pair of meshes, or a static scene and the links of a robot run
as one batch) and a query kind, the hierarchy parameters (branching factor, treelet budget,
quantisation bits, treelet packing) and the launch options (shared-memory treelet staging,
work mapping, task budget) that serve a sample of poses fastest on the current GPU.

The search has two stages: every hierarchy candidate is built and timed under the default
launch options, then the launch options are searched on the best hierarchy (the options do
not change the hierarchy, and the two interact little).  ``exhaustive=True`` times the full
product instead.  Every candidate is timed on the device (library-owned CUDA events around
the traversal kernels) after a warm-up.  Results are cached in a JSON file keyed by a hash
of the meshes, k, the query kind and the search space, so a later call returns at once.
Tuning changes scheduling and layout only; every candidate returns the same results.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import numpy as np

from . import (BUDGET0_DEFAULT, BVH, OPT_BUDGET0, OPT_SPLIT, OPT_STAGE_BYTES, OPT_TREELET_PACKING, PACK_TOP_DOWN,
               SPLIT_DEFAULT, Batch, collide, distance, profile_collect, profile_enable, set_option)

DEFAULT_SPACE = dict(branching=(4, 8, 16), treelet_bytes=(4096, 16384, 65536), quant_bits=(8, 16),
                     packing=(PACK_TOP_DOWN,), stage_bytes=(0, 16384), split=(4, 1, 2, 3, 0),
                     budget0=(64, 256, 1024))
HIERARCHY_KEYS = ("branching", "treelet_bytes", "quant_bits", "packing")
LAUNCH_KEYS = ("stage_bytes", "split", "budget0")
DEFAULT_LAUNCH = dict(stage_bytes=0, split=SPLIT_DEFAULT, budget0=BUDGET0_DEFAULT)


def mesh_key(meshes, k: int, kind: str, space: dict) -> str:
    h = hashlib.sha1()
    for verts, tris in meshes:
        for arr in (verts, tris):
            a = np.ascontiguousarray(arr)
            h.update(str(a.shape).encode())
            h.update(a.tobytes())
    h.update(f"k={k};kind={kind};space={json.dumps(space, sort_keys=True)}".encode())
    return h.hexdigest()


def _time(fn, reps: int) -> float:
    fn()  # warm-up
    profile_collect()
    profile_enable(True)
    for _ in range(reps):
        fn()
    profile_enable(False)
    r = profile_collect()
    return (r["collide"][0] + r["distance"][0]) / reps


def apply(config: dict) -> None:
    """Set the launch options and the treelet packing of a tuned configuration (the other
    hierarchy parameters are arguments of the BVH builds); an empty dict restores the
    defaults."""
    set_option(OPT_STAGE_BYTES, int(config.get("stage_bytes", 0)))
    set_option(OPT_SPLIT, int(config.get("split", SPLIT_DEFAULT)))
    set_option(OPT_BUDGET0, int(config.get("budget0", BUDGET0_DEFAULT)))
    set_option(OPT_TREELET_PACKING, int(config.get("packing", PACK_TOP_DOWN)))


def _search(build, make_fn, space: dict, reps: int, exhaustive: bool):
    """build(m, treelet_bytes, bits) -> objects (or raises for an invalid combination);
    make_fn(objects) -> the timed callable.  Returns (best config, trials)."""
    trials = []
    hier = list(itertools.product(*(space[k] for k in HIERARCHY_KEYS)))
    launch = [lo for lo in itertools.product(*(space[k] for k in LAUNCH_KEYS))
              if lo[1] != 0 or lo[2] == space["budget0"][0]]  # the budget is unused at split 0
    built = {}

    def objects(h):
        if h not in built:
            m, tb, bits, pk = h
            set_option(OPT_TREELET_PACKING, pk)
            try:
                built[h] = build(m, tb, bits)
            except Exception:  # e.g. a treelet budget too small for this branching and k
                built[h] = None
            finally:
                set_option(OPT_TREELET_PACKING, PACK_TOP_DOWN)
        return built[h]

    def timed(h, lo):
        obj = objects(h)
        if obj is None:
            return None
        cfg = dict(zip(HIERARCHY_KEYS, h), **dict(zip(LAUNCH_KEYS, lo)))
        apply(cfg)
        try:
            ms = _time(make_fn(obj), reps)
        finally:
            apply({})
        trials.append((cfg, ms))
        return ms

    try:
        if exhaustive:
            for h in hier:
                for lo in launch:
                    timed(h, lo)
        else:
            d = tuple(DEFAULT_LAUNCH[k] for k in LAUNCH_KEYS)
            scores = {h: timed(h, d) for h in hier}
            scores = {h: v for h, v in scores.items() if v is not None}
            if not scores:
                raise RuntimeError("no candidate hierarchy could be built")
            best_h = min(scores, key=scores.get)
            # keep only the best hierarchy's objects alive for the second stage
            for h in list(built):
                if h != best_h:
                    built.pop(h)
            for lo in launch:
                if lo != d:
                    timed(best_h, lo)
    finally:
        built.clear()
    if not trials:
        raise RuntimeError("no candidate could be timed")
    best = min(trials, key=lambda t: t[1])[0]
    return best, trials


def _cached(cache, key, run):
    store = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            store = json.load(f)
        if key in store:
            return store[key]["best"], [tuple(t) for t in store[key]["trials"]]
    best, trials = run()
    if cache:
        store[key] = dict(best=best, trials=trials)
        tmp = cache + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(store, f, indent=1)
        os.replace(tmp, cache)
    return best, trials


def autotune(mesh_a, mesh_b, poses, k: int = 24, kind: str = "collide", early_exit: bool = False,
             space: dict | None = None, cache: str | None = None, reps: int = 2, device="cuda",
             exhaustive: bool = False):
    """Tune one pair of meshes.  mesh_a / mesh_b: (verts, tris); poses: device float32
    (n, 12) sample of the workload.  Returns (best config dict, [(config, ms), ...])."""
    space = dict(DEFAULT_SPACE, **(space or {}))
    key = mesh_key([mesh_a, mesh_b], k, kind + ("/early" if early_exit else ""), space)

    def build(m, tb, bits):
        return BVH(*mesh_a, k, m, bits, tb, device=device), BVH(*mesh_b, k, m, bits, tb, device=device)

    def make_fn(obj):
        A, B = obj
        if kind == "collide":
            return lambda: collide(A, B, poses, pairs=False, early_exit=early_exit)
        return lambda: distance(A, B, poses)

    return _cached(cache, key, lambda: _search(build, make_fn, space, reps, exhaustive))


def autotune_batch(env, robots, poses, k: int = 24, kind: str = "collide", early_exit: bool = True,
                   space: dict | None = None, cache: str | None = None, reps: int = 2, device="cuda",
                   exhaustive: bool = False):
    """Tune a batch: the static scene ``env`` against every robot mesh of ``robots`` (for
    instance the links of an arm), with poses[i] (device float32 (n, 12)) for robots[i], all
    in one batch launch (cbvh_batch_*).  Returns (best config dict, [(config, ms), ...])."""
    space = dict(DEFAULT_SPACE, **(space or {}))
    key = mesh_key([env, *robots], k, "batch/" + kind + ("/early" if early_exit else ""), space)

    def build(m, tb, bits):
        A = BVH(*env, k, m, bits, tb, device=device)
        Bs = [BVH(*r, k, m, bits, tb, device=device) for r in robots]
        items = [dict(A=A, B=B, kind=kind, poses=P, early_exit=early_exit) for B, P in zip(Bs, poses)]
        return A, Bs, Batch(items, device=device)

    def make_fn(obj):
        return obj[2].run

    return _cached(cache, key, lambda: _search(build, make_fn, space, reps, exhaustive))
