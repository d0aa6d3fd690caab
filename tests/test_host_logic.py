"""Host-side logic that needs no GPU: the serving layer's per-configuration combination of a
chain robot's link results, and the autotuner's workload key and result cache."""
import json

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def mods():
    from paper_2012_05348_gb300 import _build
    _build.build()
    from paper_2012_05348_gb300 import autotune, serve
    return autotune, serve


def test_chain_results_combine_per_configuration(mods):
    _, serve = mods
    hits = [np.array([0, 0, 1, 0], np.uint8), np.array([0, 1, 0, 0], np.uint8), np.array([0, 0, 1, 0], np.uint8)]
    assert serve.combine("collide", hits).tolist() == [0, 1, 1, 0]  # any link in contact
    d = [np.array([0.5, 2.0, 0.0], np.float32), np.array([0.25, 3.0, 1.0], np.float32)]
    assert serve.combine("distance", d).tolist() == [0.25, 2.0, 0.0]  # the closest link
    one = np.array([1.5, 2.5], np.float32)
    out = serve.combine("distance", [one])
    assert out.tolist() == one.tolist() and out is not one  # a copy, not the output buffer


def test_tuning_key_follows_the_workload(mods):
    autotune, _ = mods
    v, t = synth.icosphere(2, 1.0, 0.1, seed=1)
    sp = autotune.DEFAULT_SPACE
    base = autotune.mesh_key([(v, t)], 24, "collide", sp)
    assert base == autotune.mesh_key([(v.copy(), t.copy())], 24, "collide", sp)  # content, not identity
    v2 = v.copy()
    v2[0, 0] += np.float32(1e-3)
    others = [autotune.mesh_key([(v2, t)], 24, "collide", sp), autotune.mesh_key([(v, t)], 18, "collide", sp),
              autotune.mesh_key([(v, t)], 24, "distance", sp),
              autotune.mesh_key([(v, t)], 24, "collide", dict(sp, split=(1,))),
              autotune.mesh_key([(v, t), (v, t)], 24, "collide", sp)]
    assert len({base, *others}) == 6


def test_tuning_cache_stores_and_returns(mods, tmp_path):
    autotune, _ = mods
    path = str(tmp_path / "tune.json")
    calls = []

    def run():
        calls.append(1)
        return {"branching": 8, "split": 3}, [({"branching": 8, "split": 3}, 1.5), ({"branching": 4, "split": 1}, 2.0)]

    best, trials = autotune._cached(path, "k1", run)
    assert best == {"branching": 8, "split": 3} and len(trials) == 2 and len(calls) == 1
    best2, trials2 = autotune._cached(path, "k1", run)  # from the file, no search
    assert best2 == best and [tuple(t) for t in trials2] == [tuple(t) for t in trials] and len(calls) == 1
    autotune._cached(path, "k2", run)  # a second workload joins the same file
    assert set(json.load(open(path))) == {"k1", "k2"} and len(calls) == 2
    best3, _ = autotune._cached(None, "k1", run)  # no cache file: always searches
    assert best3 == best and len(calls) == 3
