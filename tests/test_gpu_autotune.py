"""The autotuner: it times every candidate of a (reduced) search space, returns the fastest,
caches its result, and -- since tuning changes layout and scheduling only -- the tuned
configuration returns exactly the results of the default one."""
import json

import numpy as np
import pytest

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


SPACE = dict(branching=(4, 8), treelet_bytes=(4096, 16384), quant_bits=(8, 16), packing=(0, 1), stage_bytes=(0,),
             split=(4, 1, 0), budget0=(64, 256))


def test_autotune_pair_search_cache_and_results(cb, tmp_path):
    import torch
    from paper_2012_05348_gb300.autotune import apply, autotune
    c = synth.C1(128)
    P = torch.as_tensor(c["poses"], device="cuda")
    cache = str(tmp_path / "tune.json")
    best, trials = autotune(c["A"], c["B"], P, k=18, kind="distance", space=SPACE, cache=cache, reps=1)
    # stage 1: 2 x 2 x 2 x 2 hierarchies; stage 2: the other launch options on the best one
    n_launch = len([1 for s in SPACE["split"] for b in SPACE["budget0"] if s != 0 or b == SPACE["budget0"][0]])
    assert len(trials) == 16 + n_launch - 1
    assert best == min(trials, key=lambda t: t[1])[0]
    assert all(ms > 0 for _, ms in trials)
    stored = json.load(open(cache))
    assert len(stored) == 1 and next(iter(stored.values()))["best"] == best
    again, trials2 = autotune(c["A"], c["B"], P, k=18, kind="distance", space=SPACE, cache=cache, reps=1)
    assert again == best and len(trials2) == len(trials)
    ref = cb.distance(cb.BVH(*c["A"], 18, 8, 8, 16384), cb.BVH(*c["B"], 18, 8, 8, 16384), P).cpu().numpy()
    apply(best)
    try:
        A = cb.BVH(*c["A"], 18, best["branching"], best["quant_bits"], best["treelet_bytes"])
        B = cb.BVH(*c["B"], 18, best["branching"], best["quant_bits"], best["treelet_bytes"])
        got = cb.distance(A, B, P).cpu().numpy()
    finally:
        apply({})
    D = synth.scene_diameter(c["A"][0], c["B"][0])
    assert np.abs(got - ref).max() <= 1e-5 * D


def test_autotune_batch_arm_links(cb):
    import torch
    from paper_2012_05348_gb300.autotune import apply, autotune_batch
    c3 = synth.C3(2000, n_boxes=40, n_spheres=40)
    LP = [torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:, i]), device="cuda") for i in range(6)]
    space = dict(SPACE, packing=(0,), quant_bits=(8,))
    best, trials = autotune_batch(c3["A"], c3["links"], LP, k=24, kind="collide", early_exit=True, space=space, reps=1)
    assert best == min(trials, key=lambda t: t[1])[0]

    def flags(cfg):
        apply(cfg)
        try:
            m, tb, bits = cfg.get("branching", 8), cfg.get("treelet_bytes", 16384), cfg.get("quant_bits", 8)
            A = cb.BVH(*c3["A"], 24, m, bits, tb)
            Ls = [cb.BVH(*l, 24, m, bits, tb) for l in c3["links"]]
            outs = cb.Batch([dict(A=A, B=L, kind="collide", poses=P, early_exit=True) for L, P in zip(Ls, LP)]).run()
            return np.stack([o.cpu().numpy() for o in outs])
        finally:
            apply({})
    ref, got = flags({}), flags(best)
    assert (ref == got).all() and 0 < ref.any(0).sum() < ref.shape[1]
