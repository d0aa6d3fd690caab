"""The bounds-checked build (libcbvh_checked.so, loaded when CBVH_CHECKED=1): every node
reference, record index, decode-cache depth, leaf slot and leaf-queue position the traversal
reads or computes is checked before use, with CBVH_ERR_CHECK in the status word on failure.
On valid hierarchies no check may fire, and the results must be those of the default build:
the small case against the oracle (collision bit-exact, distances within 1e-5 D), the
terrain workload's first 1,500 poses and a batch with configuration sets against the
default build.  The checked library runs in a child process (a process loads one build)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2012_05348_gb300 as cb, synth, torch
assert cb.LIB_PATH.endswith("libcbvh_checked.so"), cb.LIB_PATH
out = sys.argv[2]
c = synth.C1(4)
P1 = np.load(out + "/p1.npy")
A = cb.BVH(*c["A"], 18, 4, 16, 4096); B = cb.BVH(*c["B"], 18, 4, 16, 4096)
r = cb.collide(A, B, torch.as_tensor(P1, device="cuda"))
d = cb.distance(A, B, torch.as_tensor(P1, device="cuda"))
np.save(out + "/c1_hit.npy", r.hit.cpu().numpy()); np.save(out + "/c1_off.npy", r.offsets.cpu().numpy())
np.save(out + "/c1_ij.npy", r.pairs.cpu().numpy()); np.save(out + "/c1_d.npy", d.cpu().numpy())
t = synth.C2(10000)
TA = cb.BVH(*t["A"], 24, 8, 8, 16384); TB = cb.BVH(*t["B"], 24, 8, 8, 16384)
P2 = torch.as_tensor(t["poses"][:1500], device="cuda")
r = cb.collide(TA, TB, P2)
np.save(out + "/t_off.npy", r.offsets.cpu().numpy()); np.save(out + "/t_ij.npy", r.pairs.cpu().numpy())
np.save(out + "/t_d.npy", cb.distance(TA, TB, P2).cpu().numpy())
c3 = synth.C3(300, n_boxes=30, n_spheres=30)
clutter = cb.BVH(*c3["A"], 24, 8, 8, 16384)
links = [cb.BVH(*l, 24, 8, 8, 16384) for l in c3["links"]]
items = [dict(A=clutter, B=L, kind="collide", poses=torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:, i]),
              device="cuda"), early_exit=True, set="arm") for i, L in enumerate(links)]
items.append(dict(A=clutter, B=links[3], kind="distance",
                  poses=torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:100, 3]), device="cuda")))
b = cb.Batch(items)
outs = b.run()
np.save(out + "/b_any.npy", b.any_hit["arm"].cpu().numpy()); np.save(out + "/b_d.npy", outs[-1].cpu().numpy())
print("checked ok")
"""


@pytest.fixture(scope="module")
def cb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_05348_gb300 import _build
    _build.build()
    import paper_2012_05348_gb300 as m
    return m


def test_checked_build_fires_no_check_and_matches(cb, tmp_path):
    import torch
    c = synth.C1(4)
    (va, ta), (vb, tb) = c["A"], c["B"]
    Ao, Bo = oracle.BVH(va, ta, 18, 4, 16, 4096), oracle.BVH(vb, tb, 18, 4, 16, 4096)
    D = synth.scene_diameter(va, vb)
    P1 = oracle.filtered_poses(Ao, Bo, lambda cnt, r: synth.poses_box(cnt, seed=2001 + 7919 * r), 256, 1e-6 * D)
    np.save(tmp_path / "p1.npy", P1)
    env = dict(os.environ, CBVH_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
    ld = lambda n: np.load(tmp_path / f"{n}.npy")  # noqa: E731
    o_hit, o_off, o_ij, _ = oracle.collide(Ao, Bo, P1)
    o_d, _ = oracle.distance(Ao, Bo, P1)
    assert (ld("c1_hit") == o_hit).all() and (ld("c1_off") == o_off).all() and (ld("c1_ij") == o_ij).all()
    assert np.abs(ld("c1_d") - o_d).max() <= 1e-5 * D
    # the terrain and the batch against the default build in this process
    t = synth.C2(10000)
    TA, TB = cb.BVH(*t["A"], 24, 8, 8, 16384), cb.BVH(*t["B"], 24, 8, 8, 16384)
    P2 = torch.as_tensor(t["poses"][:1500], device="cuda")
    ref = cb.collide(TA, TB, P2)
    assert (ld("t_off") == ref.offsets.cpu().numpy()).all() and (ld("t_ij") == ref.pairs.cpu().numpy()).all()
    Dt = synth.scene_diameter(t["A"][0], t["B"][0])
    assert np.abs(ld("t_d") - cb.distance(TA, TB, P2).cpu().numpy()).max() <= 1e-5 * Dt
    c3 = synth.C3(300, n_boxes=30, n_spheres=30)
    clutter = cb.BVH(*c3["A"], 24, 8, 8, 16384)
    links = [cb.BVH(*l, 24, 8, 8, 16384) for l in c3["links"]]
    hits = [cb.collide(clutter, L, torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:, i]), device="cuda"),
                       pairs=False).hit.cpu().numpy() for i, L in enumerate(links)]
    assert (ld("b_any") == np.maximum.reduce(hits)).all()
    dref = cb.distance(clutter, links[3], torch.as_tensor(np.ascontiguousarray(c3["link_poses"][:100, 3]),
                                                          device="cuda")).cpu().numpy()
    assert np.abs(ld("b_d") - dref).max() <= 1e-5 * 8.0
