"""The request loop (continuous batching): every request's result is the same whether it is
served alone or batched with others (CD bit-exact, PQ within 1e-5 D), under concurrent
submission from several planner threads and under a memory budget that forces admission
to wait; chain robots (one pose per link) resolve to any-link collision and the smallest
distance over their links."""
import threading

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


@pytest.fixture(scope="module")
def models(cb):
    c1 = synth.C1(4)
    va, ta, _ = synth.heightfield(64, seed=7)
    link = synth.arm_links()[2]
    return dict(
        sphereA=cb.BVH(*c1["A"], 18, 4, 16, 4096), sphereB=cb.BVH(*c1["B"], 18, 4, 16, 4096),
        terrain=cb.BVH(va, ta, 18, 4, 16, 4096), link=cb.BVH(*link, 18, 4, 16, 4096))


ROBOTS = {"chain": ["link", "sphereB"]}


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        env, robot = [("sphereA", "sphereB"), ("terrain", "sphereB"), ("terrain", "link"), ("sphereA", "link"),
                      ("terrain", "chain")][i % 5]
        n = int(np.exp(rng.uniform(0, np.log(300))))
        if robot == "chain":
            P = np.stack([synth.poses_box(n, seed=int(rng.integers(1 << 30)), lo=-1.5, hi=1.5) for _ in range(2)], 1)
        else:
            P = synth.poses_box(n, seed=int(rng.integers(1 << 30)), lo=-1.5, hi=1.5)
        kind = "collide" if rng.uniform() < 0.5 else "distance"
        out.append((env, robot, kind, P, bool(kind == "collide" and rng.uniform() < 0.5)))
    return out


def _alone(cb, models, env, robot, kind, P, early):
    import torch
    names = ROBOTS.get(robot, [robot])
    res = []
    for i, name in enumerate(names):
        Pd = torch.as_tensor(np.ascontiguousarray(P[:, i] if len(names) > 1 else P), device="cuda")
        if kind == "collide":
            res.append(cb.collide(models[env], models[name], Pd, pairs=False, early_exit=early).hit.cpu().numpy())
        else:
            res.append(cb.distance(models[env], models[name], Pd).cpu().numpy())
    return np.maximum.reduce(res) if kind == "collide" else np.minimum.reduce(res)


@pytest.mark.parametrize("budget", [1 << 31, 600 << 20])
def test_served_results_equal_alone(cb, models, budget):
    from paper_2012_05348_gb300.serve import Server
    reqs = _requests(11, 48)
    srv = Server(models, mem_budget=budget, robots=ROBOTS)
    futures = [None] * len(reqs)

    def planner(k):
        for i in range(k, len(reqs), 4):
            env, robot, kind, P, early = reqs[i]
            futures[i] = srv.submit(env, robot, kind, P, early_exit=early)

    th = [threading.Thread(target=planner, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    got = [f.result(timeout=120) for f in futures]
    srv.close()
    st = srv.stats()
    assert st["requests"] == len(reqs) and st["batches"] >= 1
    for (env, robot, kind, P, early), g in zip(reqs, got):
        ref = _alone(cb, models, env, robot, kind, P, early)
        assert g.shape == ref.shape
        if kind == "collide":
            assert (g == ref).all()
        else:
            assert np.allclose(g, ref, rtol=0, atol=1e-5 * 10.0)


def test_failed_batch_retried_on_the_plain_path(cb, models):
    """A batch whose device status reports an error is not lost: each of its requests is
    retried once on the plain path and resolves to the result it has alone.  The error is
    made on the host (the batch's status word is overwritten after its launch with the code
    of an expired device wait); no kernel is made to fail."""
    from paper_2012_05348_gb300.serve import Server

    class Failing(Server):
        def _launch(self, slot, reqs, nbytes):
            super()._launch(slot, reqs, nbytes)
            batch = self.busy[slot][4]
            with _torch_stream(self.streams[slot]):
                batch.status.fill_(-6)

    reqs = _requests(23, 10)
    srv = Failing(models, robots=ROBOTS)
    futures = [srv.submit(env, robot, kind, P, early_exit=early) for env, robot, kind, P, early in reqs]
    got = [f.result(timeout=120) for f in futures]
    srv.close()
    assert srv.stats()["retries"] == len(reqs)
    for (env, robot, kind, P, early), g in zip(reqs, got):
        ref = _alone(cb, models, env, robot, kind, P, early)
        if kind == "collide":
            assert (g == ref).all()
        else:
            assert np.allclose(g, ref, rtol=0, atol=1e-5 * 10.0)


def _torch_stream(stream):
    import torch
    return torch.cuda.stream(stream)
