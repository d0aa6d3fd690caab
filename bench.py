#!/usr/bin/env python3
"""Benchmark of the compressed k-DOP BVH engine: batched collision detection (CD) and
proximity query (PQ) of many rigid poses on one GB300.

Workload (terrain against sphere, 10,000 poses): A = 512 x 512 fractal heightfield (524,288
triangles) and B = displaced level-5 icosphere (20,480 triangles); 24-DOP, branching 8,
8-bit predictor-corrector deltas, 16 KB treelets.  One step = CD with every intersecting
triangle pair (sorted CSR lists) for all poses, then PQ (minimum distance) for all poses.
Metric: pose queries/s, a CD query and a PQ query of one pose counting as two.

Prints one JSON line (rank 0).  After the timed headline step the same line carries the
comparisons of `--sections`: the batched arm sweep against one query per link and launch,
the served request loop against one call per request, the terrain step under every way
of storing the bounds (8/16-bit deltas, FP16, FP32), the device refit of a deforming mesh
(terrain and 10M-triangle field), and the scale-and-compression workload (a 10M-triangle
field that does not fit in L2) at every compression setting.
`--impl reference` times the FP64 CPU oracle instead, on a bounded sample of the same
poses; `--scale-only` runs just the scale comparison (an entry point for profiling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pose queries/s (CD and PQ) + BV-pair tests/s on 1 GB300, % of HBM roofline; p50/p99"
K_DOP, BRANCH, BITS, TREELET = 24, 8, 8, 16384
# algorithmic bytes per unit of work for this configuration (24-DOP, 8-bit deltas):
# one BV-pair test reads an A-member descriptor (12 slabs x 2 x 1 B + 4 B topology) and a
# B-member axis box (3 slabs x 2 x 1 B); one leaf test reads two 36-byte triangles; one pose
# reads 48 bytes of pose and writes 1 B flag + 4 B distance + 8 B offset.
BYTES_BV = 24 + 4 + 6
BYTES_LEAF = 72
BYTES_POSE = 48 + 1 + 4 + 8
BYTES_PAIR = 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--poses", type=int, default=10000)
    ap.add_argument("--cpu-sample", type=int, default=0, help="poses in the oracle sample (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and served comparisons")
    ap.add_argument("--arm-configs", type=int, default=200000)
    ap.add_argument("--sections", default="small,noalloc,batched,served,compression,refit,scale",
                    help="comparisons run after the headline step: small, noalloc, batched, served, compression, "
                         "refit, scale (comma list)")
    ap.add_argument("--scale-poses", type=int, default=1_000_000)
    ap.add_argument("--scale-pq-poses", type=int, default=20_000)
    ap.add_argument("--scale-pair-poses", type=int, default=100_000)
    ap.add_argument("--scale-variants", default="8:16384,16:16384,1:16384,0:16384,8:131072",
                    help="storage modes of the scale comparison, bits:treelet_bytes (comma list)")
    ap.add_argument("--scale-only", action="store_true",
                    help="run only the scale-and-compression comparison (a profiling entry point)")
    return ap.parse_args()


def scale_variants(args):
    return tuple(tuple(int(x) for x in v.split(":")) for v in args.scale_variants.split(",") if v.strip())


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def rank_poses(n_poses: int, rank: int, height_fn):
    """Weak scaling: every rank gets its own poses of the terrain distribution (rank 0 the
    workload's own, seed 2002; rank r seed 2002 + 7919 r).  No data-path collective."""
    return synth.poses_terrain(n_poses, seed=2002 + 7919 * rank, height_fn=height_fn)


def workload(n_poses: int, rank: int):
    c = synth.C2(n_poses)
    if rank:
        c["poses"] = rank_poses(n_poses, rank, c["height"])
    return c


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's value (all ranks get it); x itself with one process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Units of all ranks per second of the slowest rank."""
    return units_per_rank * world / (max_ms / 1e3)


# ------------------------------------------------------------------ CPU (oracle) timing
def oracle_rate(c, sample: int, target_s: float = 15.0, threads: int = 0):
    """Pose queries/s of the FP64 oracle (CD with pairs + PQ) on a bounded sample; the
    sample grows until it takes about target_s seconds or reaches `sample` poses.
    threads: OpenMP threads (0 = all the host's cores)."""
    import oracle
    A = oracle.BVH(*c["A"], K_DOP, BRANCH, BITS, TREELET)
    B = oracle.BVH(*c["B"], K_DOP, BRANCH, BITS, TREELET)
    if threads:
        all_threads = oracle.num_threads()
        oracle.set_threads(threads)
        try:
            return oracle_rate(c, sample, target_s)
        finally:
            oracle.set_threads(all_threads)
    P = c["poses"]
    n, done, t_tot = 16, 0, 0.0
    while True:
        take = P[done:done + n]
        t0 = time.perf_counter()
        oracle.collide(A, B, take)
        oracle.distance(A, B, take)
        t_tot += time.perf_counter() - t0
        done += len(take)
        if t_tot >= target_s or done >= len(P) or (sample and done >= sample):
            break
        n = min(len(P) - done, max(16, int(n * 2)))
        if sample:
            n = min(n, sample - done)
    return 2 * done / t_tot, done, t_tot, oracle.num_threads()


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    c = workload(args.poses, 0)
    import oracle
    A = oracle.BVH(*c["A"], K_DOP, BRANCH, BITS, TREELET)
    B = oracle.BVH(*c["B"], K_DOP, BRANCH, BITS, TREELET)
    per_step = args.cpu_sample or 64
    P = c["poses"]
    for w in range(args.warmup):
        take = P[(w * per_step) % len(P):][:per_step]
        oracle.collide(A, B, take)
        oracle.distance(A, B, take)
    times = []
    for s in range(args.steps):
        take = P[(s * per_step) % len(P):][:per_step]
        t0 = time.perf_counter()
        oracle.collide(A, B, take)
        oracle.distance(A, B, take)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = 2 * per_step * args.steps / total
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pose queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "terrain 512x512 (524,288 tris) vs displaced level-5 icosphere (20,480 tris), "
                               "24-DOP, branching 8, 8-bit deltas, 16 KB treelets",
                   "poses_per_step": per_step, "sample": f"first {per_step} poses per step of the 10,000-pose set"},
        "cpu_baseline": {"value": value, "unit": "pose queries/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{per_step} poses per step (CD with pairs + PQ), FP64 oracle, OpenMP over poses"},
        "e2e": {"value": value, "unit": "pose queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,uuid")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out = self.proc.communicate(timeout=5)[0]
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = self.proc.communicate()[0]

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            if self.uuid and self.uuid not in f[7]:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[3:7]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}




# ------------------------------------------------------------------ batched and served forms
def _events_ms(fn, torch, reps=3):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _launch_latencies(fn, torch, reps=7):
    """p50 / p99 of single launches of fn, each timed by its own CUDA events after a warm-up."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return {"p50": ts[len(ts) // 2], "p99": ts[min(len(ts) - 1, int(round(0.99 * (len(ts) - 1))))], "launches": reps}


def arm_sweep(cb, torch, dev, n_configs, tune_configs=20000):
    """Motion-planning sweep: 6 arm links against a 1,026,400-triangle clutter scene, early-exit
    CD for every configuration.  The autotuner first picks branching, treelet size,
    quantisation bits and launch options (work mapping, budget) on the first `tune_configs`
    configurations.  Then the whole sweep runs batched (one set of persistent launches over
    all links, replayed from a CUDA graph; the six links of a configuration form one set, so
    a configuration stops at its first colliding link) against the plain traversal (one
    query per link and launch, one warp per pose) on the same hierarchies; both give every
    configuration's answer (some link collides)."""
    from paper_2012_05348_gb300.autotune import DEFAULT_LAUNCH, apply, autotune_batch
    c = synth.C3(n_configs)
    LP = [torch.as_tensor(np.ascontiguousarray(c["link_poses"][:, i]), device=dev) for i in range(6)]
    t0 = time.perf_counter()
    best, trials = autotune_batch(c["A"], c["links"], [P[:tune_configs] for P in LP], k=24, kind="collide",
                                  early_exit=True, space=dict(stage_bytes=(0,)), reps=1, device=dev)
    tune_s = time.perf_counter() - t0
    default = dict(branching=8, treelet_bytes=16384, quant_bits=8, packing=cb.PACK_TOP_DOWN, **DEFAULT_LAUNCH)
    default_ms = next((ms for cfg, ms in trials if cfg == default), None)
    best_ms = min(ms for _, ms in trials)
    m, tb, bits = best["branching"], best["treelet_bytes"], best["quant_bits"]
    apply(best)
    try:
        A = cb.BVH(*c["A"], 24, m, bits, tb, device=dev)
        links = [cb.BVH(*l, 24, m, bits, tb, device=dev) for l in c["links"]]
        items = [dict(A=A, B=L, kind="collide", poses=P, early_exit=True, set="arm") for L, P in zip(links, LP)]
        batch = cb.Batch(items, device=dev)
        outs = batch.run()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            batch.launch(s)
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            batch.launch()
        ms_batched = _events_ms(g.replay, torch)
        lat_batched = _launch_latencies(g.replay, torch)
        collide_cfg = batch.any_hit["arm"].cpu().numpy().astype(bool)
        # self-collision: every non-adjacent link pair, link j posed in link i's frame
        sp = synth.self_pairs(6)
        rel = [torch.as_tensor(synth.relative_poses(c["link_poses"], i, j), device=dev) for i, j in sp]
        self_items = [dict(A=links[i], B=links[j], kind="collide", poses=R, early_exit=True, set="self")
                      for (i, j), R in zip(sp, rel)]
        self_batch = cb.Batch(self_items, device=dev)
        self_batch.run()
        ms_self = _events_ms(self_batch.run, torch)
        self_cfg = self_batch.any_hit["self"].cpu().numpy().astype(bool)
        # validity in one launch: the six links against the scene and the ten link pairs
        # against each other as one configuration set (a configuration is invalid once any
        # of the sixteen items intersects)
        valid_batch = cb.Batch([dict(it, set="valid") for it in items] +
                               [dict(it, set="valid") for it in self_items], device=dev)
        valid_batch.run()
        ms_valid = _events_ms(valid_batch.run, torch)
        invalid_cfg = valid_batch.any_hit["valid"].cpu().numpy().astype(bool)

        # clearance: the smallest distance over the six links of each configuration, as one
        # distance set (each link prunes with the configuration's best so far), against the
        # same items without the set and one cbvh_distance per link
        n_cl = min(4096, n_configs)
        LPc = [P[:n_cl] for P in LP]
        cl_set = cb.Batch([dict(A=A, B=L, kind="distance", poses=P, set="arm") for L, P in zip(links, LPc)], device=dev)
        cl_items = cb.Batch([dict(A=A, B=L, kind="distance", poses=P) for L, P in zip(links, LPc)], device=dev)
        ms_cl_set = _events_ms(cl_set.run, torch, reps=2)
        ms_cl_items = _events_ms(cl_items.run, torch, reps=2)
        cl_plain = []

        def cl_plain_fn():
            cl_plain.clear()
            for L, P in zip(links, LPc):
                cl_plain.append(cb.distance(A, L, P, check=False))
        ms_cl_plain = _events_ms(cl_plain_fn, torch, reps=1)
        cl_ref = torch.stack(cl_plain).min(0).values
        cl_diff = float((cl_set.min_dist["arm"] - cl_ref).abs().max().item())
        clearance = {"configurations": n_cl, "set_ms": ms_cl_set, "items_ms": ms_cl_items, "plain_ms": ms_cl_plain,
                     "set_configurations_per_s": n_cl / (ms_cl_set / 1e3),
                     "speedup_set_vs_items": ms_cl_items / ms_cl_set, "speedup_set_vs_plain": ms_cl_plain / ms_cl_set,
                     "max_abs_diff_vs_plain": cl_diff,
                     "what": "smallest distance over the six links of each configuration"}
        plain_out = []

        def plain():
            plain_out.clear()
            for L, P in zip(links, LP):
                plain_out.append(cb.collide(A, L, P, pairs=False, early_exit=True, check=False).hit)
        cb.set_option(cb.OPT_SPLIT, cb.SPLIT_POSE)
        ms_plain = _events_ms(plain, torch, reps=2)
        plain_cfg = torch.stack(plain_out).any(0).cpu().numpy()
    finally:
        apply({})
    q = 6 * n_configs
    return {"workload": f"6-link DH arm (5,120..40k tris per link) vs 1,026,400-tri clutter, {n_configs} configurations, "
                        "early-exit CD, 24-DOP",
            "autotuned": {"best": best, "sample_configurations": tune_configs, "candidates": len(trials),
                          "tuning_s": tune_s, "sample_ms_best": best_ms, "sample_ms_default": default_ms},
            "link_queries": q, "configs_in_collision": int(collide_cfg.sum()),
            "answers_equal_plain": bool((plain_cfg == collide_cfg).all()),
            "self_collision": {"link_pairs": len(sp), "pair_queries": len(sp) * n_configs,
                               "configs_self_colliding": int(self_cfg.sum()), "ms": ms_self,
                               "pair_queries_per_s": len(sp) * n_configs / (ms_self / 1e3)},
            "configs_free": int((~collide_cfg & ~self_cfg).sum()),
            "validity": {"items": len(items) + len(self_items), "ms": ms_valid,
                         "configurations_per_s": n_configs / (ms_valid / 1e3),
                         "configs_valid": int((~invalid_cfg).sum()),
                         "equals_separate_sets": bool((invalid_cfg == (collide_cfg | self_cfg)).all()),
                         "what": "links against the scene and link pairs against each other, one set per "
                                 "configuration, one launch"},
            "batched_link_queries_per_s": q / (ms_batched / 1e3), "batched_ms": ms_batched,
            "batched_latency_ms": dict(lat_batched, per="graph replay of the whole sweep"),
            "plain_link_queries_per_s": q / (ms_plain / 1e3), "plain_ms": ms_plain,
            "batched_configurations_per_s": n_configs / (ms_batched / 1e3),
            "clearance": clearance,
            "plain_configurations_per_s": n_configs / (ms_plain / 1e3),
            "speedup_vs_plain": ms_plain / ms_batched,
            "batched": "one graph-captured persistent launch set, autotuned hierarchy and launch options, the six "
                       "links of a configuration as one set (a configuration stops at its first colliding link)",
            "plain": "one cbvh_collide per link, one warp per pose, same hierarchies"}


def serving(cb, torch, dev, models, robots, height_fn, rates=(20, 100, 2000, 10000, 50000), max_requests=400,
            seed=2004):
    """Request loop under open-loop Poisson arrivals (the serving workload: terrain and clutter
    environments; the 6-link arm and the level-5 and level-3 spheres as robots; collision and
    distance 1:1; log-uniform 1..4096 configurations per request).  Each offered rate runs
    for min(2 s, max_requests / rate) of arrivals; the last rate's mix is then replayed at
    50 % and 80 % of its served rate.  Reports p50/p99 latency and throughput;
    the plain form serves the same requests one call per model pair (per link for the arm),
    in arrival order."""
    from paper_2012_05348_gb300.serve import Server
    import threading
    out = []
    # the listed rates; then the last rate's request mix replayed at 50 % and 80 % of the
    # request rate it was served at (its saturation rate: at that offered rate every request
    # arrives while the server is busy), the Poisson gaps rescaled to the new rate
    todo = [(r, None) for r in rates]
    last = None
    while todo:
        rate, frac = todo.pop(0)
        if frac is None:
            secs = min(2.0, max_requests / rate)
            gaps, reqs = synth.C4(rate, secs, height_fn, seed=seed + int(rate))
        else:
            gaps0, reqs, rate0 = last
            gaps = [g * rate0 / rate for g in gaps0]
            secs = float(sum(gaps))
        srv = Server(models, mem_budget=8 << 30, device=dev, robots=robots)
        futs = []

        def gen():
            t0 = time.perf_counter()
            t = 0.0
            for (env, rob, kind, P), gap in zip(reqs, gaps):
                t += gap
                d = t0 + t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                futs.append(srv.submit(env, rob, kind, P))
        t_start = time.perf_counter()
        th = threading.Thread(target=gen)
        th.start()
        th.join()
        for f in futs:
            f.result(timeout=900)
        t_end = time.perf_counter()
        srv.close()
        st = srv.stats()
        configs = sum(len(r[3]) for r in reqs)
        link_poses = sum(len(r[3]) * (6 if r[1] == "arm" else 1) for r in reqs)
        # plain: the same requests, one call per model pair, results back on the host
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for env, rob, kind, P in reqs:
            names = robots.get(rob, [rob])
            res = []
            for i, name in enumerate(names):
                Pd = torch.as_tensor(np.ascontiguousarray(P[:, i] if len(names) > 1 else P), device=dev)
                if kind == "collide":
                    res.append(cb.collide(models[env], models[name], Pd, pairs=False).hit.cpu())
                else:
                    res.append(cb.distance(models[env], models[name], Pd).cpu())
        t_plain = time.perf_counter() - t0
        out.append({"offered_req_per_s": rate, "arrival_window_s": secs, "requests": len(reqs),
                    "configurations": configs, "link_poses": link_poses, "batches": st["batches"],
                    "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                    "served_req_per_s": len(reqs) / (t_end - t_start),
                    "served_configs_per_s": configs / (t_end - t_start),
                    "plain_configs_per_s": configs / t_plain,
                    "speedup_vs_plain": t_plain / (t_end - t_start)})
        if frac is not None:
            out[-1]["fraction_of_saturation"] = frac
            out[-1]["request_mix"] = f"that of {last[2]:g} req/s, gaps rescaled"
        if not todo and frac is None:
            last = (gaps, reqs, rate)
            sat = out[-1]["served_req_per_s"]
            todo = [(0.5 * sat, 0.5), (0.8 * sat, 0.8)]
    return out


def compression(cb, torch, dev, c, steps=3):
    """The terrain step (CD with sorted pair lists + PQ, every pose) for each way of storing
    the bounds: 8- and 16-bit predictor-corrector deltas, FP16 descriptors (the paper's
    measured mode, Sec. III-A), uncompressed FP32, and the integer compression the
    conclusion proposes (exact lattice deltas in Stream VByte).  Same hierarchy shape
    (24-DOP, branching 8, 16 KB treelets); L2 flushed before every step; kernel time from
    the library's events; BV-pair tests of the collision query from the device counters."""
    import ctypes as C
    L = cb.lib
    sp = cb._stream_ptr(None)
    n = len(c["poses"])
    P = torch.as_tensor(c["poses"], device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    out = []
    for bits in (8, 16, 1, 0, 2):
        A = cb.BVH(*c["A"], K_DOP, BRANCH, bits, TREELET, device=dev)
        B = cb.BVH(*c["B"], K_DOP, BRANCH, bits, TREELET, device=dev)
        cap = 16_000_000
        hit = torch.empty(n, dtype=torch.uint8, device=dev)
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        prs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
        need = torch.zeros(1, dtype=torch.int64, device=dev)
        dist = torch.empty(n, dtype=torch.float32, device=dev)
        st = torch.zeros(2, dtype=torch.int32, device=dev)
        wc = cb.workspace_bytes(A, B, n, 0, cap)
        wp = cb.workspace_bytes(A, B, n, 1)
        ws_c = torch.empty(wc, dtype=torch.uint8, device=dev)
        ws_p = torch.empty(wp, dtype=torch.uint8, device=dev)
        ptr = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
        st1 = C.c_void_p(st.data_ptr() + 4)

        def step():
            rc = L.cbvh_collide(A.handle, B.handle, ptr(P), n, ptr(hit), ptr(off), ptr(prs), cap, ptr(need),
                                cb.SORT_PAIRS, ptr(ws_c), wc, ptr(st), sp)
            rc |= L.cbvh_distance(A.handle, B.handle, ptr(P), n, ptr(dist), ptr(ws_p), wp, st1, sp)
            if rc:
                raise cb.CbvhError(rc, L.cbvh_last_error().decode())
        step()
        torch.cuda.synchronize()
        if int(st.abs().sum().item()):
            raise RuntimeError("device status in the compression comparison")
        ms = {"collide": 0.0, "distance": 0.0}
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            cb.profile_collect()
            cb.profile_enable(True)
            step()
            torch.cuda.synchronize()
            cb.profile_enable(False)
            pr = cb.profile_collect()
            ms["collide"] += pr["collide"][0] / steps
            ms["distance"] += pr["distance"][0] / steps
        bv_cd = int(cb.query_stats(ws_c)[0])
        out.append({"mode": {8: "8-bit deltas", 16: "16-bit deltas", 1: "FP16", 0: "FP32",
                             2: "Stream VByte exact deltas"}[bits],
                    "quant_bits": bits, "node_bytes": A.info["node_bytes"], "cd_bv_tests": bv_cd, "cd_ms": ms["collide"],
                    "pq_ms": ms["distance"], "pose_queries_per_s": 2 * n / ((ms["collide"] + ms["distance"]) / 1e3)})
        del A, B
        torch.cuda.empty_cache()
    return {"workload": "terrain step (10,000 poses, CD with sorted pairs + PQ), 24-DOP, branching 8, 16 KB treelets",
            "modes": out}


def refit_rate(cb, torch, dev, verts, tris, k, m, bits, tb, packing, reps=5):
    """Device refit (deforming meshes) and device build (per-frame meshes) of one hierarchy.

    Refit: the mesh breathes (every vertex scaled about the origin by 1 +- 0.1 %), the tree
    is kept and every bound recomputed and re-encoded on the GPU.  Algorithmic bytes: per
    triangle its index, three vertex indices, three vertices in and the triangle out
    (88 B); per node the plan (24 B), the exact bounds written, merged and read back and
    the decoded bounds (24 B per direction) and its record.

    Build: the host builder (one core) against cbvh_build_device on a plan made once (the
    median splits, lattice exponent, bounds and encoding on the GPU; the call synchronises),
    without and with the copy of the blob back to the host; the device blob must equal the
    host build's byte for byte."""
    cb.set_option(cb.OPT_TREELET_PACKING, packing)
    cb.set_option(cb.OPT_LATTICE_HEADROOM, 1)  # room for the larger breath
    try:
        t0 = time.perf_counter()
        h = cb.BVH(verts, tris, k, m, bits, tb, device=dev)
        host_build_s = time.perf_counter() - t0
        p = cb.BVH.plan(len(verts), len(tris), k, m, bits, tb, device=dev)
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
        cb.set_option(cb.OPT_LATTICE_HEADROOM, 0)
    T = torch.as_tensor(tris, device=dev)
    V0 = torch.as_tensor(verts, device=dev)
    p.build_device(V0, T, host_copy=False)  # first build: workspace and plan upload
    build_ms = []
    n0 = cb.kernel_launches()
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.build_device(V0, T, host_copy=False)
        build_ms.append((time.perf_counter() - t0) * 1e3)
    launches = (cb.kernel_launches() - n0) // reps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p.build_device(V0, T, host_copy=True)
    copy_ms = (time.perf_counter() - t0) * 1e3
    identical = bool((p.blob_host() == h.blob_host()).all())
    del p
    V = [torch.as_tensor((verts * s).astype(np.float32), device=dev) for s in (1.001, 0.999)]
    h.refit(V[0], T)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for r in range(reps):
        h.refit(V[r & 1], T, check=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nn, nt = h.info["n_nodes"], h.info["n_tris"]
    rec = 8 + (4 * k // 2 if bits == 1 else (8 * k // 2 if bits == 0 else k * bits // 8))
    algo = nt * 88 + nn * (24 + 24 * (k // 2) + rec)
    bms = float(np.median(build_ms))
    return {"triangles": nt, "nodes": nn, "quant_bits": bits, "ms": ms, "triangles_per_s": nt / (ms / 1e3),
            "algorithmic_gbs": algo / (ms * 1e6),
            "build": {"host_build_s": host_build_s, "device_build_ms": bms,
                      "device_build_with_host_copy_ms": copy_ms, "speedup_vs_host": host_build_s * 1e3 / bms,
                      "kernel_launches": launches, "identical_to_host_build": identical}}


def _bv_bytes(k: int, bits: int) -> int:
    """Algorithmic bytes of one BV-pair test: A's k/2 slabs (2 values each) + 4 B topology,
    and B's axis box (3 slabs); FP32 values when bits = 0, FP16 values when bits = 1."""
    w = 4 if bits == 0 else (2 if bits == 1 else bits // 8)
    return (k // 2) * 2 * w + 4 + 3 * 2 * w


def scale(cb, torch, dev, n_poses, pq_poses, pair_poses,
          variants=((8, 16384), (16, 16384), (1, 16384), (0, 16384), (8, 131072))):
    """Scale and compression: 32 fractal-displaced level-7 spheres (10,485,760 triangles) in a
    20 m cube, probed by a displaced level-6 sphere (81,920 triangles); 18-DOP, branching 4,
    bottom-up treelets.  For 8- and 16-bit deltas at 16 and 128 KB treelets and for FP32
    bounds: footprint, collision flags for every pose (each pose stops at its first pair),
    collision with sorted pair lists on the first poses, distances on the first poses, and
    the algorithmic bytes each query moves per second.  The hierarchy (about 1-1.8 GB) does
    not fit in L2, so HBM is the roofline here."""
    import ctypes as C
    L = cb.lib
    sp = cb._stream_ptr(None)
    c = synth.C5(n_poses)
    P = torch.as_tensor(c["poses"], device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_BOTTOM_UP)
    out = []
    try:
        B = cb.BVH(*c["B"], 18, 4, 8, 16384, device=dev)

        def run(A, n, kind, cap=0):
            Pq = P[:n]
            status = torch.zeros(1, dtype=torch.int32, device=dev)
            if kind == "dist":
                wsb = cb.workspace_bytes(A, B, n, 1)
                ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
                dist = torch.empty(n, dtype=torch.float32, device=dev)
                args = (A.handle, B.handle, C.c_void_p(Pq.data_ptr()), n, C.c_void_p(dist.data_ptr()),
                        C.c_void_p(ws.data_ptr()), wsb, C.c_void_p(status.data_ptr()), sp)
                fn = lambda: L.cbvh_distance(*args)  # noqa: E731
            else:
                wsb = cb.workspace_bytes(A, B, n, 0, cap)
                ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
                hit = torch.empty(n, dtype=torch.uint8, device=dev)
                off = torch.empty(n + 1, dtype=torch.int64, device=dev) if cap else None
                prs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev) if cap else None
                need = torch.zeros(1, dtype=torch.int64, device=dev)
                ptr = lambda t: C.c_void_p(t.data_ptr() if t is not None else 0)  # noqa: E731
                args = (A.handle, B.handle, C.c_void_p(Pq.data_ptr()), n, C.c_void_p(hit.data_ptr()), ptr(off),
                        ptr(prs), cap, C.c_void_p(need.data_ptr()), cb.SORT_PAIRS if cap else 0,
                        C.c_void_p(ws.data_ptr()), wsb, C.c_void_p(status.data_ptr()), sp)
                fn = lambda: L.cbvh_collide(*args)  # noqa: E731
            flush.zero_()
            torch.cuda.synchronize()
            cb.profile_collect()
            cb.profile_enable(True)
            rc = fn()
            torch.cuda.synchronize()
            cb.profile_enable(False)
            pr = cb.profile_collect()
            code = rc or int(status.item())
            if kind == "pairs" and code == -4:  # pair capacity: the device reported the size needed
                return run(A, n, kind, cap=int(need.item()) + 1024)
            if code:
                raise cb.CbvhError(code, L.cbvh_last_error().decode())
            ms = pr["distance"][0] if kind == "dist" else pr["collide"][0]
            extra = {}
            if kind == "pairs":
                extra["pairs"] = int(need.item())
                extra["compaction_ms"] = pr["compaction"][0]
            if kind != "dist":
                extra["hits"] = int(hit.sum().item())
            return ms, cb.query_stats(ws), extra

        for bits, tb in variants:
            t0 = time.perf_counter()
            A = cb.BVH(*c["A"], 18, 4, bits, tb, device=dev)
            build_s = time.perf_counter() - t0
            bvb = _bv_bytes(18, bits)
            r = {"quant_bits": bits, "treelet_bytes": tb, "node_bytes": A.info["node_bytes"],
                 "blob_bytes": A.info["blob_bytes"], "treelets": A.info["n_treelets"], "host_build_s": build_s}
            ms, (bv, leaf, _), ex = run(A, n_poses, "hits")
            r["cd_flags"] = {"poses": n_poses, "ms": ms, "pose_queries_per_s": n_poses / (ms / 1e3),
                             "hits": ex["hits"], "bv_tests": bv, "leaf_tests": leaf,
                             "algorithmic_gbs": (bv * bvb + leaf * BYTES_LEAF + n_poses * 49) / (ms * 1e6)}
            if bits == 8 and tb == 16384 and pair_poses:
                ms, (bv, leaf, _), ex = run(A, pair_poses, "pairs", cap=2000 * pair_poses)
                r["cd_pairs"] = {"poses": pair_poses, "ms": ms, "compaction_ms": ex["compaction_ms"],
                                 "pose_queries_per_s": pair_poses / (ms / 1e3), "pairs": ex["pairs"],
                                 "algorithmic_gbs": (bv * bvb + leaf * BYTES_LEAF + pair_poses * 57
                                                     + ex["pairs"] * 12) / (ms * 1e6)}
            if not pq_poses:
                out.append(r)
                del A
                torch.cuda.empty_cache()
                continue
            ms, (bv, leaf, _), _ = run(A, pq_poses, "dist")
            r["pq"] = {"poses": pq_poses, "ms": ms, "pose_queries_per_s": pq_poses / (ms / 1e3), "bv_tests": bv,
                       "leaf_tests": leaf, "algorithmic_gbs": (bv * bvb + leaf * BYTES_LEAF + pq_poses * 52) / (ms * 1e6)}
            out.append(r)
            del A
            torch.cuda.empty_cache()
    finally:
        cb.set_option(cb.OPT_TREELET_PACKING, cb.PACK_TOP_DOWN)
    return {"workload": "32 fractal level-7 spheres (10,485,760 tris) in a 20 m cube vs displaced level-6 sphere "
                        "(81,920 tris), 18-DOP, branching 4, bottom-up treelets; L2 flushed before each query",
            "variants": out}


def small_case(cb, torch, dev, launches=200):
    """The small case exactly as configured: two displaced level-3 spheres (1,280 triangles
    each), 18-DOP, branching 4, 16-bit deltas, 4 KB treelets; 256 poses, CD with sorted pair
    lists, one query per launch.  Each launch is timed by CUDA events on its stream; the
    inputs (a few hundred KB) stay in L2 from launch to launch, as they would in a loop of
    such queries."""
    import ctypes as C
    L = cb.lib
    c = synth.C1(256)
    A = cb.BVH(*c["A"], 18, 4, 16, 4096, device=dev)
    B = cb.BVH(*c["B"], 18, 4, 16, 4096, device=dev)
    P = torch.as_tensor(c["poses"], device=dev)
    n = len(c["poses"])
    cap = int(cb.collide(A, B, P).pairs.shape[0] * 1.25) + 1024
    hit = torch.empty(n, dtype=torch.uint8, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    prs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    need = torch.zeros(1, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    wsb = cb.workspace_bytes(A, B, n, 0, cap)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    sp = cb._stream_ptr(None)
    stream = torch.cuda.current_stream(dev)
    ptr = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    args = (A.handle, B.handle, ptr(P), n, ptr(hit), ptr(off), ptr(prs), cap, ptr(need), cb.SORT_PAIRS, ptr(ws), wsb,
            ptr(st), sp)
    for _ in range(5):
        L.cbvh_collide(*args)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(launches)]
    n0 = cb.kernel_launches()
    for a, b in ev:
        a.record(stream)
        rc = L.cbvh_collide(*args)
        b.record(stream)
        if rc:
            raise cb.CbvhError(rc, L.cbvh_last_error().decode())
    torch.cuda.synchronize()
    kernels = (cb.kernel_launches() - n0) / launches
    if int(st.item()):
        raise cb.CbvhError(int(st.item()), "device status in the small case")
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    bv, leaf, _ = cb.query_stats(ws)
    total = sum(ms)
    return {"workload": "two displaced level-3 icospheres (1,280 tris each), 18-DOP, branching 4, 16-bit deltas, "
                        "4 KB treelets; 256 poses, CD with sorted pair lists, one query per launch",
            "launches": launches, "kernels_per_query": kernels, "pairs_per_query": int(need.item()),
            "pose_queries_per_s": n * launches / (total / 1e3), "bv_pair_tests_per_s": bv * launches / (total / 1e3),
            "latency_ms": {"p50": ms[len(ms) // 2], "p99": ms[min(len(ms) - 1, int(round(0.99 * (len(ms) - 1))))]}}


def noalloc_compare(cb, torch, dev, A, B, poses, dist_out, ws_pq, flush, reps=3):
    """The terrain step's proximity query through cbvh_distance_noalloc (fixed scratch inside
    the library) beside cbvh_distance (caller's workspace); L2 flushed before each call,
    CUDA events on the stream, the two results compared."""
    import ctypes as C
    L = cb.lib
    sp = cb._stream_ptr(None)
    stream = torch.cuda.current_stream(dev)
    n = int(poses.shape[0])
    ptr = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    out2 = torch.empty_like(dist_out)
    st = torch.zeros(2, dtype=torch.int32, device=dev)
    st1 = C.c_void_p(st.data_ptr() + 4)
    calls = {"distance": lambda: L.cbvh_distance(A.handle, B.handle, ptr(poses), n, ptr(dist_out), ptr(ws_pq),
                                                 ws_pq.numel(), ptr(st), sp),
             "distance_noalloc": lambda: L.cbvh_distance_noalloc(A.handle, B.handle, ptr(poses), n, ptr(out2), st1, sp)}
    res = {}
    for name, fn in calls.items():
        fn()
        times = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rc = fn()
            b.record(stream)
            if rc:
                raise cb.CbvhError(rc, L.cbvh_last_error().decode())
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        res[name] = {"ms": statistics.median(times), "pose_queries_per_s": n / (statistics.median(times) / 1e3)}
    if int(st.abs().sum().item()):
        raise RuntimeError("device status in the allocation-free comparison")
    res["max_abs_diff"] = float((dist_out - out2).abs().max().item())
    res["workload"] = "terrain step's proximity query (10,000 poses), both passes"
    return res


def l2_ceiling(cb, dev):
    """Measured L2 read bandwidth (GB/s): the best of three sizes that stay in L2."""
    best = 0.0
    for mb in (16, 32, 64):
        best = max(best, cb.probe_l2_read(mb << 20, 20, device=dev))
    return best


# ------------------------------------------------------------------ engine
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, local_rank, world = dist_env()
    import torch
    import paper_2012_05348_gb300 as cb
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if args.scale_only:
        if rank == 0:
            print(json.dumps({"scale": scale(cb, torch, dev, args.scale_poses, args.scale_pq_poses,
                                             args.scale_pair_poses, scale_variants(args))}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    c = workload(args.poses, rank)
    A = cb.BVH(*c["A"], K_DOP, BRANCH, BITS, TREELET, device=dev)
    B = cb.BVH(*c["B"], K_DOP, BRANCH, BITS, TREELET, device=dev)
    n = len(c["poses"])
    poses_host = torch.from_numpy(c["poses"]).pin_memory()
    poses = poses_host.to(dev)
    stream = torch.cuda.current_stream(dev)
    sp = cb._stream_ptr(stream)
    L = cb.lib
    import ctypes as C

    def P(t):
        return C.c_void_p(t.data_ptr())

    # size the pair buffer from a first run
    first = cb.collide(A, B, poses)
    cap = int(first.pairs.shape[0] * 1.25) + 1024
    hit = torch.empty(n, dtype=torch.uint8, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    need = torch.zeros(1, dtype=torch.int64, device=dev)
    dist_out = torch.empty(n, dtype=torch.float32, device=dev)
    st_cd = torch.zeros(1, dtype=torch.int32, device=dev)
    st_pq = torch.zeros(1, dtype=torch.int32, device=dev)
    ws_cd_b = cb.workspace_bytes(A, B, n, 0, cap)
    ws_pq_b = cb.workspace_bytes(A, B, n, 1)
    ws_cd = torch.empty(ws_cd_b, dtype=torch.uint8, device=dev)
    ws_pq = torch.empty(ws_pq_b, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB of L2

    def step(src):
        rc = L.cbvh_collide(A.handle, B.handle, P(src), n, P(hit), P(off), P(pairs), cap, P(need), cb.SORT_PAIRS,
                            P(ws_cd), ws_cd_b, P(st_cd), sp)
        rc |= L.cbvh_distance(A.handle, B.handle, P(src), n, P(dist_out), P(ws_pq), ws_pq_b, P(st_pq), sp)
        if rc:
            raise cb.CbvhError(rc, L.cbvh_last_error().decode())

    for _ in range(max(3, args.warmup)):
        step(poses)
    torch.cuda.synchronize()
    if int(st_cd.item()) or int(st_pq.item()):
        raise RuntimeError(f"device status {int(st_cd.item())} / {int(st_pq.item())}")
    bv_cd, leaf_cd, exp_cd = cb.query_stats(ws_cd)
    bv_pq, leaf_pq, exp_pq = cb.query_stats(ws_pq)
    n_pairs = int(need.item())

    # ---- timed: device-resident inputs; L2 flushed (untimed) before every step ----
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    cb.profile_collect()
    cb.profile_enable(True)
    launches0 = cb.kernel_launches()
    with ClockSampler(uuid or None) as clk:
        for s in range(K):
            flush.zero_()
            ev[s][0].record(stream)
            step(poses)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    gpu_launches = cb.kernel_launches() - launches0  # the library's own count, timed region only
    cb.profile_enable(False)
    prof = cb.profile_collect()

    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    value = whole_job_rate(2 * n * K, world, total_ms)

    # ---- end to end: pinned host poses in, results out, every step ----
    hit_h = torch.empty(n, dtype=torch.uint8).pin_memory()
    off_h = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    pairs_h = torch.empty((cap, 2), dtype=torch.int32).pin_memory()
    dist_h = torch.empty(n, dtype=torch.float32).pin_memory()
    poses_e = torch.empty_like(poses)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for s in range(K):
        poses_e.copy_(poses_host, non_blocking=True)
        step(poses_e)
        hit_h.copy_(hit, non_blocking=True)
        off_h.copy_(off, non_blocking=True)
        pairs_h[:n_pairs].copy_(pairs[:n_pairs], non_blocking=True)
        dist_h.copy_(dist_out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dev)
    e2e_val = whole_job_rate(2 * n * K, world, e2e_ms)
    h2d = n * 48
    d2h = n * 1 + (n + 1) * 8 + n_pairs * 8 + n * 4

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    # ---- roofline of the dominant kernel (the traversal, CD or PQ) ----
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    cd_bytes = bv_cd * BYTES_BV + leaf_cd * BYTES_LEAF + n * BYTES_POSE + n_pairs * 3 * 4
    pq_bytes = bv_pq * BYTES_BV + leaf_pq * BYTES_LEAF + n * BYTES_POSE
    cd_avg = prof["collide"][0] / max(1, prof["collide"][1])
    pq_avg = prof["distance"][0] / max(1, prof["distance"][1] // 2)  # two passes per distance query
    dom = (("traverse_kernel<CD>", cd_bytes, cd_avg, exp_cd) if cd_avg >= pq_avg
           else ("traverse_kernel<PQ>", pq_bytes, pq_avg, exp_pq))
    achieved = dom[1] / (dom[2] / 1e3) / 1e9
    # ncu counters of the traversal kernels from the committed capture, only while the
    # kernels are the ones it measured: DRAM bytes per query (cold cache, the full-size
    # launch list), L2 bytes and warp instructions per node-pair expansion (a smaller case,
    # scaled by this run's expansion count)
    traffic = None
    ctr = {}
    tr_file = os.path.join(ROOT, "profiles", "counters.json")
    if os.path.exists(tr_file):
        try:
            import hashlib
            tr = json.load(open(tr_file))
            src = open(os.path.join(ROOT, "paper_2012_05348_gb300", "csrc", "kernels.cu"), "rb").read()
            if tr.get("kernels_cu_sha1") == hashlib.sha1(src).hexdigest():
                ctr = tr.get(dom[0], {})
                traffic = ctr.get("dram_bytes_per_query")
        except (OSError, ValueError):
            traffic = None
    clocks = clk.summary()
    sm_mhz = (clocks or {}).get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    l2_gbs = l2_ceiling(cb, dev)
    n_sm = props.multi_processor_count
    issue_peak = n_sm * 4 * sm_mhz * 1e6  # one warp instruction per scheduler and cycle
    l2 = {"achieved": achieved, "peak": l2_gbs, "unit": "GB/s", "frac": achieved / l2_gbs,
          "peak_source": "measured: cbvh_probe_l2_read, L1-bypassing 16-byte loads over an L2-resident buffer "
                         "(best of 16, 32, 64 MB), this run",
          "lts_bytes_per_query": None, "lts_frac": None}
    issue = {"achieved": None, "peak": issue_peak, "unit": "warp instructions/s", "frac": None,
             "peak_source": f"{n_sm} SMs x 4 schedulers x 1 warp instruction per cycle x {sm_mhz:.0f} MHz "
                            "(median SM clock sampled during the timed steps)", "inst_per_query": None}
    if ctr.get("lts_bytes_per_expansion"):
        lts = ctr["lts_bytes_per_expansion"] * dom[3]
        l2["lts_bytes_per_query"] = lts
        l2["lts_frac"] = lts / (dom[2] / 1e3) / 1e9 / l2_gbs
    if ctr.get("inst_per_expansion"):
        inst = ctr["inst_per_expansion"] * dom[3]
        issue["inst_per_query"] = inst
        issue["achieved"] = inst / (dom[2] / 1e3)
        issue["frac"] = issue["achieved"] / issue_peak
    extra = {}
    sections = set() if args.no_extra else {x.strip() for x in args.sections.split(",") if x.strip()}
    if "small" in sections:
        extra["small"] = small_case(cb, torch, dev)
    if "noalloc" in sections:
        extra["noalloc"] = noalloc_compare(cb, torch, dev, A, B, poses, dist_out, ws_pq, flush)
    if "batched" in sections:
        extra["batched"] = arm_sweep(cb, torch, dev, args.arm_configs)
    if "served" in sections:
        c3 = synth.C3(8)
        models = {"terrain": A, "clutter": cb.BVH(*c3["A"], 24, 8, 8, 16384, device=dev), "sphere5": B,
                  "sphere3": cb.BVH(*synth.C1(1)["B"], 24, 8, 8, 16384, device=dev)}
        for i, link in enumerate(c3["links"]):
            models[f"link{i}"] = cb.BVH(*link, 24, 8, 8, 16384, device=dev)
        robots = {"arm": [f"link{i}" for i in range(6)]}
        extra["served"] = serving(cb, torch, dev, models, robots, c["height"])
        del models
    if "compression" in sections:
        extra["compression"] = compression(cb, torch, dev, c)
    if "refit" in sections:
        extra["refit"] = {"terrain": refit_rate(cb, torch, dev, c["A"][0], c["A"][1], K_DOP, BRANCH, BITS, TREELET,
                                                cb.PACK_TOP_DOWN)}
        c5 = synth.C5(1)
        extra["refit"]["field10m"] = refit_rate(cb, torch, dev, c5["A"][0], c5["A"][1], 18, 4, 8, 16384,
                                                cb.PACK_BOTTOM_UP)
        del c5
    if "scale" in sections:
        torch.cuda.empty_cache()
        extra["scale"] = scale(cb, torch, dev, args.scale_poses, args.scale_pq_poses, args.scale_pair_poses,
                               scale_variants(args))
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, done, secs, cores = oracle_rate(c, args.cpu_sample)
        rate1, done1, secs1, _ = oracle_rate(c, args.cpu_sample, target_s=6.0, threads=1)
        cpu = {"value": rate, "unit": "pose queries/s", "cores": cores, "kind": "oracle",
               "sample": f"first {done} poses of the 10,000-pose set, CD with pairs + PQ, {secs:.1f} s",
               "single_thread": {"value": rate1, "cores": 1,
                                 "sample": f"first {done1} poses, CD with pairs + PQ, {secs1:.1f} s"}}
    sm = sorted(step_ms)
    out = {
        "metric": METRIC, "value": value, "unit": "pose queries/s", "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "terrain 512x512 (524,288 tris) vs displaced level-5 icosphere (20,480 tris), "
                               "24-DOP, branching 8, 8-bit deltas, 16 KB treelets",
                   "poses": n, "step": "CD with sorted pair lists + PQ, every pose",
                   "l2": "flushed (256 MB write, untimed) before every timed step",
                   "parallelism": f"replicas x{world}"},
        "cd_pose_queries_per_s": n / (cd_avg / 1e3),
        "pq_pose_queries_per_s": n / (pq_avg / 1e3),
        "bv_pair_tests_per_s": (bv_cd + bv_pq) * K / (total_ms / 1e3),
        "bv_pair_tests_per_step": bv_cd + bv_pq, "leaf_tests_per_step": leaf_cd + leaf_pq,
        "work_per_step": {"cd": {"bv_tests": bv_cd, "leaf_tests": leaf_cd, "expansions": exp_cd},
                          "pq": {"bv_tests": bv_pq, "leaf_tests": leaf_pq, "expansions": exp_pq}},
        "pairs_per_step": n_pairs,
        "latency_ms": {"p50": sm[len(sm) // 2], "p99": sm[min(len(sm) - 1, int(round(0.99 * (len(sm) - 1))))],
                       "per": f"step of {n} poses (one CD + one PQ launch group)"},
        "roofline": {"bound": "hbm", "kernel": dom[0], "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "peak_source": f"{peak_src} HBM copy bandwidth",
                     "bytes": "algorithmic: BV tests x 34 B + leaf tests x 72 B + poses x 61 B (+ 12 B per pair)",
                     "l2": l2, "issue": issue,
                     "binding": "instruction issue: the hierarchies stay in L2, so neither HBM nor L2 bandwidth is "
                                "the limit; the issue fraction is the one to raise"},
        "kernel_ms": {"traverse_cd": cd_avg, "traverse_pq": pq_avg,
                      "compaction": prof["compaction"][0] / max(1, prof["compaction"][1])},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "pose queries/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
        "gpu_launches": gpu_launches,
    }
    out.update(extra)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
