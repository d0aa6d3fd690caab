"""Request loop with continuous batching for collision and distance queries.

Planners submit requests -- (environment, robot, kind, poses) -- from any thread and get a
future.  A serving thread keeps every hierarchy resident on the device and admits waiting
requests into batches as stream slots and device memory free up: requests that arrive while
others are on the GPU join the next batch, each batch runs as one set of persistent launches
(cbvh_batch_launch) on its own stream, and up to ``slots`` batches overlap on the device.
Admission is by a device-memory budget: a batch takes requests in arrival order while the
memory it needs (poses, outputs, workspace) fits in what the budget has left.  Per-request
latency (submit to result) is recorded for p50 / p99.

A robot is either one hierarchy or a chain of links (``robots``: name -> link model names);
a request for a chain carries one pose per link and configuration, runs as one batch item
per link, and resolves to "any link collides" or "smallest distance over the links".  The
links of a collision request form one configuration set of the batch, so a configuration
stops at its first colliding link; the links of a distance request share the
configuration's best distance, with which each link's branch and bound prunes.

A batch whose device status reports an error (for example a node-pair stack or a wait that
ran out) does not fail its requests at once: each is retried once on the plain path, one
query per model pair on the serving thread, and fails only if that fails too.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import Batch, _torch, collide, distance


def combine(kind: str, parts: list) -> np.ndarray:
    """One configuration's result from its links' results: a chain collides when any link
    does (largest flag), and its distance is the smallest over the links."""
    if len(parts) == 1:
        return np.array(parts[0], copy=True)
    return np.maximum.reduce(parts) if kind == "collide" else np.minimum.reduce(parts)


class Request:
    __slots__ = ("env", "robot", "kind", "poses", "early_exit", "future", "t_submit", "t_done")

    def __init__(self, env, robot, kind, poses, early_exit):
        self.env, self.robot, self.kind, self.poses, self.early_exit = env, robot, kind, poses, early_exit
        self.future = Future()
        self.t_submit = time.perf_counter()
        self.t_done = None


class Server:
    """models: name -> attached BVH.  robots: name -> list of link model names (chains such as
    an arm); a plain model name also serves as a robot.  mem_budget: device bytes that batches
    in flight may use.  max_poses: cap on the link poses of one batch."""

    def __init__(self, models: dict, mem_budget: int = 1 << 30, slots: int = 4, max_poses: int = 1 << 16,
                 device="cuda", robots: dict | None = None):
        torch = _torch()
        self.models = models
        self.robots = dict(robots or {})
        self.mem_budget = int(mem_budget)
        self.max_poses = int(max_poses)
        dev = torch.device(device)
        self.device = torch.device("cuda", dev.index if dev.index is not None else torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.busy = [None] * slots  # per slot: (event, requests, host outputs, bytes, batch)
        self.used = 0
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.latencies = []
        self.batches = 0
        self.retries = 0
        self.running = True
        self.error = None
        self.thread = threading.Thread(target=self._loop, name="cbvh-serve", daemon=True)
        self.thread.start()

    # ---------------------------------------------------------------- client side
    def links(self, robot: str) -> list:
        return list(self.robots[robot]) if robot in self.robots else [robot]

    def submit(self, env: str, robot: str, kind: str, poses: np.ndarray, early_exit: bool = False) -> Future:
        """Queue a request; the future resolves to uint8 hit flags ('collide') or float32
        distances ('distance'), one per configuration.  poses: (n, 12) for a single model,
        (n, L, 12) for a chain of L links.  Collision requests return flags only, so every
        configuration stops at its first intersecting pair whatever ``early_exit`` says."""
        if kind not in ("collide", "distance"):
            raise ValueError("kind must be 'collide' or 'distance'")
        if env not in self.models:
            raise KeyError("unknown model")
        links = self.links(robot)
        if any(l not in self.models for l in links):
            raise KeyError("unknown model")
        L = len(links)
        poses = np.ascontiguousarray(poses, dtype=np.float32)
        poses = poses.reshape(-1, L, 12) if L > 1 else poses.reshape(-1, 12)
        r = Request(env, robot, kind, poses, early_exit)
        with self.cv:
            if not self.running:
                raise RuntimeError("server is closed")
            self.pending.append(r)
            self.cv.notify()
        return r.future

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify()
        self.thread.join()

    def stats(self):
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        return dict(requests=len(self.latencies), batches=self.batches, retries=self.retries,
                    p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3))

    # ---------------------------------------------------------------- serving thread
    @staticmethod
    def _bytes(n_poses: int) -> int:
        # admission estimate of a batch: poses + outputs + the batch workspace: two task buffers
        # of 16-byte entries and their ready flags (at least 2^22 entries, else 512 per pose) +
        # stacks and counters (the launch then charges the plan's exact workspace)
        return n_poses * (48 + 4 + 1) + max(1 << 22, 512 * n_poses) * (2 * 16 + 4) + (96 << 20)

    @staticmethod
    def _link_poses(r) -> int:
        return r.poses.shape[0] * (r.poses.shape[1] if r.poses.ndim == 3 else 1)

    def _plain(self, r) -> np.ndarray:
        """One request on the plain path: one query per model pair, synchronously."""
        torch = _torch()
        links = self.links(r.robot)
        parts = []
        for i, name in enumerate(links):
            P = torch.as_tensor(np.ascontiguousarray(r.poses[:, i] if len(links) > 1 else r.poses),
                                device=self.device)
            if r.kind == "collide":
                parts.append(collide(self.models[r.env], self.models[name], P, pairs=False,
                                     early_exit=r.early_exit).hit.cpu().numpy())
            else:
                parts.append(distance(self.models[r.env], self.models[name], P).cpu().numpy())
        return combine(r.kind, parts)

    def _complete(self, slot):
        ev, reqs, outs, nbytes, batch = self.busy[slot]
        ev.synchronize()
        code = int(batch.status.item())
        self.busy[slot] = None
        self.used -= nbytes
        for r, parts in zip(reqs, outs):
            if code != 0:  # retried once on the plain path
                self.retries += 1
                try:
                    res = self._plain(r)
                except Exception as e:  # noqa: BLE001 -- reported through the future
                    res = e
            else:
                res = combine(r.kind, [o.numpy() for o in parts])
            r.t_done = time.perf_counter()
            self.latencies.append(r.t_done - r.t_submit)
            if isinstance(res, Exception):
                r.future.set_exception(res)
            else:
                r.future.set_result(res)

    def _admit(self):
        """Requests for the next batch: in arrival order, while memory and size allow."""
        take, n, need = [], 0, 0
        while self.pending:
            r = self.pending[0]
            rn = self._link_poses(r)
            b = self._bytes(n + rn)
            if take and (n + rn > self.max_poses or self.used + b > self.mem_budget):
                break
            if not take and self.used + b > self.mem_budget and any(self.busy):
                break  # wait for memory to come back
            take.append(self.pending.popleft())
            n += rn
            need = b
        return take, need

    def _launch(self, slot, reqs, est_bytes):
        """Launch one batch of the admitted requests on the slot's stream (est_bytes: the
        admission estimate; the slot is charged the batch's exact bytes)."""
        torch = _torch()
        stream = self.streams[slot]
        with torch.cuda.stream(stream):
            # one part per (request, link): its poses are contiguous in one pinned buffer
            parts = []
            for r in reqs:
                links = self.links(r.robot)
                for i, name in enumerate(links):
                    parts.append((r, name, r.poses[:, i] if len(links) > 1 else r.poses))
            n_total = sum(len(P) for _, _, P in parts)
            host = torch.empty((max(1, n_total), 12), dtype=torch.float32, pin_memory=True)
            o = 0
            for _, _, P in parts:
                host[o:o + len(P)] = torch.from_numpy(np.ascontiguousarray(P))
                o += len(P)
            dev = host.to(self.device, non_blocking=True)
            items, o = [], 0
            for r, name, P in parts:
                n = len(P)
                chain = len(self.links(r.robot)) > 1
                items.append(dict(A=self.models[r.env], B=self.models[name], kind=r.kind,
                                  poses=dev[o:o + n], early_exit=r.early_exit, set=id(r) if chain else None))
                o += n
            batch = Batch(items, device=self.device)
            batch.launch(stream)
            outs, k = [], 0
            for r in reqs:
                nl = len(self.links(r.robot))
                if nl > 1:  # the configuration set's answer
                    srcs = [batch.any_hit[id(r)] if r.kind == "collide" else batch.min_dist[id(r)]]
                else:
                    srcs = batch.outputs[k:k + nl]
                k += nl
                mine = []
                for out in srcs:
                    h = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
                    h.copy_(out, non_blocking=True)
                    mine.append(h)
                outs.append(mine)
            ev = torch.cuda.Event()
            ev.record(stream)
        # charge what the batch holds: its poses and outputs and the workspace its plan asked
        # for (task buffers sized by its pose count, one node-pair stack per resident warp);
        # admission used the estimate, which leaves out the stacks' dependence on the depths
        nbytes = int(dev.numel()) * 4 + sum(int(o.numel()) * o.element_size() for o in batch.outputs) + \
            int(batch.workspace.numel())
        self.busy[slot] = (ev, reqs, outs, nbytes, batch)
        self.used += nbytes
        self.batches += 1

    def _loop(self):
        try:
            self._serve()
        except BaseException as e:  # the loop itself failed: fail everything still queued
            self.error = e
            with self.cv:
                self.running = False
                waiting = list(self.pending)
                self.pending.clear()
            for r in waiting:
                r.future.set_exception(e)
            for b in self.busy:
                if b is not None:
                    for r in b[1]:
                        if not r.future.done():
                            r.future.set_exception(e)

    def _serve(self):
        torch = _torch()
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while self.running and not self.pending and not any(self.busy):
                    self.cv.wait(0.01)
                if not self.running and not self.pending and not any(self.busy):
                    return
            try:
                for s, b in enumerate(self.busy):
                    if b is not None and b[0].query():
                        self._complete(s)
                free = [s for s, b in enumerate(self.busy) if b is None]
                if free:
                    with self.cv:
                        reqs, need = self._admit()
                    if reqs:
                        try:
                            self._launch(free[0], reqs, need)
                        except Exception as e:  # these requests never reached the device
                            self.error = e
                            for r in reqs:
                                r.future.set_exception(e)
                        continue
                if any(self.busy):
                    time.sleep(20e-6)
            except Exception as e:  # fail the affected requests, keep serving
                self.error = e
                for s, b in enumerate(self.busy):
                    if b is not None:
                        for r in b[1]:
                            if not r.future.done():
                                r.future.set_exception(e)
                        self.used -= b[3]
                        self.busy[s] = None
