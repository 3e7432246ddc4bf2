"""Serving loop: many resident sections, render and track requests of uneven
resolution and size, continuously batched on one GPU.

* Sections (colour / opacity / radius in FP16 or FP32) stay resident on the
  device; requests name a section, a camera pose and a resolution bucket.
* A request is either ``render`` (forward: colour, depth, silhouette; the
  colour image is copied to the host) or ``track`` (one tracking iteration:
  forward, Eq. 1 L1 loss against the request's observation, pose backward;
  the 6-vector pose gradient is copied to the host).
* The server has ``n_slots`` slots, each with its own CUDA stream and render
  context whose workspace is sized once for the largest request; the device
  memory budget decides how many slots are backed.  Requests wait in arrival
  order and are admitted into a slot as soon as one frees up; admitted
  requests run concurrently on their slots' streams, so their kernels overlap
  on the GPU (continuous batching at request granularity).
* With ``graphs=True`` the work of each (slot, section, resolution, kind) is
  captured once as a CUDA graph and replayed for every later request of that
  kind; the inputs (pose, observation) live in the graph's fixed buffers.
* Latency is measured from arrival to the result being visible on the host
  (a CUDA event after the device-to-host copy, polled without blocking).
"""

from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import api


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "render" or "track"
    section: int
    pose: np.ndarray          # (3, 4) camera-to-world
    bucket: int               # index into the server's resolutions
    arrival: float = 0.0      # seconds from the start of the run
    done: float = -1.0
    result: torch.Tensor | None = None


class _Work:
    """Fixed buffers and (optionally) a captured graph for one
    (slot, section, bucket, kind)."""

    def __init__(self, slot, server, section, bucket, kind):
        dev = server.device
        W, H = server.resolutions[bucket]
        self.slot, self.kind, self.W, self.H = slot, kind, W, H
        self.K = server.intrinsics[bucket]
        self.sec = server.sections[section]
        self.pose = torch.zeros(12, dtype=torch.float64, device=dev)
        self.rgb = torch.empty(3, H, W, device=dev)
        self.depth = torch.empty(H, W, device=dev)
        self.sil = torch.empty(H, W, device=dev)
        self.d_twist = torch.zeros(6, dtype=torch.float64, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.g_rgb = torch.zeros(3, H, W, device=dev)
        self.g_depth = torch.zeros(H, W, device=dev)
        self.obs_rgb, self.obs_depth = server.observations[bucket]
        self.host = torch.empty((3, H, W) if kind == "render" else (6,),
                                dtype=torch.float32 if kind == "render" else torch.float64
                                ).pin_memory()
        self.graph = None

    def run(self):
        R = self.slot.renderer
        R.render([self.sec], self.pose, self.K, self.W, self.H, self.rgb, self.depth, self.sil)
        if self.kind == "track":   # Eq. 1 masked L1 (alpha 0.5, beta 0.025), pose gradient
            R.masked_l1(self.rgb, self.depth, self.sil, self.obs_rgb, self.obs_depth, 0.5, 0.025,
                        sil_min=0.99, rgb_needs_depth=True, d_rgb=self.g_rgb,
                        d_depth=self.g_depth, loss=self.loss)
            self.d_twist.zero_()
            R.backward(self.g_rgb, self.g_depth, None, pose_grad=True, d_twist=self.d_twist)


class _Slot:
    def __init__(self, server, index):
        self.index = index
        self.stream = torch.cuda.Stream(device=server.device)
        self.renderer = api.Renderer()
        self.works = {}
        self.request = None
        self.event = None
        self.reserved = (0, 0, 0)    # Gaussians, pixels, instances
        self.work = None


class Server:
    def __init__(self, sections, resolutions, observations, n_slots: int = 4,
                 graphs: bool = True, memory_budget: int | None = None, device="cuda"):
        """sections: list of api.Section (resident); resolutions: list of
        (W, H); observations: per bucket (rgb (3,H,W), depth (H,W)) device
        tensors used as the tracking target."""
        from . import synthetic as syn
        self.device = torch.device(device)
        self.sections = sections
        self.resolutions = [tuple(r) for r in resolutions]
        self.intrinsics = [syn.scaled_intrinsics(W, H).astuple() for W, H in self.resolutions]
        self.observations = observations
        self.graphs = graphs
        self.slots = [_Slot(self, i) for i in range(n_slots)]
        free, total = torch.cuda.mem_get_info(self.device)
        self.memory_budget = memory_budget if memory_budget is not None else int(free * 0.8)
        self.max_instances_per_gaussian = 3.0

    # -- memory ---------------------------------------------------------------
    # Every slot's workspace is sized once, before any graph is captured, for
    # the largest request it may serve (captured graphs hold the workspace's
    # addresses, so it must never move afterwards).  The memory budget decides
    # how many slots can be backed: slots beyond it are not used.
    def _need(self, req):
        n = self.sections[req.section].n
        return n, int(self.max_instances_per_gaussian * n) + 65536

    def _size_slots(self, requests):
        n_max = max(self._need(r)[0] for r in requests)
        i_max = max(self._need(r)[1] for r in requests)
        b_max = max(range(len(self.resolutions)),
                    key=lambda b: self.resolutions[b][0] * self.resolutions[b][1])
        W, H = self.resolutions[b_max]
        per_slot = api.L.lib().vt_workspace_bytes(n_max, W, H, i_max) + 8 * 256 * W * H
        usable = max(1, min(len(self.slots), self.memory_budget // max(per_slot, 1)))
        self.slots = self.slots[:usable]
        for slot in self.slots:
            with torch.cuda.stream(slot.stream):
                slot.renderer.reserve(n_max, W, H, i_max)
                # a render at the largest size allocates the per-pixel lists
                work = _Work(slot, self, max(range(len(self.sections)),
                                             key=lambda s: self.sections[s].n), b_max, "render")
                work.run()
            slot.reserved = (n_max, W * H, i_max)
        torch.cuda.synchronize()
        self.per_slot_bytes = per_slot

    def _fits(self, slot, req):
        n, inst = self._need(req)
        W, H = self.resolutions[req.bucket]
        g, p, i = slot.reserved
        return n <= g and W * H <= p and inst <= i

    # -- execution --------------------------------------------------------------
    def _launch(self, slot, req):
        key = (req.section, req.bucket, req.kind)
        work = slot.works.get(key)
        with torch.cuda.stream(slot.stream):
            if work is None:
                if not self._fits(slot, req):
                    raise RuntimeError("request larger than the slot workspaces sized in warm()")
                work = _Work(slot, self, req.section, req.bucket, req.kind)
                slot.works[key] = work
                if self.graphs:
                    work.pose.copy_(api.pose12(req.pose, self.device))
                    work.run()                      # warm-up outside the capture
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=slot.stream):
                        work.run()
                    work.graph = g
            work.pose.copy_(api.pose12(req.pose, self.device), non_blocking=True)
            if work.graph is not None:
                work.graph.replay()
            else:
                work.run()
            src = work.rgb if req.kind == "render" else work.d_twist
            work.host.copy_(src, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.request, slot.event, slot.work = req, ev, work

    def warm(self, requests):
        """Size the slot workspaces and capture the graphs for every
        (slot, section, bucket, kind) the requests use."""
        self._size_slots(requests)
        keys = sorted({(r.section, r.bucket, r.kind, tuple(r.pose.reshape(-1))) for r in requests},
                      key=lambda k: k[:3])
        seen = set()
        for s, b, k, p in keys:
            if (s, b, k) in seen:
                continue
            seen.add((s, b, k))
            req = Request(-1, k, s, np.asarray(p).reshape(3, 4), b)
            for slot in self.slots:
                self._launch(slot, req)
                slot.event.synchronize()
                slot.request = None
        torch.cuda.synchronize()

    def run(self, requests, timeout: float = 600.0):
        """Serve ``requests`` (sorted by arrival time, in seconds from now).
        Returns the requests with ``done`` set and their results."""
        queue = collections.deque()
        pending = list(sorted(requests, key=lambda r: r.arrival))
        nxt = 0
        finished = []
        t0 = time.perf_counter()
        busy = 0
        while len(finished) < len(requests):
            now = time.perf_counter() - t0
            if now > timeout:
                raise TimeoutError("serving run exceeded its time limit")
            while nxt < len(pending) and pending[nxt].arrival <= now:
                queue.append(pending[nxt])
                nxt += 1
            for slot in self.slots:     # completions (non-blocking)
                if slot.request is not None and slot.event.query():
                    r = slot.request
                    r.done = time.perf_counter() - t0
                    r.result = slot.work.host.clone()
                    finished.append(r)
                    slot.request = None
                    busy -= 1
            for slot in self.slots:     # admissions in arrival order
                if not queue:
                    break
                if slot.request is None:
                    self._launch(slot, queue.popleft())
                    busy += 1
            if busy == len(self.slots) or (not queue and nxt < len(pending)):
                time.sleep(20e-6)
        return finished


def latency_summary(done, resolutions):
    lat = np.array([(r.done - r.arrival) * 1e3 for r in done])
    span = max(r.done for r in done) - min(r.arrival for r in done)
    pix = sum(resolutions[r.bucket][0] * resolutions[r.bucket][1] for r in done)
    return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "mpix_s": pix / span / 1e6, "span_s": span}


def poisson_requests(n, rate_per_s, n_sections, n_buckets, poses, seed=3, track_frac=0.7):
    """Seeded request stream: Poisson arrivals, 70% track / 30% render,
    uniform section and resolution; poses drawn from ``poses``."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    out = []
    for i in range(n):
        kind = "track" if rng.random() < track_frac else "render"
        s = int(rng.integers(n_sections))
        b = int(rng.integers(n_buckets))
        out.append(Request(i, kind, s, poses[s][int(rng.integers(len(poses[s])))], b,
                           arrival=float(t[i])))
    return out
